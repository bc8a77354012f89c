"""ctypes binding of libstag.so: the functions of include/stag.h under the same names.

Argument marshalling only -- every step of the computation runs in the CUDA
library.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays, C
contiguous, dtype complex128 (or float64 with a trailing (re, im) axis).  A
missing library raises; there is no CPU fallback.

Layouts (see include/stag.h): links (4, V, 3, 3) complex128 with V in
lexicographic order (x fastest); checkerboard vectors (V/2, 3) complex128.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

STAG_OK = 0
STAG_NOT_CONVERGED = 1
STAG_ERR_ARG = -1
STAG_ERR_CUDA = -2
STAG_ERR_OOM = -3
STAG_ERR_NOT_SU3 = -4
STAG_ERR_BREAKDOWN = -5
STAG_ERR_TIMEOUT = -6
STAG_ERR_STATE = -7

STAG_FP64, STAG_FP32, STAG_FP16, STAG_BF16 = 0, 1, 2, 3
STAG_ROUND_OUTPUT = 0x100
STAG_HALF_VECTORS = 0x200
STAG_VEC_FP16 = 0x400
STAG_VEC_BF16 = 0x800
STAG_ANTIPERIODIC_T = 1
STAG_RECON12 = 2

PRECISIONS = {"fp64": STAG_FP64, "fp32": STAG_FP32, "fp16": STAG_FP16, "bf16": STAG_BF16}

_lib = None
_lock = threading.Lock()


class SolveDesc(ctypes.Structure):
    """struct stag_solve_desc: one lattice of a ragged batch."""
    _fields_ = [("ctx", ctypes.c_void_p), ("src", ctypes.POINTER(ctypes.c_void_p)), ("nrhs", ctypes.c_int),
                ("masses", ctypes.c_void_p), ("nmass", ctypes.c_int), ("x", ctypes.POINTER(ctypes.c_void_p)),
                ("iters", ctypes.c_void_p), ("true_res", ctypes.c_void_p)]


class StagError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load():
    """Load libstag.so (built by __graft_entry__.build() / paper_1511_00088_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libstag.so not built ({path}); run paper_1511_00088_gb300.build.build()")
        lib = ctypes.CDLL(path)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        PP = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "stag_create": (I, [ctypes.POINTER(ctypes.c_int), I, P, PP]),
            "stag_destroy": (I, [P]),
            "stag_links_upload": (I, [P, P]),
            "stag_dslash_oe": (I, [P, I, P, P]),
            "stag_dslash_eo": (I, [P, I, P, P]),
            "stag_mdagm": (I, [P, I, D, P, P]),
            "stag_cg_solve": (I, [P, PP, I, P, I, D, I, I, PP, P, P]),
            "stag_solve_full": (I, [P, PP, I, P, I, D, I, I, PP, P, P]),
            "stag_cg_solve_multishift": (I, [P, PP, I, P, I, D, I, I, PP, P, P]),
            "stag_hyp_smear": (I, [P, P, P, P]),
            "stag_npr_contract": (I, [P, P, P, P, P, P, P, P]),
            "stag_time_dslash": (I, [P, I, I, P, P]),
            "stag_time_cg_kernel": (I, [P, I, I, I, P, P]),
            "stag_solve_counters": (I, [P, P, P]),
            "stag_solve_form": (I, [P, P]),
            "stag_solve_stats": (I, [P, I, P, P, P]),
            "stag_mdagm_dot_noalloc": (I, [P, D, P, P, P, P]),
            "stag_force": (I, [P, P, P, P]),
            "stag_action": (I, [P, D, P, P, P]),
            "stag_action_backward": (I, [P, P, D, P, P]),
            "stag_cg_solve_ragged": (I, [ctypes.POINTER(SolveDesc), I, D, I, I]),
            "stag_last_error": (ctypes.c_char_p, [P]),
            "stag_status_string": (ctypes.c_char_p, [I]),
            "stag_abi_version": (I, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def status_name(status: int) -> str:
    try:
        return load().stag_status_string(int(status)).decode()
    except Exception:  # noqa: BLE001 - naming a status must not raise
        return f"status {status}"


def _ptr(a):
    """Raw pointer of a contiguous complex128/float64 torch tensor or numpy array."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            if a.dtype not in (torch.complex128, torch.float64):
                raise ValueError("tensor must be complex128 or float64")
            return a.data_ptr()
    except ImportError:  # pragma: no cover
        pass
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C contiguous")
        if a.dtype not in (np.complex128, np.float64):
            raise ValueError("array must be complex128 or float64")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


# ---------------------------------------------------------------------------
# the C functions under their own names (return the status code)
# ---------------------------------------------------------------------------
def stag_create(dims, flags=STAG_ANTIPERIODIC_T, cuda_stream=None):
    lib = load()
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    h = ctypes.c_void_p()
    st = lib.stag_create(d, int(flags), ctypes.c_void_p(cuda_stream or 0), ctypes.byref(h))
    return st, h


def stag_destroy(ctx):
    return load().stag_destroy(ctx)


def stag_links_upload(ctx, links):
    return load().stag_links_upload(ctx, _ptr(links))


def stag_dslash_oe(ctx, precision, in_even, out_odd):
    return load().stag_dslash_oe(ctx, int(precision), _ptr(in_even), _ptr(out_odd))


def stag_dslash_eo(ctx, precision, in_odd, out_even):
    return load().stag_dslash_eo(ctx, int(precision), _ptr(in_odd), _ptr(out_even))


def stag_mdagm(ctx, precision, mass, in_even, out_even):
    return load().stag_mdagm(ctx, int(precision), float(mass), _ptr(in_even), _ptr(out_even))


def stag_cg_solve(ctx, srcs, masses, tol, maxiter, precision, xs, iters=None, true_res=None):
    """srcs: list of nrhs vectors; xs: list of nrhs*nmass output vectors (slot r*nmass+k)."""
    lib = load()
    nrhs, nmass = len(srcs), len(masses)
    sp = (ctypes.c_void_p * nrhs)(*[_ptr(s) for s in srcs])
    xp = (ctypes.c_void_p * (nrhs * nmass))(*[_ptr(x) for x in xs])
    m = np.ascontiguousarray(np.asarray(masses, dtype=np.float64))
    it = np.zeros(nrhs * nmass, np.int32) if iters is None else iters
    tr = np.zeros(nrhs * nmass, np.float64) if true_res is None else true_res
    st = lib.stag_cg_solve(ctx, sp, nrhs, m.ctypes.data, nmass, float(tol), int(maxiter),
                           int(precision), xp, it.ctypes.data, tr.ctypes.data)
    return st, it, tr


def stag_npr_contract(ctx, spin_taste, chibar1, chi2, chibar3, chi4, O_hyp=None, O_sum=None):
    """NPR contraction; spin_taste = (S1, F1, S2, F2); O_sum a complex128 array of one element."""
    st = (ctypes.c_int * 4)(*[int(v) for v in spin_taste])
    return load().stag_npr_contract(ctx, st, _ptr(chibar1), _ptr(chi2), _ptr(chibar3), _ptr(chi4),
                                    None if O_hyp is None else _ptr(O_hyp), None if O_sum is None else _ptr(O_sum))


def stag_hyp_smear(ctx, alpha, links_in, links_out):
    """HYP smearing; alpha None = (0.75, 0.6, 0.3)."""
    a = None if alpha is None else np.ascontiguousarray(np.asarray(alpha, dtype=np.float64))
    return load().stag_hyp_smear(ctx, None if a is None else a.ctypes.data, _ptr(links_in), _ptr(links_out))


def stag_cg_solve_multishift(ctx, srcs, masses, tol, maxiter, precision, xs, iters=None, true_res=None):
    """As stag_cg_solve, by a multi-shift CG plus per-mass refinement."""
    lib = load()
    nrhs, nmass = len(srcs), len(masses)
    sp = (ctypes.c_void_p * nrhs)(*[_ptr(s) for s in srcs])
    xp = (ctypes.c_void_p * (nrhs * nmass))(*[_ptr(x) for x in xs])
    m = np.ascontiguousarray(np.asarray(masses, dtype=np.float64))
    it = np.zeros(nrhs * nmass, np.int32) if iters is None else iters
    tr = np.zeros(nrhs * nmass, np.float64) if true_res is None else true_res
    st = lib.stag_cg_solve_multishift(ctx, sp, nrhs, m.ctypes.data, nmass, float(tol), int(maxiter),
                                      int(precision), xp, it.ctypes.data, tr.ctypes.data)
    return st, it, tr


def stag_solve_full(ctx, srcs, masses, tol, maxiter, precision, xs, iters=None, true_res=None):
    """Full-lattice M x = b: srcs list of nrhs (V, 3) vectors; xs nrhs*nmass (V, 3) outputs."""
    lib = load()
    nrhs, nmass = len(srcs), len(masses)
    sp = (ctypes.c_void_p * nrhs)(*[_ptr(s) for s in srcs])
    xp = (ctypes.c_void_p * (nrhs * nmass))(*[_ptr(x) for x in xs])
    m = np.ascontiguousarray(np.asarray(masses, dtype=np.float64))
    it = np.zeros(nrhs * nmass, np.int32) if iters is None else iters
    tr = np.zeros(nrhs * nmass, np.float64) if true_res is None else true_res
    st = lib.stag_solve_full(ctx, sp, nrhs, m.ctypes.data, nmass, float(tol), int(maxiter),
                             int(precision), xp, it.ctypes.data, tr.ctypes.data)
    return st, it, tr


def stag_time_dslash(ctx, precision, nlaunch):
    ms = ctypes.c_double(0.0)
    by = ctypes.c_double(0.0)
    st = load().stag_time_dslash(ctx, int(precision), int(nlaunch), ctypes.byref(ms), ctypes.byref(by))
    return st, ms.value, by.value


def stag_solve_counters(ctx):
    passes = ctypes.c_int(0)
    ups = ctypes.c_int(0)
    st = load().stag_solve_counters(ctx, ctypes.byref(passes), ctypes.byref(ups))
    return st, passes.value, ups.value


def stag_solve_form(ctx):
    out = (ctypes.c_int * 8)()
    st = load().stag_solve_form(ctx, out)
    return st, list(out)


def stag_time_cg_kernel(ctx, precision, kernel, nlaunch):
    ms = ctypes.c_double(0.0)
    by = ctypes.c_double(0.0)
    st = load().stag_time_cg_kernel(ctx, int(precision), int(kernel), int(nlaunch), ctypes.byref(ms),
                                    ctypes.byref(by))
    return st, ms.value, by.value


def stag_solve_stats(ctx, sys):
    it = ctypes.c_int(0)
    nu = ctypes.c_int(0)
    tr = ctypes.c_double(0.0)
    st = load().stag_solve_stats(ctx, int(sys), ctypes.byref(it), ctypes.byref(nu), ctypes.byref(tr))
    return st, it.value, nu.value, tr.value


def stag_mdagm_dot_noalloc(ctx, mass, in_even, tmp_odd, out_even, dot=None):
    """No-allocation M^dag M with FP64 <in, out>; every argument a CUDA tensor."""
    return load().stag_mdagm_dot_noalloc(ctx, float(mass), _ptr(in_even), _ptr(tmp_odd), _ptr(out_even),
                                         None if dot is None else _ptr(dot))


def stag_cg_solve_ragged(entries, tol, maxiter, precision):
    """entries: list of (ctx, srcs, masses, xs).  Returns (status, [iters], [true_res])."""
    n = len(entries)
    descs = (SolveDesc * n)()
    keep = []
    its, trs = [], []
    for i, (ctx, srcs, masses, xs) in enumerate(entries):
        sp = (ctypes.c_void_p * len(srcs))(*[_ptr(a) for a in srcs])
        xp = (ctypes.c_void_p * len(xs))(*[_ptr(a) for a in xs])
        m = np.ascontiguousarray(np.asarray(masses, dtype=np.float64))
        it = np.zeros(len(xs), np.int32)
        tr = np.zeros(len(xs), np.float64)
        keep += [sp, xp, m]
        its.append(it)
        trs.append(tr)
        descs[i] = SolveDesc(ctx, ctypes.cast(sp, ctypes.POINTER(ctypes.c_void_p)), len(srcs), m.ctypes.data,
                             len(masses), ctypes.cast(xp, ctypes.POINTER(ctypes.c_void_p)), it.ctypes.data,
                             tr.ctypes.data)
    st = load().stag_cg_solve_ragged(descs, n, float(tol), int(maxiter), int(precision))
    return st, its, trs


def stag_force(ctx, x_even, grad_links=None, lie_force=None):
    return load().stag_force(ctx, _ptr(x_even), None if grad_links is None else _ptr(grad_links),
                             None if lie_force is None else _ptr(lie_force))


def stag_action(ctx, mass, phi_even, x_even):
    """(status, S) with S = 2 Re<phi, x> - Re<x, A x> (double-word FP64 sums on the GPU)."""
    S = ctypes.c_double(0.0)
    st = load().stag_action(ctx, float(mass), _ptr(phi_even), _ptr(x_even), ctypes.byref(S))
    return st, S.value


def stag_action_backward(ctx, x_even, gS, grad_links=None, grad_phi=None):
    return load().stag_action_backward(ctx, _ptr(x_even), float(gS),
                                       None if grad_links is None else _ptr(grad_links),
                                       None if grad_phi is None else _ptr(grad_phi))


def stag_last_error(ctx):
    return load().stag_last_error(ctx).decode()


def stag_status_string(status):
    return load().stag_status_string(int(status)).decode()


def stag_abi_version():
    return load().stag_abi_version()


# ---------------------------------------------------------------------------
# a small object wrapper that raises on errors
# ---------------------------------------------------------------------------
def cg_solve_ragged(batch, tol=1e-10, maxiter=100000, precision=STAG_FP32, allow_not_converged=False):
    """Solve several lattices in one graph launch.  batch: list of
    (Context, srcs, masses).  Returns (list of xs per lattice, status, iters, true_res)."""
    entries, outs = [], []
    for ctx, srcs, masses in batch:
        xs = [ctx._like(srcs[r]) for r in range(len(srcs)) for _ in masses]
        outs.append(xs)
        entries.append((ctx.h, srcs, masses, xs))
    st, its, trs = stag_cg_solve_ragged(entries, tol, maxiter, precision)
    ok = (STAG_OK, STAG_NOT_CONVERGED) if allow_not_converged else (STAG_OK,)
    if st not in ok:
        raise StagError(st, stag_last_error(batch[0][0].h))
    return outs, st, its, trs


class Context:
    """One lattice on the current CUDA device (see stag_create)."""

    def __init__(self, dims, antiperiodic=True, recon12=False, stream=None):
        flags = (STAG_ANTIPERIODIC_T if antiperiodic else 0) | (STAG_RECON12 if recon12 else 0)
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:  # noqa: BLE001
                stream = 0
        st, h = stag_create(dims, flags, stream)
        if st != STAG_OK:
            raise StagError(st, "stag_create failed")
        self.h = h
        self.dims = tuple(int(v) for v in dims)
        self.V = int(np.prod(self.dims))
        self.Ve = self.V // 2

    def _check(self, st, ok=(STAG_OK,)):
        if st not in ok:
            raise StagError(st, stag_last_error(self.h))
        return st

    def close(self):
        if getattr(self, "h", None):
            stag_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def links_upload(self, links):
        return self._check(stag_links_upload(self.h, links))

    def _like(self, a):
        try:
            import torch
            if isinstance(a, torch.Tensor):
                return torch.empty((self.Ve, 3), dtype=torch.complex128, device=a.device)
        except ImportError:  # pragma: no cover
            pass
        return np.empty((self.Ve, 3), np.complex128)

    def dslash_oe(self, x, precision=STAG_FP64, out=None):
        out = self._like(x) if out is None else out
        self._check(stag_dslash_oe(self.h, precision, x, out))
        return out

    def dslash_eo(self, x, precision=STAG_FP64, out=None):
        out = self._like(x) if out is None else out
        self._check(stag_dslash_eo(self.h, precision, x, out))
        return out

    def mdagm(self, x, mass, precision=STAG_FP64, out=None):
        out = self._like(x) if out is None else out
        self._check(stag_mdagm(self.h, precision, mass, x, out))
        return out

    def cg_solve(self, srcs, masses, tol=1e-10, maxiter=100000, precision=STAG_FP32, xs=None,
                 allow_not_converged=False):
        """Returns (xs, status, iters, true_res); xs[r * nmass + k] solves source r, mass k."""
        if xs is None:
            xs = [self._like(srcs[r]) for r in range(len(srcs)) for _ in masses]
        st, it, tr = stag_cg_solve(self.h, srcs, masses, tol, maxiter, precision, xs)
        ok = (STAG_OK, STAG_NOT_CONVERGED) if allow_not_converged else (STAG_OK,)
        self._check(st, ok)
        return xs, st, it, tr

    def npr_contract(self, spin_taste, chibar1, chi2, chibar3, chi4):
        """(O per hypercube (V/16,) complex128, their sum) of the one-colour-trace
        four-fermion contraction on the uploaded links."""
        try:
            import torch
            dev = chibar1.device if isinstance(chibar1, torch.Tensor) else None
        except ImportError:  # pragma: no cover
            dev = None
        if dev is not None:
            import torch
            O = torch.empty(self.V // 16, dtype=torch.complex128, device=dev)
        else:
            O = np.empty(self.V // 16, np.complex128)
        tot = np.zeros(1, np.complex128)
        self._check(stag_npr_contract(self.h, spin_taste, chibar1, chi2, chibar3, chi4, O, tot))
        return O, complex(tot[0])

    def hyp_smear(self, links, alpha=None, out=None):
        """HYP-smeared copy of links (4, V, 3, 3) complex128 (out may be links)."""
        if out is None:
            try:
                import torch
                out = torch.empty_like(links) if isinstance(links, torch.Tensor) else np.empty_like(links)
            except ImportError:  # pragma: no cover
                out = np.empty_like(links)
        self._check(stag_hyp_smear(self.h, alpha, links, out))
        return out

    def cg_solve_multishift(self, srcs, masses, tol=1e-10, maxiter=100000, precision=STAG_FP32, xs=None,
                            allow_not_converged=False):
        """Multi-shift CG; returns (xs, status, iters, true_res) like cg_solve."""
        if xs is None:
            xs = [self._like(srcs[r]) for r in range(len(srcs)) for _ in masses]
        st, it, tr = stag_cg_solve_multishift(self.h, srcs, masses, tol, maxiter, precision, xs)
        ok = (STAG_OK, STAG_NOT_CONVERGED) if allow_not_converged else (STAG_OK,)
        self._check(st, ok)
        return xs, st, it, tr

    def solve_full(self, srcs, masses, tol=1e-10, maxiter=100000, precision=STAG_FP32, xs=None,
                   allow_not_converged=False):
        """Full-lattice M x = b (M = 2m + D); srcs and xs are (V, 3) vectors in
        lexicographic site order.  Returns (xs, status, iters, true_res)."""
        if xs is None:
            xs = []
            for r in range(len(srcs)):
                for _ in masses:
                    try:
                        import torch
                        if isinstance(srcs[r], torch.Tensor):
                            xs.append(torch.empty((self.V, 3), dtype=torch.complex128, device=srcs[r].device))
                            continue
                    except ImportError:  # pragma: no cover
                        pass
                    xs.append(np.empty((self.V, 3), np.complex128))
        st, it, tr = stag_solve_full(self.h, srcs, masses, tol, maxiter, precision, xs)
        ok = (STAG_OK, STAG_NOT_CONVERGED) if allow_not_converged else (STAG_OK,)
        self._check(st, ok)
        return xs, st, it, tr

    def solve_stats(self, sys=0):
        """(iters, reliable_updates, true_res) of system `sys` of the last solve."""
        st, it, nu, tr = stag_solve_stats(self.h, sys)
        self._check(st)
        return it, nu, tr

    def force(self, x_even, grad=True, lie=False):
        """(grad_links (4, V, 3, 3) complex128 or None, lie (4, V, 8) float64 or None)
        for S = phi^dag A^{-1} phi at the solution x_even = A^{-1} phi."""
        try:
            import torch
            dev = x_even.device if isinstance(x_even, torch.Tensor) else None
        except ImportError:  # pragma: no cover
            dev = None
        if dev is not None:
            import torch
            g = torch.empty((4, self.V, 3, 3), dtype=torch.complex128, device=dev) if grad else None
            f = torch.empty((4, self.V, 8), dtype=torch.float64, device=dev) if lie else None
        else:
            g = np.empty((4, self.V, 3, 3), np.complex128) if grad else None
            f = np.empty((4, self.V, 8), np.float64) if lie else None
        self._check(stag_force(self.h, x_even, g, f))
        return g, f

    def action(self, phi_even, x_even, mass):
        """S = phi^dag A^{-1} phi at the solution x_even, stationary form (a float)."""
        st, S = stag_action(self.h, mass, phi_even, x_even)
        self._check(st)
        return S

    def action_backward(self, x_even, gS, grad_links=None, grad_phi=None):
        """Fill grad_links (4, V, 3, 3) = gS K^dag and grad_phi (V/2, 3) = 2 gS x (either may be None)."""
        self._check(stag_action_backward(self.h, x_even, gS, grad_links, grad_phi))
        return grad_links, grad_phi

    def time_dslash(self, precision=STAG_FP32, nlaunch=50):
        st, ms, by = stag_time_dslash(self.h, precision, nlaunch)
        self._check(st)
        return ms, by

    def solve_counters(self):
        """(loop passes, reliable-update steps) of the most recent solve."""
        st, passes, ups = stag_solve_counters(self.h)
        self._check(st)
        return passes, ups

    def solve_form(self):
        """The autotuner's launch form of the CG kernels of the last solve."""
        st, f = stag_solve_form(self.h)
        self._check(st)
        return {"systems_per_thread": f[0], "groups": f[1], "lanes_k1": f[2], "lanes_k2": f[3],
                "link_path": ("planes", "tiled_smem", "tiled")[f[4]], "l2_persisting_links": f[5] == 1,
                "l2_persisting": ("none", "links", "vectors")[f[5]],
                "iterations_per_pass": f[6], "shared_memory_links": bool(f[7]),
                "kernels": ("k_dslash", "k_dslash_mrhs", "k_cg_nrhs", "k_cg_nrhs")[f[7]],
                "k1_systems_per_pass": 2 if f[7] == 3 else 1}

    def time_cg_kernel(self, kernel, precision=STAG_FP32, nlaunch=50):
        """(ms per launch, algorithmic bytes per launch) of CG kernel 0 or 1."""
        st, ms, by = stag_time_cg_kernel(self.h, precision, kernel, nlaunch)
        self._check(st)
        return ms, by
