"""FP64 CPU oracle for the even-odd staggered operator and CG (test infrastructure).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the CUDA product path
never does.  The arithmetic lives in ``stag_oracle.c`` (plain C, FP64, no FMA
contraction); this module only compiles it with gcc and marshals numpy arrays.

Layouts (complex128 numpy arrays, C order):
  links       (4, V, 3, 3)   direction, lexicographic site (x fastest), row, col
  full vector (V, 3)
  cb vector   (V/2, 3)       checkerboard index = lex // 2 of the sites of one parity
with dims = (Lx, Ly, Lz, Lt).

Parity notes: ``quantize_vectors``/``round_links`` are pinned to numpy's
float16 and torch's bfloat16 rounding; the operator, CG and force are pinned by
the free-field closed form, anti-Hermiticity, gauge covariance, translation
invariance, dense brute force and central finite differences (tests/).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stag_oracle.c")
_LIB = os.path.join(_HERE, "libstag_oracle.so")
_lock = threading.Lock()
_lib = None

_LIB_OMP = os.path.join(_HERE, "libstag_oracle_omp.so")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (once; again when the source is newer).
    openmp=True builds the all-core timing copy (the per-site loop of the
    operator in parallel, results bit-identical to the serial build)."""
    lib = _LIB_OMP if openmp else _LIB
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(_SRC)):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, *(["-fopenmp"] if openmp else []), _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, lib)
    return lib


def _bind(path):
    """Load a compiled oracle library from `path` and declare its signatures."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    L = ctypes.c_long
    sig = {
        "orc_dslash_full": (None, [P, I, P, P, P]),
        "orc_gather_parity": (None, [P, I, P, P]),
        "orc_scatter_parity": (None, [P, I, P, P]),
        "orc_dslash_oe": (None, [P, I, P, P, P]),
        "orc_dslash_eo": (None, [P, I, P, P, P]),
        "orc_mdagm": (None, [P, I, P, D, P, P]),
        "orc_true_residual": (D, [P, I, P, D, P, P]),
        "orc_cg": (I, [P, I, P, D, P, P, D, I, P, P]),
        "orc_solve_full": (I, [P, I, P, D, P, P, D, I, P, P]),
        "orc_cg_masses": (I, [P, I, P, I, P, P, P, D, I, P, P]),
        "orc_round_format": (D, [D, I, I]),
        "orc_quantize_vectors": (None, [I, L, P, P]),
        "orc_round_links": (None, [I, L, P, P]),
        "orc_force_K": (None, [P, I, P, P, P]),
        "orc_force_lie": (None, [L, P, P, P]),
        "orc_set_threads": (None, [I]),
        "orc_su3_project": (None, [P, P]),
        "orc_hyp": (None, [P, P, P, P]),
        "orc_spin_taste": (None, [I, I, P]),
        "orc_hypercube_path": (None, [P, P, P, I, I, P]),
        "orc_npr_contract": (None, [P, P, I, I, I, I, P, P, P, P, P]),
        "orc_threads": (I, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


class using:
    """Context manager: route this module's functions to another compiled copy
    of the oracle (used by the tests that plant mistakes in a copy)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        _lib = _bind(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


class threads:
    """Context manager: route this module's functions to the all-core build of
    the oracle with n threads (n = 0: every core).  Results are bit-identical
    to the serial build; only the operator's per-site loop runs in parallel.
    If the compiler cannot build it, the serial build stays in use."""

    def __init__(self, n=0):
        self.n = int(n) if n else (os.cpu_count() or 1)

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        try:
            lib = _bind(build(openmp=True))
            lib.orc_set_threads(self.n)
            _lib = lib
        except (OSError, subprocess.CalledProcessError):
            pass
        return self

    def count(self):
        """Threads the routed library actually uses."""
        return int(_load().orc_threads())

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB)
    return _lib


def _dims(L):
    a = np.ascontiguousarray(np.asarray(L, dtype=np.int32))
    assert a.shape == (4,)
    return a


def _c128(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def volume(L):
    return int(np.prod(np.asarray(L, dtype=np.int64)))


def dslash_full(L, links, v, antiperiodic=True):
    """D v on the full lattice."""
    lib = _load()
    d, U, x = _dims(L), _c128(links), _c128(v)
    out = np.empty_like(x)
    lib.orc_dslash_full(_p(d), int(antiperiodic), _p(U), _p(x), _p(out))
    return out


def gather_parity(L, par, full):
    lib = _load()
    d, f = _dims(L), _c128(full)
    out = np.empty((volume(L) // 2, 3), np.complex128)
    lib.orc_gather_parity(_p(d), int(par), _p(f), _p(out))
    return out


def scatter_parity(L, par, cb):
    lib = _load()
    d, c = _dims(L), _c128(cb)
    out = np.empty((volume(L), 3), np.complex128)
    lib.orc_scatter_parity(_p(d), int(par), _p(c), _p(out))
    return out


def dslash_oe(L, links, v_even, antiperiodic=True):
    """D_oe v: even-site input, odd-site output."""
    lib = _load()
    d, U, x = _dims(L), _c128(links), _c128(v_even)
    out = np.empty_like(x)
    lib.orc_dslash_oe(_p(d), int(antiperiodic), _p(U), _p(x), _p(out))
    return out


def dslash_eo(L, links, v_odd, antiperiodic=True):
    """D_eo v: odd-site input, even-site output."""
    lib = _load()
    d, U, x = _dims(L), _c128(links), _c128(v_odd)
    out = np.empty_like(x)
    lib.orc_dslash_eo(_p(d), int(antiperiodic), _p(U), _p(x), _p(out))
    return out


def mdagm(L, links, mass, v_even, antiperiodic=True):
    """(4 m^2 - D_eo D_oe) v on even sites."""
    lib = _load()
    d, U, x = _dims(L), _c128(links), _c128(v_even)
    out = np.empty_like(x)
    lib.orc_mdagm(_p(d), int(antiperiodic), _p(U), float(mass), _p(x), _p(out))
    return out


def true_residual(L, links, mass, b, x, antiperiodic=True):
    """||b - A x|| / ||b|| in FP64."""
    lib = _load()
    d, U, bb, xx = _dims(L), _c128(links), _c128(b), _c128(x)
    return float(lib.orc_true_residual(_p(d), int(antiperiodic), _p(U), float(mass),
                                       _p(bb), _p(xx)))


def cg(L, links, mass, b, tol=1e-10, maxiter=100000, antiperiodic=True):
    """Plain FP64 CG on A = M^dag M.  Returns (x, status, iters, true_res)."""
    lib = _load()
    d, U, bb = _dims(L), _c128(links), _c128(b)
    x = np.empty_like(bb)
    it = ctypes.c_int(0)
    tr = ctypes.c_double(0.0)
    st = lib.orc_cg(_p(d), int(antiperiodic), _p(U), float(mass), _p(bb), _p(x), float(tol),
                    int(maxiter), ctypes.byref(it), ctypes.byref(tr))
    return x, int(st), int(it.value), float(tr.value)


def cg_masses(L, links, masses, b, tol=1e-10, maxiter=100000, antiperiodic=True):
    """Plain FP64 CG for every mass (the shifted systems of one source), each
    independently.  Returns (xs (nmass, V/2, 3), worst status, iters, true_res)."""
    lib = _load()
    d, U, bb = _dims(L), _c128(links), _c128(b)
    m = np.ascontiguousarray(np.asarray(masses, dtype=np.float64))
    x = np.empty((len(m),) + bb.shape, np.complex128)
    it = np.zeros(len(m), np.int32)
    tr = np.zeros(len(m), np.float64)
    st = lib.orc_cg_masses(_p(d), int(antiperiodic), _p(U), len(m), _p(m), _p(bb), _p(x), float(tol),
                           int(maxiter), _p(it), _p(tr))
    return x, int(st), it, tr


def solve_full(L, links, mass, b_full, tol=1e-12, maxiter=100000, antiperiodic=True):
    """M x = b on the whole lattice, M = 2m + D, by the even-odd Schur route.
    b_full (V, 3).  Returns (x_full, status, iters, true_res of the even system)."""
    lib = _load()
    d, U, bb = _dims(L), _c128(links), _c128(b_full)
    x = np.empty_like(bb)
    it = ctypes.c_int(0)
    tr = ctypes.c_double(0.0)
    st = lib.orc_solve_full(_p(d), int(antiperiodic), _p(U), float(mass), _p(bb), _p(x), float(tol),
                            int(maxiter), ctypes.byref(it), ctypes.byref(tr))
    return x, int(st), int(it.value), float(tr.value)


HYP_ALPHA = (0.75, 0.6, 0.3)


def su3_project(X):
    """P(X): unitary polar factor (Newton's iteration) with the determinant's
    phase removed by the principal cube root; X (..., 3, 3)."""
    lib = _load()
    X = _c128(X)
    out = np.empty_like(X)
    flat_in = X.reshape(-1, 3, 3)
    flat_out = out.reshape(-1, 3, 3)
    for k in range(flat_in.shape[0]):
        a = np.ascontiguousarray(flat_in[k])
        b = np.empty_like(a)
        lib.orc_su3_project(_p(a), _p(b))
        flat_out[k] = b
    return out


def hyp(L, links, alpha=HYP_ALPHA):
    """HYP-smeared links (4, V, 3, 3) of `links` (Hasenfratz-Knechtli levels)."""
    lib = _load()
    d, U = _dims(L), _c128(links)
    a = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64))
    out = np.empty_like(U)
    lib.orc_hyp(_p(d), _p(U), _p(a), _p(out))
    return out


def spin_taste(S, F):
    """16 x 16 complex matrix (g_S x x_F)_AB = Tr(g_A^dag g_S g_B g_F^dag) / 4 (4-bit S, F)."""
    out = np.empty((16, 16), np.complex128)
    _load().orc_spin_taste(int(S), int(F), _p(out))
    return out


def hypercube_path(L, links, zc, A, D):
    """Average over the shortest paths from corner A to corner D of hypercube zc of the link products."""
    W = np.empty((3, 3), np.complex128)
    z = np.ascontiguousarray(np.asarray(zc, dtype=np.int32))
    _load().orc_hypercube_path(_p(_dims(L)), _p(_c128(links)), _p(z), int(A), int(D), _p(W))
    return W


def npr_contract(L, links, S1, F1, S2, F2, chibar1, chi2, chibar3, chi4):
    """O(z) of every hypercube ([V/16] complex) of the one-colour-trace four-fermion contraction."""
    V = volume(L)
    out = np.empty(V // 16, np.complex128)
    f = [_c128(v) for v in (chibar1, chi2, chibar3, chi4)]
    _load().orc_npr_contract(_p(_dims(L)), _p(_c128(links)), int(S1), int(F1), int(S2), int(F2),
                             _p(f[0]), _p(f[1]), _p(f[2]), _p(f[3]), _p(out))
    return out


def round_format(v, mant_bits, emin):
    return float(_load().orc_round_format(float(v), int(mant_bits), int(emin)))


PREC_FP32, PREC_FP16, PREC_BF16 = 1, 2, 3


def quantize_vectors(prec, v):
    """Values a (n, 3) complex vector holds after storage at `prec` (1/2/3)."""
    lib = _load()
    x = _c128(v)
    out = np.empty_like(x)
    lib.orc_quantize_vectors(int(prec), x.shape[0], _p(x), _p(out))
    return out


def round_links(prec, links):
    """Values link elements hold after storage at `prec` (1/2/3)."""
    lib = _load()
    x = _c128(links)
    out = np.empty_like(x)
    lib.orc_round_links(int(prec), x.size * 2, _p(x), _p(out))
    return out


def force_K(L, links, x_even, antiperiodic=True):
    """K_mu(x) with dS = Re Tr(K dU) for S = phi^dag A^{-1} phi, X = A^{-1} phi."""
    lib = _load()
    d, U, X = _dims(L), _c128(links), _c128(x_even)
    K = np.empty((4, volume(L), 3, 3), np.complex128)
    lib.orc_force_K(_p(d), int(antiperiodic), _p(U), _p(X), _p(K))
    return K


def force_lie(links, K):
    """f_a = Re Tr(i T_a U K), T_a = lambda_a/2; shape (4, V, 8)."""
    lib = _load()
    U, KK = _c128(links), _c128(K)
    n = U.size // 9
    f = np.empty(U.shape[:-2] + (8,), np.float64)
    lib.orc_force_lie(n, _p(U), _p(KK), _p(f))
    return f
