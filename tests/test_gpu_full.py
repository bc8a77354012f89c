"""The full-lattice solve M x = b, M = 2m + D (stag_solve_full), against the
oracle: the even-site source 2m b_e - D_eo b_o and the odd-site
reconstruction x_o = (b_o - D_oe x_e) / (2m) run on the GPU around the CG.

The bar: ||b - M x|| / ||b|| <= 1e-10 recomputed with the oracle's own full
operator (M x = 2m x + D x), the library's reported residual agreeing with it,
and the solution matching the oracle's Schur-route solve (orc_solve_full,
itself pinned against a dense LU solve of M) to what the conditioning allows.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1511_00088_gb300 import stag, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1511_00088_gb300 import build
    build.build()
    stag.load()
    assert torch.cuda.is_available()


def full_residual(L, U, m, b, x):
    Mx = 2.0 * m * x + oracle.dslash_full(L, U, x)
    return np.linalg.norm(b - Mx) / np.linalg.norm(b)


@pytest.mark.parametrize("L", [(2, 2, 2, 2), (4, 2, 2, 4), (6, 6, 6, 12)])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32vbf"])
def test_full_solve_small_lattices(L, prec):
    P = {"fp64": stag.STAG_FP64, "fp32": stag.STAG_FP32, "fp32vbf": stag.STAG_FP32 | stag.STAG_VEC_BF16}[prec]
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 401)
    bs = [synth.gaussian_vector(V, 402 + r) for r in range(2)]
    masses = [0.05, 0.2]
    with stag.Context(L) as ctx:
        ctx.links_upload(U)
        xs, st, it, tr = ctx.solve_full(bs, masses, tol=1e-10, maxiter=20000, precision=P)
    assert st == stag.STAG_OK
    for r, b in enumerate(bs):
        for k, m in enumerate(masses):
            j = r * len(masses) + k
            res = full_residual(L, U, m, b, xs[j])
            assert res <= 1e-10, (j, res)
            assert abs(res - tr[j]) <= 1e-13 + 0.05 * res, (res, tr[j])
            xo, st_o, _, _ = oracle.solve_full(L, U, m, b, tol=1e-13)
            assert st_o == 0
            # |x - x*| <= |M^-1| |b - M x|; |M^-1| <= 1/(2m) (M = 2m + anti-Hermitian D)
            bound = 2 * (res + 1e-13) * np.linalg.norm(b) / (2 * m)
            assert np.linalg.norm(xs[j] - xo) <= bound, (np.linalg.norm(xs[j] - xo), bound)


def test_full_solve_production_lattice_device_buffers():
    """20^3 x 64, m = 0.01, FP32 reconstruct-12 inner iteration, device buffers."""
    L = (20, 20, 20, 64)
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, synth.seed_for(1, 1))
    b = synth.gaussian_vector(V, synth.seed_for(1, 7))
    m = 0.01
    with stag.Context(L, recon12=True) as ctx:
        ctx.links_upload(torch.from_numpy(U).cuda())
        bd = torch.from_numpy(b).cuda()
        xs, st, it, tr = ctx.solve_full([bd], [m], tol=1e-10, maxiter=30000, precision=stag.STAG_FP32)
        torch.cuda.synchronize()
    assert st == stag.STAG_OK
    x = xs[0].cpu().numpy()
    res = full_residual(L, U, m, b, x)
    assert res <= 1e-10 and abs(res - tr[0]) <= 1e-13 + 0.05 * res, (res, tr[0])


def test_full_solve_zero_source_and_bad_mass():
    L = (4, 4, 4, 4)
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 411)
    z = np.zeros((V, 3), np.complex128)
    b = synth.gaussian_vector(V, 412)
    with stag.Context(L) as ctx:
        ctx.links_upload(U)
        xs, st, it, tr = ctx.solve_full([z, b], [0.1], tol=1e-10, maxiter=3000, precision=stag.STAG_FP32)
        assert st == stag.STAG_OK and it[0] == 0 and tr[0] == 0.0 and np.all(xs[0] == 0)
        assert full_residual(L, U, 0.1, b, xs[1]) <= 1e-10
        x = np.empty_like(b)
        for bad in (0.0, -0.1, float("nan")):
            assert stag.stag_solve_full(ctx.h, [b], [bad], 1e-10, 100, stag.STAG_FP32, [x])[0] \
                == stag.STAG_ERR_ARG
