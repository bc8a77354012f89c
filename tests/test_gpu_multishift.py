"""Multi-shift CG (stag_cg_solve_multishift): several masses of each source on
one Krylov space, then a per-mass mixed-precision refinement, against the FP64
oracle (an independent plain CG per mass, pinned against dense LU solves).

Every system's true residual, recomputed by the oracle, is <= 1e-10; the
solutions agree with the oracle's to what the conditioning allows.
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


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 6, 6, 12), (2, 2, 2, 2)])
@pytest.mark.parametrize("prec", ["fp32", "fp32vbf"])
def test_multishift_small(L, prec):
    P = {"fp32": stag.STAG_FP32, "fp32vbf": stag.STAG_FP32 | stag.STAG_VEC_BF16}[prec]
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 601)
    bs = [synth.gaussian_vector(V // 2, 602 + r) for r in range(2)]
    masses = [0.05, 0.02, 0.3, 0.02]  # unsorted, with a repeated mass (a zero shift)
    with stag.Context(L) as ctx:
        ctx.links_upload(U)
        xs, st, it, tr = ctx.cg_solve_multishift(bs, masses, tol=1e-10, maxiter=20000, precision=P)
    assert st == stag.STAG_OK
    for r, b in enumerate(bs):
        xo, st_o, it_o, tro = oracle.cg_masses(L, U, masses, b, tol=1e-12)
        for k, m in enumerate(masses):
            j = r * len(masses) + k
            t = oracle.true_residual(L, U, m, b, xs[j])
            assert t <= 1e-10, (r, k, t)
            assert abs(t - tr[j]) <= 1e-12 + 0.05 * t, (t, tr[j])
            # |x - x*| <= |b - A x| / lambda_min, lambda_min >= 4 m^2
            bound = (t + 1e-12) * np.linalg.norm(b) / (4 * m * m)
            assert np.linalg.norm(xs[j] - xo[k]) <= bound


def test_multishift_config2_masses():
    """20^3 x 64, links exp(0.4 i H), 4 sources x m = {0.01, 0.02, 0.03, 0.05}
    (the 12-source x 4-mass workload's masses), FP32 reconstruct-12 links."""
    L = (20, 20, 20, 64)
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, synth.seed_for(2, 1))
    bs = [synth.gaussian_vector(V // 2, synth.seed_for(2, 100 + r)) for r in range(4)]
    masses = [0.01, 0.02, 0.03, 0.05]
    with stag.Context(L, recon12=True) as ctx:
        ctx.links_upload(torch.from_numpy(U).cuda())
        xs, st, it, tr = ctx.cg_solve_multishift([torch.from_numpy(b).cuda() for b in bs], masses, tol=1e-10,
                                                 maxiter=40000, precision=stag.STAG_FP32)
        torch.cuda.synchronize()
    assert st == stag.STAG_OK and np.all(tr <= 1e-10), tr
    for j in (0, 5, 10, 15):
        r, k = divmod(j, len(masses))
        t = oracle.true_residual(L, U, masses[k], bs[r], xs[j].cpu().numpy())
        assert t <= 1e-10, (j, t)
        assert abs(t - tr[j]) <= 1e-12 + 0.05 * t


def test_multishift_arguments():
    L = (4, 4, 4, 4)
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 611)
    b = synth.gaussian_vector(V // 2, 612)
    xs = [np.empty_like(b) for _ in range(2)]
    with stag.Context(L) as ctx:
        ctx.links_upload(U)
        assert stag.stag_cg_solve_multishift(ctx.h, [b], [0.1, 0.2], 1e-10, 100, stag.STAG_FP64, xs)[0] \
            == stag.STAG_ERR_ARG
        # one mass: the plain solve
        x1, st, it, tr = ctx.cg_solve_multishift([b], [0.1], tol=1e-10)
        assert oracle.true_residual(L, U, 0.1, b, x1[0]) <= 1e-10
