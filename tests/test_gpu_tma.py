"""The single-system CG kernels reading the tiled site-owned link copy -- staged
through shared memory by bulk copies (link path 1) or loaded straight into
registers (link path 2) -- against the plane-layout path (0) and the oracle.

The paths read the same link values and do the same arithmetic per site; their
one-wave grids may differ in size (shared memory limits path 1's residency), so
the reduction order may differ and the comparison is at the solve tolerance:
both reach ||b - A x|| / ||b|| <= 1e-10 by the oracle's own residual, and agree
to the accuracy the condition number allows.
"""
import os

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


def solve_with(L, U, b, m, prec, recon, tma, lanes):
    old = {k: os.environ.get(k) for k in ("STAG_TMA", "STAG_LANES")}
    os.environ["STAG_TMA"] = str(tma)
    os.environ["STAG_LANES"] = str(lanes)
    try:
        with stag.Context(L, recon12=recon) as ctx:
            ctx.links_upload(U)
            xs, st, it, tr = ctx.cg_solve([b], [m], tol=1e-10, maxiter=20000, precision=prec)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return xs[0], int(it[0]), float(tr[0])


@pytest.mark.parametrize("L", [(2, 2, 2, 2), (4, 2, 6, 8), (6, 6, 6, 12), (8, 8, 8, 16)])
@pytest.mark.parametrize("recon", [False, True])
@pytest.mark.parametrize("lanes", [1, 2])
@pytest.mark.parametrize("path", [1, 2])
def test_tiled_links_match(L, recon, lanes, path):
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 71)
    b = synth.gaussian_vector(V // 2, 72)
    m = 0.05
    x1, it1, tr1 = solve_with(L, U, b, m, stag.STAG_FP32, recon, path, lanes)
    x0, it0, tr0 = solve_with(L, U, b, m, stag.STAG_FP32, recon, 0, lanes)
    for x, tr in ((x1, tr1), (x0, tr0)):
        t = oracle.true_residual(L, U, m, b, x)
        assert t <= 1e-10 and abs(t - tr) <= 1e-12 + 0.05 * t, (t, tr)
    kappa = (4 * m * m + 16) / (4 * m * m)
    assert np.linalg.norm(x1 - x0) / np.linalg.norm(x0) <= 2 * kappa * 1e-10
    assert abs(it1 - it0) <= max(3, it0 // 50), (it1, it0)


@pytest.mark.parametrize("prec", [stag.STAG_FP16, stag.STAG_FP16 | stag.STAG_HALF_VECTORS])
@pytest.mark.parametrize("path", [1, 2])
def test_tiled_half_links(prec, path):
    """FP16 links (and FP16 Krylov vectors, the gather form of the first kernel)."""
    L = (6, 6, 6, 12)
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 81)
    b = synth.gaussian_vector(V // 2, 82)
    m = 0.1
    x1, it1, tr1 = solve_with(L, U, b, m, prec, False, path, 2)
    t = oracle.true_residual(L, U, m, b, x1)
    assert t <= 1e-10 and abs(t - tr1) <= 1e-12 + 0.05 * t


@pytest.mark.parametrize("eager", [False, True])
def test_wait_giveup_reports_timeout_promptly(eager):
    """The bounded wait of the shared-memory link path, made to give up at once
    (STAG_TEST_WAIT_GIVEUP=1): the solve stops after the pass in which it gave
    up, returns STAG_ERR_TIMEOUT ("void") within seconds, every bulk copy has
    landed before its block exits, and the GPU context stays usable."""
    import time
    L = (6, 6, 6, 12)
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 91)
    b = synth.gaussian_vector(V // 2, 92)
    keys = ("STAG_TMA", "STAG_LANES", "STAG_TEST_WAIT_GIVEUP", "STAG_EAGER")
    old = {k: os.environ.get(k) for k in keys}
    os.environ.update({"STAG_TMA": "1", "STAG_LANES": "1", "STAG_TEST_WAIT_GIVEUP": "1",
                       "STAG_EAGER": "1" if eager else "0"})
    try:
        with stag.Context(L) as ctx:
            ctx.links_upload(U)
            bt = torch.from_numpy(b).cuda()
            xt = torch.empty_like(bt)
            t0 = time.perf_counter()
            st, it, tr = stag.stag_cg_solve(ctx.h, [bt], [0.05], 1e-10, 20000, stag.STAG_FP32, [xt])
            dt = time.perf_counter() - t0
            assert st == stag.STAG_ERR_TIMEOUT, stag.status_name(st)
            assert "void" in stag.stag_last_error(ctx.h)
            assert dt < 10.0, dt
            passes, _ = ctx.solve_counters()
            assert passes <= 8, passes  # the loop ended right after the give-up
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    torch.cuda.synchronize()
    # the same link path without the forced give-up still solves
    x, it, tr = solve_with(L, U, b, 0.05, stag.STAG_FP32, False, 1, 1)
    assert oracle.true_residual(L, U, 0.05, b, x) <= 1e-10
