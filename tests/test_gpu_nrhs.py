"""The batched CG kernels that run every system in every block on links staged
once per tile in shared memory (k_cg_nrhs), forced with STAG_NRHS, against the
oracle and the one-system-per-block form.

Lattices with a ragged last tile (Ve not a multiple of 64), 2..48 systems
(sources x masses), full and reconstruct-12 links, 2 and 4 threads per site
with two link stages, 4 with one stage, and 4 with two systems per pass
(reconstruct-12; STAG_NRHS = 2, 4, 14, 24):
every system's true residual recomputed by the oracle is <= 1e-10.
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


def solve_forced(L, U, bs, masses, recon, nrhs):
    old = os.environ.get("STAG_NRHS")
    os.environ["STAG_NRHS"] = str(nrhs)
    try:
        with stag.Context(L, recon12=recon) as ctx:
            ctx.links_upload(U)
            xs, st, it, tr = ctx.cg_solve(bs, masses, tol=1e-10, maxiter=20000, precision=stag.STAG_FP32)
            form = ctx.solve_form()
    finally:
        if old is None:
            os.environ.pop("STAG_NRHS", None)
        else:
            os.environ["STAG_NRHS"] = old
    return xs, st, it, tr, form


@pytest.mark.parametrize("L", [(4, 2, 6, 8), (6, 6, 6, 12), (2, 2, 2, 2), (8, 8, 8, 16)])
@pytest.mark.parametrize("recon", [False, True])
@pytest.mark.parametrize("sl", [2, 4, 14, 24])
def test_nrhs_form_matches_oracle(L, recon, sl):
    if sl == 24 and not recon:
        pytest.skip("two systems per pass: reconstruct-12 links only")
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 701)
    bs = [synth.gaussian_vector(V // 2, 702 + r) for r in range(3)]
    masses = [0.03, 0.1]
    xs, st, it, tr, form = solve_forced(L, U, bs, masses, recon, sl)
    assert st == stag.STAG_OK
    assert form["kernels"] == "k_cg_nrhs" and form["lanes_k1"] == sl % 10, form
    for r, b in enumerate(bs):
        for k, m in enumerate(masses):
            j = r * len(masses) + k
            t = oracle.true_residual(L, U, m, b, xs[j])
            assert t <= 1e-10, (j, t)
            assert abs(t - tr[j]) <= 1e-12 + 0.05 * t
    # the one-system-per-block form reaches the same solutions (solve tolerance)
    ys, st0, it0, tr0, form0 = solve_forced(L, U, bs, masses, recon, 0)
    assert form0["kernels"] != "k_cg_nrhs"
    for j in range(len(xs)):
        m = masses[j % len(masses)]
        bound = 2e-10 * np.linalg.norm(bs[j // len(masses)]) / (4 * m * m)
        assert np.linalg.norm(xs[j] - ys[j]) <= bound
        assert abs(int(it[j]) - int(it0[j])) <= max(3, int(it0[j]) // 50)


@pytest.mark.parametrize("sl", [4, 24])
def test_nrhs_form_48_systems_production_lattice(sl):
    """20^3 x 64, 12 sources x {0.01, 0.02, 0.03, 0.05}: the 48-system batch in
    this form (reconstruct-12 FP32 links), oracle residual of a sample."""
    L = (20, 20, 20, 64)
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, synth.seed_for(2, 1))
    bs = [synth.gaussian_vector(V // 2, synth.seed_for(2, 100 + r)) for r in range(12)]
    masses = [0.01, 0.02, 0.03, 0.05]
    bd = [torch.from_numpy(b).cuda() for b in bs]
    xs, st, it, tr, form = solve_forced(L, torch.from_numpy(U).cuda(), bd, masses, True, sl)
    torch.cuda.synchronize()
    assert st == stag.STAG_OK and np.all(tr <= 1e-10)
    assert form["kernels"] == "k_cg_nrhs"
    for j in (0, 13, 26, 47):
        r, k = divmod(j, len(masses))
        t = oracle.true_residual(L, U, masses[k], bs[r], xs[j].cpu().numpy())
        assert t <= 1e-10, (j, t)


@pytest.mark.parametrize("nsrc,masses", [(16, [0.05, 0.07, 0.1, 0.2]), (13, [0.05, 0.07, 0.1, 0.15, 0.2])])
def test_nrhs_at_and_beyond_max_systems(nsrc, masses):
    """64 systems, the most this form takes (one shared-memory slot per
    system), run in it; 65 systems fall back to another form: every system's
    true residual by the oracle <= 1e-10 in both."""
    L = (4, 4, 4, 8)
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 711)
    bs = [synth.gaussian_vector(V // 2, 712 + r) for r in range(nsrc)]
    xs, st, it, tr, form = solve_forced(L, U, bs, masses, True, 4)
    assert st == stag.STAG_OK
    nsys = nsrc * len(masses)
    assert (form["kernels"] == "k_cg_nrhs") == (nsys <= 64), form
    for j in range(nsys):
        r, k = divmod(j, len(masses))
        t = oracle.true_residual(L, U, masses[k], bs[r], xs[j])
        assert t <= 1e-10, (j, t)
        assert abs(t - tr[j]) <= 1e-12 + 0.05 * t
