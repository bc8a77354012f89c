"""Batched solves: many sources and masses in one launch sequence, and a ragged
batch of lattices of different sizes in one graph (the multi-RHS/mass and
ragged workloads), against the FP64 oracle.

Each system's true residual, recomputed by the CPU oracle, is <= 1e-10; the
ragged batch returns bit-for-bit the solutions of the lattices solved one at a
time (same kernels, same order, fixed-order reductions).
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


RAGGED = [(8, 8, 8, 8), (12, 12, 12, 24), (16, 16, 16, 32), (20, 20, 20, 64)]


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_ragged_batch_of_four_lattices(prec):
    P = stag.PRECISIONS[prec]
    masses = [0.05, 0.1]
    fields = []
    for n, L in enumerate(RAGGED):
        V = synth.volume(L)
        U = synth.random_links(L, 0.4, synth.seed_for(2, 10 * n + 1))
        bs = [synth.gaussian_vector(V // 2, synth.seed_for(2, 10 * n + 2 + r)) for r in range(2)]
        fields.append((L, U, bs))
    ctxs = []
    try:
        batch = []
        for L, U, bs in fields:
            c = stag.Context(L)
            c.links_upload(torch.from_numpy(U).cuda())
            ctxs.append(c)
            batch.append((c, [torch.from_numpy(b).cuda() for b in bs], masses))
        outs, st, its, trs = stag.cg_solve_ragged(batch, tol=1e-10, maxiter=20000, precision=P)
        assert st == stag.STAG_OK
        torch.cuda.synchronize()
        for (L, U, bs), xs, it, tr in zip(fields, outs, its, trs):
            for r, b in enumerate(bs):
                for k, m in enumerate(masses):
                    j = r * len(masses) + k
                    x = xs[j].cpu().numpy()
                    t = oracle.true_residual(L, U, m, b, x)
                    assert t <= 1e-10, (L, j, t)
                    assert abs(t - tr[j]) <= 1e-12 + 0.05 * t
        # the same lattices one at a time: identical results
        for (c, srcs, ms), xs in zip(batch, outs):
            ys, _, _, _ = c.cg_solve(srcs, ms, tol=1e-10, maxiter=20000, precision=P)
            for a, b in zip(xs, ys):
                assert torch.equal(a, b)
    finally:
        for c in ctxs:
            c.close()


def test_config2_twelve_sources_four_masses():
    """20^3 x 64, 12 complex-Gaussian sources x masses {0.01, 0.02, 0.03, 0.05}
    = 48 systems in one solve (links loaded once per site for 8 systems at a
    time); FP32 Krylov vectors with FP16 links, FP64 reliable updates."""
    L = (20, 20, 20, 64)
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, synth.seed_for(2, 1))
    bs = [synth.gaussian_vector(V // 2, synth.seed_for(2, 100 + r)) for r in range(12)]
    masses = [0.01, 0.02, 0.03, 0.05]
    with stag.Context(L) as ctx:
        ctx.links_upload(torch.from_numpy(U).cuda())
        xs, st, it, tr = ctx.cg_solve([torch.from_numpy(b).cuda() for b in bs], masses, tol=1e-10,
                                      maxiter=40000, precision=stag.STAG_FP16)
        torch.cuda.synchronize()
    assert st == stag.STAG_OK and np.all(tr <= 1e-10)
    # the oracle recomputes the true residual of a sample of the 48 systems
    for j in (0, 13, 26, 47):
        r, k = divmod(j, len(masses))
        t = oracle.true_residual(L, U, masses[k], bs[r], xs[j].cpu().numpy())
        assert t <= 1e-10, (j, t)
        assert abs(t - tr[j]) <= 1e-12 + 0.05 * t


@pytest.mark.parametrize("vec", ["fp16", "bf16"])
def test_config2_half_vectors_fp32_links(vec):
    """The 12-source x 4-mass workload (m = 0.01 ... 0.05) with the Krylov
    vectors p and D_oe p stored at FP16 / BF16 (per-site scale) and FP32
    reconstruct-12 links, FP32 arithmetic, FP64 reliable updates: all 48
    systems reach the 1e-10 true residual (BF16 links do not converge at
    these masses)."""
    L = (20, 20, 20, 64)
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, synth.seed_for(2, 1))
    bs = [synth.gaussian_vector(V // 2, synth.seed_for(2, 100 + r)) for r in range(12)]
    masses = [0.01, 0.02, 0.03, 0.05]
    P = stag.STAG_FP32 | (stag.STAG_VEC_FP16 if vec == "fp16" else stag.STAG_VEC_BF16)
    with stag.Context(L, recon12=True) as ctx:
        ctx.links_upload(torch.from_numpy(U).cuda())
        xs, st, it, tr = ctx.cg_solve([torch.from_numpy(b).cuda() for b in bs], masses, tol=1e-10,
                                      maxiter=40000, precision=P)
        torch.cuda.synchronize()
    assert st == stag.STAG_OK and np.all(tr <= 1e-10), (stag.status_name(st), tr.max())
    for j in (0, 13, 26, 47):
        r, k = divmod(j, len(masses))
        t = oracle.true_residual(L, U, masses[k], bs[r], xs[j].cpu().numpy())
        assert t <= 1e-10, (j, t)
        assert abs(t - tr[j]) <= 1e-12 + 0.05 * t
