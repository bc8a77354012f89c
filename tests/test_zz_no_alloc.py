"""The no-allocation entry point stag_mdagm_dot_noalloc, through the C ABI.

It serves callers that cannot allocate device memory (their memory belongs to
another allocator, or they must not allocate after set-up): every vector is
caller-owned and the reduction scratch is a fixed device array inside the
library.  Two calls in a row must both agree with the allocating entry points
(stag_mdagm, stag_dslash_oe) -- the second call reuses the shared scratch
left by the first.  This file is collected last on purpose.
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


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_noalloc_matches_allocating_entry_points_on_two_calls():
    L = (6, 6, 6, 12)  # 1296 sites per parity: the last block is ragged
    V = synth.volume(L)
    Ve = V // 2
    U = synth.random_links(L, 0.4, 301)
    m = 0.07
    with stag.Context(L) as ctx:
        ctx.links_upload(torch.from_numpy(U).cuda())
        for seed in (302, 303):
            x = torch.from_numpy(synth.gaussian_vector(Ve, seed)).cuda()
            t = torch.empty_like(x)
            out = torch.empty_like(x)
            dot = torch.zeros(1, dtype=torch.float64, device="cuda")
            st = stag.stag_mdagm_dot_noalloc(ctx.h, m, x, t, out, dot)
            assert st == stag.STAG_OK, stag.stag_last_error(ctx.h)
            torch.cuda.synchronize()
            ref = ctx.mdagm(x, m, stag.STAG_FP64)
            ref_t = ctx.dslash_oe(x, stag.STAG_FP64)
            assert rel(out, ref) <= 1e-13
            assert rel(t, ref_t) <= 1e-13
            d_ref = torch.vdot(x.flatten(), ref.flatten()).real.item()
            assert abs(dot.item() - d_ref) <= 1e-12 * abs(d_ref)
            # and against the FP64 CPU oracle directly: A x, D_oe x and <x, A x>
            xh = x.cpu().numpy()
            o_ref = oracle.mdagm(L, U, m, xh)
            t_ref = oracle.dslash_oe(L, U, xh)
            assert np.linalg.norm(out.cpu().numpy() - o_ref) <= 1e-13 * np.linalg.norm(o_ref)
            assert np.linalg.norm(t.cpu().numpy() - t_ref) <= 1e-13 * np.linalg.norm(t_ref)
            d_orc = float(np.vdot(xh.reshape(-1), o_ref.reshape(-1)).real)
            assert abs(dot.item() - d_orc) <= 1e-12 * abs(d_orc)


def test_noalloc_rejects_oversized_lattice_and_host_pointers():
    # 64^3 x 66: more sites per parity than the fixed scratch covers; no links
    # are needed for the size check, so nothing large is allocated here
    st, h = stag.stag_create((64, 64, 64, 66), stag.STAG_ANTIPERIODIC_T, 0)
    assert st == stag.STAG_OK
    try:
        x = torch.zeros((4, 3), dtype=torch.complex128, device="cuda")
        assert stag.stag_mdagm_dot_noalloc(h, 0.1, x, x.clone(), x.clone()) == stag.STAG_ERR_ARG
        assert "too large" in stag.stag_last_error(h)
    finally:
        stag.stag_destroy(h)
    L = (4, 4, 4, 4)
    with stag.Context(L) as ctx:
        ctx.links_upload(synth.random_links(L, 0.3, 304))
        xh = synth.gaussian_vector(128, 305)
        xd = torch.from_numpy(xh).cuda()
        assert stag.stag_mdagm_dot_noalloc(ctx.h, 0.1, xh, np.empty_like(xh), np.empty_like(xh)) \
            == stag.STAG_ERR_ARG
        assert stag.stag_mdagm_dot_noalloc(ctx.h, 0.1, xd, torch.empty_like(xd), torch.empty_like(xd)) \
            == stag.STAG_OK
        torch.cuda.synchronize()
