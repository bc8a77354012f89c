"""HYP smearing on the GPU (stag_hyp_smear) against the oracle's three-level
construction (pinned by path counting, gauge covariance, translations and the
unit fixed point), and the CG on the smeared field.

Bar: every smeared link within 1e-13 of the oracle's (both FP64; the two
projections reach the same unique polar factor by different iterations),
SU(3) to 1e-14, and solves on the smeared links with true residual <= 1e-10.
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


@pytest.mark.parametrize("L", [(2, 2, 2, 2), (4, 2, 6, 8), (6, 6, 6, 12)])
@pytest.mark.parametrize("alpha", [None, (0.6, 0.5, 0.4)])
def test_hyp_matches_oracle(L, alpha):
    U = synth.random_links(L, 0.4, 801)
    ref = oracle.hyp(L, U, oracle.HYP_ALPHA if alpha is None else alpha)
    with stag.Context(L) as ctx:
        H = ctx.hyp_smear(U, alpha)  # host buffers
        Ud = torch.from_numpy(U).cuda()
        Hd = ctx.hyp_smear(Ud, alpha).cpu().numpy()  # device buffers
        ctx.hyp_smear(Ud, alpha, out=Ud)  # in place
        Hi = Ud.cpu().numpy()
    for X in (H, Hd, Hi):
        assert np.abs(X - ref).max() <= 1e-13
    assert np.abs(H @ np.conj(np.swapaxes(H, -1, -2)) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(H) - 1).max() < 1e-14


def test_unit_field_and_cg_on_smeared_links():
    L = (8, 8, 8, 8)
    V = synth.volume(L)
    with stag.Context(L, recon12=True) as ctx:
        I = synth.unit_links(L)
        assert np.abs(ctx.hyp_smear(I) - I).max() < 1e-15
        U = synth.random_links(L, 0.4, 802)
        H = ctx.hyp_smear(torch.from_numpy(U).cuda())
        ctx.links_upload(H)  # SU(3): reconstruct-12 accepts it
        b = synth.gaussian_vector(V // 2, 803)
        xs, st, it, tr = ctx.cg_solve([b], [0.02], tol=1e-10, maxiter=20000, precision=stag.STAG_FP32)
        Hh = H.cpu().numpy()
    assert np.abs(Hh - oracle.hyp(L, U)).max() <= 1e-13
    t = oracle.true_residual(L, Hh, 0.02, b, xs[0])
    assert t <= 1e-10 and abs(t - tr[0]) <= 1e-12 + 0.05 * t


@pytest.mark.parametrize("scale", [1e-6, 1e6])
def test_hyp_of_scaled_links(scale):
    """The projection's polar factor is scale-invariant: links scaled by 1e-6 or
    1e6 (|det|^2 of the first-level sums near 1e-36 or 1e108, outside the range
    where the determinant scale comes from FP32 arithmetic, so its FP64 branch
    runs) smear to the oracle's links within the same bound."""
    L = (4, 2, 6, 8)
    U = scale * synth.random_links(L, 0.4, 804)
    ref = oracle.hyp(L, U)
    with stag.Context(L) as ctx:
        H = ctx.hyp_smear(U)
    assert np.abs(H - ref).max() <= 1e-13
    assert np.abs(H @ np.conj(np.swapaxes(H, -1, -2)) - np.eye(3)).max() < 1e-14
