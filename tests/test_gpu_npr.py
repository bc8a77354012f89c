"""The NPR one-colour-trace four-fermion contraction on the GPU
(stag_npr_contract) against the oracle (explicit gamma matrices and path
enumeration; pinned by the staggered-phase and Clifford correspondences,
orthogonality, gauge invariance, translations and a unit-link closed form).

The GPU takes the spin-taste signs from bit algebra and the path averages by
a last-step recursion; bar: every O(z) within 1e-13 of the largest |O| of
the oracle (both FP64), the sum likewise, on several spin-taste choices.
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


@pytest.mark.parametrize("L", [(2, 2, 2, 2), (4, 2, 6, 4), (4, 4, 4, 8)])
@pytest.mark.parametrize("st", [(0, 0, 0, 0), (1, 1, 1, 1), (5, 10, 15, 0), (7, 3, 2, 12), (15, 15, 9, 6)])
def test_npr_matches_oracle(L, st):
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 1001)
    fs = [synth.gaussian_vector(V, 1002 + k) for k in range(4)]
    ref = oracle.npr_contract(L, U, *st, *fs)
    scale = np.abs(ref).max()
    with stag.Context(L) as ctx:
        ctx.links_upload(U)
        O, tot = ctx.npr_contract(st, *fs)  # host fields
        Od, totd = ctx.npr_contract(st, *[torch.from_numpy(f).cuda() for f in fs])  # device fields
        Od = Od.cpu().numpy()
    for X, T in ((O, tot), (Od, totd)):
        assert np.abs(X - ref).max() <= 1e-13 * scale
        assert abs(T - ref.sum()) <= 1e-12 * np.abs(ref).sum()
    assert tot == totd  # fixed summation order


def test_npr_arguments():
    L = (2, 2, 2, 2)
    V = synth.volume(L)
    f = synth.gaussian_vector(V, 1010)
    with stag.Context(L) as ctx:
        out = np.zeros(1, np.complex128)
        assert stag.stag_npr_contract(ctx.h, (0, 0, 0, 0), f, f, f, f, None, out) == stag.STAG_ERR_STATE
        ctx.links_upload(synth.random_links(L, 0.4, 1011))
        assert stag.stag_npr_contract(ctx.h, (0, 16, 0, 0), f, f, f, f, None, out) == stag.STAG_ERR_ARG
        assert stag.stag_npr_contract(ctx.h, (0, 0, 0, 0), f, f, f, f, None, None) == stag.STAG_ERR_ARG
