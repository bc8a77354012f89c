"""48^3 x 96, links exp(0.4 i H), 16 sources solved together at m = 0.005 with
reconstruct-12 FP32 links, FP32 inner iteration and FP64 reliable updates:
the large batched workload (two groups of 8 systems per thread).

Every system must reach ||b - A x|| / ||b|| <= 1e-10 by the library's FP64
residual; the oracle recomputes that residual for a sample of four systems
(each an FP64 operator application on 10.6 M sites), which must agree and be
<= 1e-10 too.
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


def test_config4_batched_16_sources():
    L = (48, 48, 48, 96)
    Ve = synth.volume(L) // 2
    m = 0.005
    Ud = synth.random_links_device(L, 0.4, synth.seed_for(4, 1), device="cuda")
    bs = [synth.gaussian_vector(Ve, synth.seed_for(4, 2 + r)) for r in range(16)]
    with stag.Context(L, recon12=True) as ctx:
        ctx.links_upload(Ud)
        xs, st, it, tr = ctx.cg_solve([torch.from_numpy(b).cuda() for b in bs], [m], tol=1e-10,
                                      maxiter=40000, precision=stag.STAG_FP32)
        torch.cuda.synchronize()
        xs = [x.cpu().numpy() for x in xs]
    assert st == stag.STAG_OK
    assert np.all(np.asarray(tr) <= 1e-10), tr
    U = Ud.cpu().numpy()
    del Ud
    for j in (0, 5, 10, 15):
        t = oracle.true_residual(L, U, m, bs[j], xs[j])
        assert t <= 1e-10 and abs(t - tr[j]) <= 1e-12 + 0.05 * t, (j, t, tr[j])
