"""The kernel-timing entry point the roofline uses (stag_time_cg_kernel):
positive times, the algorithmic byte model of its documentation, and no
effect on the solver -- it runs the CG kernels on the context's own vectors
and states (each kernel folding its predecessor's partial sums, as in the
solve), so a solve after it must return exactly what it returned before."""
import pytest
import torch

from paper_1511_00088_gb300 import stag, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1511_00088_gb300 import build
    build.build()
    stag.load()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("nsrc,recon", [(1, True), (1, False), (6, True)])
def test_time_cg_kernel_model_and_no_side_effect(nsrc, recon):
    L = (8, 8, 8, 16)
    V = synth.volume(L)
    Ve = V // 2
    U = torch.from_numpy(synth.random_links(L, 0.4, 901)).cuda()
    bs = [torch.from_numpy(synth.gaussian_vector(Ve, 902 + r)).cuda() for r in range(nsrc)]
    with stag.Context(L, recon12=recon) as ctx:
        ctx.links_upload(U)
        xs, st, it, tr = ctx.cg_solve(bs, [0.05], tol=1e-10, maxiter=20000, precision=stag.STAG_FP32)
        assert st == stag.STAG_OK
        xs = [x.clone() for x in xs]
        link = 8 * (6 if recon else 9)  # FP32 complex elements of a stored link
        for k, per_system in ((0, 3 * 24), (1, 7 * 24)):  # t_old, r gathered, t | t gathered, p, r, x
            ms, by = ctx.time_cg_kernel(k, stag.STAG_FP32, nlaunch=10)
            assert ms > 0.0
            assert by == Ve * (8 * link + nsrc * per_system)
        ms, by = ctx.time_dslash(stag.STAG_FP32, nlaunch=10)
        assert ms > 0.0
        ys, st2, it2, tr2 = ctx.cg_solve(bs, [0.05], tol=1e-10, maxiter=20000, precision=stag.STAG_FP32)
        assert st2 == stag.STAG_OK and list(it2) == list(it)
        for x, y in zip(xs, ys):
            assert torch.equal(x, y)
