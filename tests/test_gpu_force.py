"""GPU fermion force (stag_force) and the autograd action against the oracle and FD.

* Kernel parity: the gradient K^dag and the Lie-algebra force f_a from the GPU
  match the oracle's general two-term K (and its Lie projection) on the same
  solution X, to 1e-12 relative.
* 16^3 x 32, m = 0.02 (the force workload): f_a against central finite
  differences of S under U -> exp(+-i eps T_a) U, eps = 1e-6, at 64 random
  (link, direction, generator) samples, with S from the library's stag_action
  (the stationary form 2 Re<phi, x> - <x, A x>, second order in the solve
  error, summed in double-word FP64 so that S carries a few ulps); the bound is
  1e-6 relative plus the rounding floor of the difference quotient,
  16 eps_mach |S| / (2 eps), which the test also requires to lie below 1e-3 of
  the median |f_a| (so that the comparison discriminates).
* Autograd: backward gives the same gradient, grad phi = 2 X, and
  torch.autograd.gradcheck passes on a small lattice.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1511_00088_gb300 import stag, synth
from paper_1511_00088_gb300.autograd import fermion_action

pytestmark = pytest.mark.gpu

GELL_MANN = np.zeros((8, 3, 3), np.complex128)
GELL_MANN[0][0, 1] = GELL_MANN[0][1, 0] = 1
GELL_MANN[1][0, 1], GELL_MANN[1][1, 0] = -1j, 1j
GELL_MANN[2][0, 0], GELL_MANN[2][1, 1] = 1, -1
GELL_MANN[3][0, 2] = GELL_MANN[3][2, 0] = 1
GELL_MANN[4][0, 2], GELL_MANN[4][2, 0] = -1j, 1j
GELL_MANN[5][1, 2] = GELL_MANN[5][2, 1] = 1
GELL_MANN[6][1, 2], GELL_MANN[6][2, 1] = -1j, 1j
GELL_MANN[7] = np.diag([1, 1, -2]) / np.sqrt(3)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1511_00088_gb300 import build
    build.build()
    stag.load()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("L", [(2, 2, 2, 2), (4, 2, 6, 8), (16, 16, 16, 32)])
def test_force_kernel_matches_oracle(L):
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 401)
    X = synth.gaussian_vector(V // 2, 402)  # the force formula holds for any X
    with stag.Context(L) as ctx:
        ctx.links_upload(U)
        G, f = ctx.force(X, grad=True, lie=True)
    K = oracle.force_K(L, U, X)
    Gref = np.conj(np.transpose(K, (0, 1, 3, 2)))
    assert np.linalg.norm(G - Gref) / np.linalg.norm(Gref) <= 1e-13
    fref = oracle.force_lie(U, K)
    assert np.linalg.norm(f - fref) / np.linalg.norm(fref) <= 1e-13


def _expm_herm(T, eps):
    w, Q = np.linalg.eigh(T)
    return Q @ np.diag(np.exp(1j * eps * w)) @ Q.conj().T


def test_force_central_differences_16x32():
    L = (16, 16, 16, 32)
    V = synth.volume(L)
    m = 0.02
    U = synth.random_links(L, 0.4, synth.seed_for(3, 1))
    phi = synth.gaussian_vector(V // 2, synth.seed_for(3, 2))
    Ud = torch.from_numpy(U).cuda()
    phid = torch.from_numpy(phi).cuda()
    ctx = stag.Context(L)
    try:
        ctx.links_upload(Ud)
        xs, _, _, _ = ctx.cg_solve([phid], [m], tol=1e-12, precision=stag.STAG_FP64)
        _, f = ctx.force(xs[0], grad=False, lie=True)
        f = f.cpu().numpy()

        def action():
            ctx.links_upload(Ud)
            x, _, _, _ = ctx.cg_solve([phid], [m], tol=1e-12, precision=stag.STAG_FP32)
            return ctx.action(phid, x[0], m)

        rng = np.random.default_rng(404)
        eps = 1e-6
        S0 = abs(action())
        # finite-difference error budget: S to a few ulps (double-word sums;
        # the solve error enters S only at second order), differenced and
        # divided by 2 eps, plus a relative 1e-6 (the O(eps^2) truncation is
        # far below it)
        fd_floor = 16 * np.finfo(np.float64).eps * S0 / (2 * eps)
        med = float(np.median(np.abs(f)))
        assert fd_floor <= 1e-3 * med, (fd_floor, med, S0)
        worst = 0.0
        for _ in range(64):
            mu = int(rng.integers(0, 4))
            i = int(rng.integers(0, V))
            a = int(rng.integers(0, 8))
            U0 = Ud[mu, i].clone()
            vals = []
            for sg in (+1, -1):
                E = torch.from_numpy(_expm_herm(GELL_MANN[a] / 2, sg * eps)).cuda()
                Ud[mu, i] = E @ U0
                vals.append(action())
                Ud[mu, i] = U0
            fd = (vals[0] - vals[1]) / (2 * eps)
            err = abs(fd - f[mu, i, a]) / (1e-6 * abs(f[mu, i, a]) + fd_floor)
            worst = max(worst, err)
        assert worst <= 1.0, (worst, fd_floor, med, S0)
    finally:
        ctx.close()


def test_autograd_backward_and_gradcheck():
    L = (4, 4, 2, 4)
    V = synth.volume(L)
    m = 0.2
    U = torch.from_numpy(synth.random_links(L, 0.4, 411)).cuda().requires_grad_(True)
    phi = torch.from_numpy(synth.gaussian_vector(V // 2, 412)).cuda().requires_grad_(True)
    with stag.Context(L) as ctx:
        S = fermion_action(U, phi, ctx, m, tol=1e-14)
        S.backward()
        xs, _, _, _ = ctx.cg_solve([phi.detach()], [m], tol=1e-14, precision=stag.STAG_FP64)
        X = xs[0]
        G, _ = ctx.force(X)
        assert torch.allclose(U.grad, G, rtol=1e-10, atol=1e-12)
        assert torch.allclose(phi.grad, 2 * X, rtol=1e-10, atol=1e-12)
        # the oracle agrees on S
        Xo = oracle.cg(L, U.detach().cpu().numpy(), m, phi.detach().cpu().numpy(), tol=1e-13)[0]
        So = float(np.real(np.vdot(phi.detach().cpu().numpy(), Xo)))
        assert abs(float(S.detach()) - So) <= 1e-10 * abs(So)
        Ls = (2, 2, 2, 2)
        Vs = synth.volume(Ls)
        Us = torch.from_numpy(synth.random_links(Ls, 0.4, 413)).cuda().requires_grad_(True)
        ps = torch.from_numpy(synth.gaussian_vector(Vs // 2, 414)).cuda().requires_grad_(True)
        with stag.Context(Ls) as cs:
            assert torch.autograd.gradcheck(lambda u, p: fermion_action(u, p, cs, 0.3, tol=1e-14), (Us, ps),
                                            eps=1e-6, atol=1e-6, rtol=1e-5)


@pytest.mark.parametrize("on_device", [False, True])
def test_action_matches_oracle(on_device):
    """stag_action against S = 2 Re<phi, x> - Re<x, A x> with the oracle's A x
    (host numpy sums), for an arbitrary x (the form holds for any x), and
    equal to phi^dag A^{-1} phi at the oracle's solution."""
    L = (6, 4, 4, 8)
    V = synth.volume(L)
    m = 0.07
    U = synth.random_links(L, 0.4, 421)
    phi = synth.gaussian_vector(V // 2, 422)
    x = synth.gaussian_vector(V // 2, 423)
    Ax = oracle.mdagm(L, U, m, x)
    S_ref = 2 * np.vdot(phi, x).real - np.vdot(x, Ax).real
    with stag.Context(L) as ctx:
        ctx.links_upload(U)
        a, b = (torch.from_numpy(phi).cuda(), torch.from_numpy(x).cuda()) if on_device else (phi, x)
        S = ctx.action(a, b, m)
        assert abs(S - S_ref) <= 1e-13 * abs(S_ref), (S, S_ref)
        assert ctx.action(a, b, m) == S  # fixed summation order
        xo, st, _, _ = oracle.cg(L, U, m, phi, tol=1e-13)
        S_exact = np.vdot(phi, xo).real
        So = ctx.action(phi, xo, m)
        assert abs(So - S_exact) <= 1e-12 * abs(S_exact)


def test_action_backward_scales():
    """stag_action_backward: grad_links = gS K^dag (the force kernel's), grad_phi = 2 gS x."""
    L = (4, 4, 2, 4)
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 431)
    X = synth.gaussian_vector(V // 2, 432)
    gS = -1.75
    with stag.Context(L) as ctx:
        ctx.links_upload(U)
        G, _ = ctx.force(X, grad=True, lie=False)
        Gs = np.empty_like(G)
        gp = np.empty_like(X)
        ctx.action_backward(X, gS, Gs, gp)
    assert np.allclose(Gs, gS * G, rtol=1e-15, atol=0)
    assert np.array_equal(gp, 2 * gS * X)
