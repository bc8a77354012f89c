"""Pins of the oracle's CG, fermion force and reduced-precision storage model.

* CG: against a dense LU solve of the assembled A (brute force on 2^4 and 4^4)
  and by its recomputed true residual.
* Force: dS = Re Tr(K dU) of S = phi^dag A^{-1} phi against central finite
  differences of S under U -> exp(i eps T_a) U, with S from dense solves.
* Storage: the oracle's FP16/BF16 rounding against numpy's float16 and torch's
  bfloat16 conversions (both round to nearest, ties to even).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1511_00088_gb300 import synth
from tests.test_oracle_operator import coords, dense_A

GELL_MANN = np.zeros((8, 3, 3), np.complex128)
GELL_MANN[0][0, 1] = GELL_MANN[0][1, 0] = 1
GELL_MANN[1][0, 1], GELL_MANN[1][1, 0] = -1j, 1j
GELL_MANN[2][0, 0], GELL_MANN[2][1, 1] = 1, -1
GELL_MANN[3][0, 2] = GELL_MANN[3][2, 0] = 1
GELL_MANN[4][0, 2], GELL_MANN[4][2, 0] = -1j, 1j
GELL_MANN[5][1, 2] = GELL_MANN[5][2, 1] = 1
GELL_MANN[6][1, 2], GELL_MANN[6][2, 1] = -1j, 1j
GELL_MANN[7] = np.diag([1, 1, -2]) / np.sqrt(3)


@pytest.mark.parametrize("L,m,c", [((2, 2, 2, 2), 0.05, 0.7), ((4, 4, 4, 4), 0.1, 0.4),
                                   ((4, 2, 2, 6), 0.02, 0.5)])
def test_cg_matches_dense_solve(L, m, c):
    U = synth.random_links(L, c, 101)
    b = synth.gaussian_vector(synth.volume(L) // 2, 102)
    A = dense_A(L, U, m)
    xd = np.linalg.solve(A, b.reshape(-1)).reshape(-1, 3)
    x, st, it, tr = oracle.cg(L, U, m, b, tol=1e-12)
    assert st == 0 and tr <= 1e-12
    # the returned true residual is the plain definition, to the rounding of
    # recomputing b - A x in FP64: first order eps |b| + eps |A||x| per
    # component (two recomputations with different summation orders -- this
    # dense product, the oracle's stencil -- differ by about that much)
    r = b.reshape(-1) - A @ x.reshape(-1)
    bnd = np.finfo(float).eps * np.linalg.norm(np.abs(b.reshape(-1)) + np.abs(A) @ np.abs(x.reshape(-1)))
    assert abs(tr - np.linalg.norm(r) / np.linalg.norm(b)) <= bnd / np.linalg.norm(b)
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 10 * kappa * 1e-12


def test_cg_degenerate_cases():
    L = (4, 4, 2, 2)
    U = synth.random_links(L, 0.4, 111)
    z = np.zeros((synth.volume(L) // 2, 3), np.complex128)
    x, st, it, tr = oracle.cg(L, U, 0.1, z)
    assert st == 0 and it == 0 and np.all(x == 0) and tr == 0.0
    b = synth.gaussian_vector(synth.volume(L) // 2, 112)
    x, st, it, tr = oracle.cg(L, U, 0.1, b, tol=1e-10, maxiter=1)
    assert st == 1 and it == 1 and tr > 1e-10


def action(L, U, m, phi):
    A = dense_A(L, U, m)
    return float(np.real(np.vdot(phi.reshape(-1), np.linalg.solve(A, phi.reshape(-1)))))


@pytest.mark.parametrize("L", [(2, 2, 2, 4), (4, 2, 2, 2)])
def test_force_central_differences(L):
    m = 0.1
    U = synth.random_links(L, 0.5, 121)
    V = synth.volume(L)
    phi = synth.gaussian_vector(V // 2, 122)
    A = dense_A(L, U, m)
    X = np.linalg.solve(A, phi.reshape(-1)).reshape(-1, 3)
    K = oracle.force_K(L, U, X)
    f = oracle.force_lie(U, K)
    rng = np.random.default_rng(123)
    eps = 1e-5
    c = coords(L)
    # sample every direction, both parities and the t-boundary links
    picks = [(mu, i) for mu in range(4) for i in range(V)]
    idx = rng.choice(len(picks), size=24, replace=False)
    chosen = [picks[k] for k in idx]
    chosen += [(3, int(np.flatnonzero(c[:, 3] == L[3] - 1)[0])),
               (3, int(np.flatnonzero(c[:, 3] == L[3] - 1)[1]))]
    for mu, i in chosen:
        a = int(rng.integers(0, 8))
        T = GELL_MANN[a] / 2
        vals = []
        for s in (+1, -1):
            w, Q = np.linalg.eigh(T)
            E = Q @ np.diag(np.exp(1j * s * eps * w)) @ Q.conj().T
            Up = U.copy()
            Up[mu, i] = E @ U[mu, i]
            vals.append(action(L, Up, m, phi))
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - f[mu, i, a]) <= 1e-6 * max(1.0, abs(fd)), (mu, i, a, fd, f[mu, i, a])
    # dS = Re Tr(K dU) for an arbitrary complex direction dU of one link
    mu, i = 1, 3
    dU = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    Up, Um = U.copy(), U.copy()
    Up[mu, i] += eps * dU
    Um[mu, i] -= eps * dU
    fd = (action(L, Up, m, phi) - action(L, Um, m, phi)) / (2 * eps)
    assert abs(fd - np.real(np.trace(K[mu, i] @ dU))) <= 1e-6 * max(1.0, abs(fd))


def test_force_single_outer_product_form():
    """The two terms of K coincide: K = 2s Y(x+mu) X(x)^dag on even x and
    K = -2s X(x+mu) Y(x)^dag on odd x (X even, Y = D_oe X odd)."""
    L = (4, 4, 2, 4)
    U = synth.random_links(L, 0.5, 131)
    V = synth.volume(L)
    X = synth.gaussian_vector(V // 2, 132)
    K = oracle.force_K(L, U, X)
    Y = oracle.dslash_oe(L, U, X)
    Xf = oracle.scatter_parity(L, 0, X)
    Yf = oracle.scatter_parity(L, 1, Y)
    c = coords(L)
    for mu in range(4):
        for i in range(V):
            x = c[i]
            xf = x.copy()
            xf[mu] = (x[mu] + 1) % L[mu]
            j = xf[0] + L[0] * (xf[1] + L[1] * (xf[2] + L[2] * xf[3]))
            eta = (-1) ** int(x[:mu].sum())
            bs = -1 if (mu == 3 and x[3] == L[3] - 1) else 1
            s = eta * bs
            if x.sum() % 2 == 0:
                ref = 2 * s * np.outer(Yf[j], Xf[i].conj())
            else:
                ref = -2 * s * np.outer(Xf[j], Yf[i].conj())
            assert np.abs(K[mu, i] - ref).max() < 1e-12


def test_round_format_ties_and_subnormals():
    # FP16: 10 fraction bits, emin -14
    assert oracle.round_format(1 + 2.0 ** -11, 10, -14) == 1.0          # tie -> even
    assert oracle.round_format(1 + 3 * 2.0 ** -11, 10, -14) == 1 + 2.0 ** -9
    assert oracle.round_format(2.0 ** -25, 10, -14) == 0.0              # half the min subnormal -> even (0)
    assert oracle.round_format(3 * 2.0 ** -25, 10, -14) == 2.0 ** -23
    assert oracle.round_format(-1.5 * 2.0 ** -24, 10, -14) == -2 * 2.0 ** -24
    rng = np.random.default_rng(5)
    v = rng.standard_normal(20000) * np.exp(rng.uniform(-20, 3, 20000))
    v32 = v.astype(np.float32).astype(np.float64)
    ref16 = v32.astype(np.float16).astype(np.float64)
    got16 = np.array([oracle.round_format(a, 10, -14) for a in v32])
    assert np.array_equal(ref16, got16)
    ref_bf = torch.from_numpy(v32.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    got_bf = np.array([oracle.round_format(a, 7, -126) for a in v32])
    assert np.array_equal(ref_bf, got_bf)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_quantize_vectors_matches_library_rounding(prec):
    rng = np.random.default_rng(6)
    n = 5000
    v = (rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))) \
        * np.exp(rng.uniform(-8, 8, (n, 1)))
    v[7] = 0.0
    got = oracle.quantize_vectors(prec, v)
    re = np.stack([v.real, v.imag], axis=-1).reshape(n, 6).astype(np.float32)
    if prec == 1:
        ref = re.astype(np.float64)
    else:
        s = np.abs(re).max(axis=1, keepdims=True)
        with np.errstate(invalid="ignore", divide="ignore"):
            q = np.where(s > 0, re / s, np.float32(0)).astype(np.float32)
        if prec == 2:
            qq = q.astype(np.float16).astype(np.float32)
        else:
            qq = torch.from_numpy(q).to(torch.bfloat16).to(torch.float32).numpy()
        ref = (qq * s).astype(np.float32).astype(np.float64)
    ref = ref.reshape(n, 3, 2)
    ref = ref[..., 0] + 1j * ref[..., 1]
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_round_links_matches_library_rounding(prec):
    U = synth.random_links((2, 2, 2, 4), 0.5, 141)
    got = oracle.round_links(prec, U)
    f = U.view(np.float64).astype(np.float32)
    if prec == 1:
        ref = f.astype(np.float64)
    elif prec == 2:
        ref = f.astype(np.float16).astype(np.float64)
    else:
        ref = torch.from_numpy(f).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(got.view(np.float64), ref)


@pytest.mark.parametrize("L,m,c", [((2, 2, 2, 2), 0.05, 0.7), ((4, 2, 2, 4), 0.1, 0.4)])
def test_full_lattice_solve_matches_dense(L, m, c):
    """M x = b on the whole lattice (M = 2m + D) by the even-odd Schur route
    equals a dense LU solve of the assembled M."""
    V = synth.volume(L)
    U = synth.random_links(L, c, 111)
    b = synth.gaussian_vector(V, 112)
    n = 3 * V
    M = np.empty((n, n), np.complex128)
    e = np.zeros(n, np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        M[:, j] = 2 * m * e + oracle.dslash_full(L, U, e.reshape(-1, 3)).reshape(-1)
    xd = np.linalg.solve(M, b.reshape(-1)).reshape(-1, 3)
    x, st, it, tr = oracle.solve_full(L, U, m, b, tol=1e-13)
    assert st == 0
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10
    r = 2 * m * x + oracle.dslash_full(L, U, x) - b
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-11


def test_all_core_build_is_bit_identical():
    """The -fopenmp timing build of the oracle parallelises only the per-site
    loop of the operator: its CG returns exactly the serial build's solution."""
    L = (4, 4, 4, 8)
    V = oracle.volume(L)
    U = synth.random_links(L, 0.4, 501)
    b = synth.gaussian_vector(V // 2, 502)
    x1, st1, it1, tr1 = oracle.cg(L, U, 0.1, b, tol=1e-10)
    with oracle.threads(4) as th:
        assert th.count() >= 1
        x2, st2, it2, tr2 = oracle.cg(L, U, 0.1, b, tol=1e-10)
    assert (st1, it1, tr1) == (st2, it2, tr2)
    assert np.array_equal(x1, x2)


@pytest.mark.parametrize("L,c", [((2, 2, 2, 2), 0.7), ((4, 2, 2, 4), 0.5)])
def test_cg_masses_matches_dense_solves(L, c):
    """The multi-mass oracle (one source, several shifts 4 m^2) against a dense
    LU solve of each assembled A_m, and each mass's own CG."""
    U = synth.random_links(L, c, 121)
    b = synth.gaussian_vector(synth.volume(L) // 2, 122)
    masses = [0.03, 0.07, 0.2, 0.5]
    xs, st, it, tr = oracle.cg_masses(L, U, masses, b, tol=1e-12)
    assert st == 0 and np.all(tr <= 1e-12)
    for k, m in enumerate(masses):
        A = dense_A(L, U, m)
        xd = np.linalg.solve(A, b.reshape(-1)).reshape(-1, 3)
        kappa = np.linalg.cond(A)
        assert np.linalg.norm(xs[k] - xd) / np.linalg.norm(xd) <= 10 * kappa * 1e-12
        x1, _, it1, _ = oracle.cg(L, U, m, b, tol=1e-12)
        assert np.array_equal(xs[k], x1) and it[k] == it1
    # heavier masses need fewer iterations
    assert list(it) == sorted(it, reverse=True)
