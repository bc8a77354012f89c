"""Pins of the oracle's NPR one-colour-trace four-fermion contraction (the DP
workload of Sec. 4, Eq. (ffop)), none a restatement of the code:

* spin-taste matrices: (g_0 x x_0) = 1; (g_mu x x_0)_{A, A+mu} is the
  staggered phase eta_mu(A) and zero elsewhere (the one-link hopping term of
  the staggered action, the classic correspondence); (g_S x x_S) is diagonal
  with the commutation sign of g_A and g_S; the 256 matrices are orthogonal,
  Tr(M_{SF}^dag M_{S'F'}) = 16 delta delta (a basis of the 16 x 16 hypercube
  matrices);
* hypercube paths: unit links give 1; one step is the link (or its adjoint
  against the direction); W(D, A) = W(A, D)^dag; gauge covariance;
* contraction: gauge invariance of O(z) with the fields transformed
  (chi -> g chi, chibar -> chibar g^dag); translation by one hypercube; with
  unit links and S = F = 0 the closed form O(z) = Tr(G14 G32) of the Gram
  matrices G14[A, C] = chibar1(z_A) . chi4(z_C), G32[C, A] = chibar3(z_C) . chi2(z_A).
"""
import numpy as np
import pytest

import oracle
from paper_1511_00088_gb300 import synth
from tests.test_oracle_hyp import lex, random_su3


def test_spin_taste_identity_phases_and_orthogonality():
    assert np.abs(oracle.spin_taste(0, 0) - np.eye(16)).max() == 0.0
    for mu in range(4):
        M = oracle.spin_taste(1 << mu, 0)
        for A in range(16):
            eta = (-1) ** sum((A >> nu) & 1 for nu in range(mu))
            ref = np.zeros(16)
            ref[A ^ (1 << mu)] = eta
            assert np.abs(M[A] - ref).max() < 1e-15
    G = np.array([oracle.spin_taste(S, F).reshape(-1) for S in range(16) for F in range(16)])
    assert np.abs(G.conj() @ G.T - 16 * np.eye(256)).max() < 1e-13
    # S = F: diagonal, entry A the sign of g_A g_S = +- g_S g_A (Clifford algebra:
    # (-1)^(n_A n_S - |A and S|), n = number of set bits)
    bits = lambda v: bin(v).count("1")
    for S in range(16):
        ref = np.diag([(-1.0) ** (bits(A) * bits(S) - bits(A & S)) for A in range(16)])
        assert np.abs(oracle.spin_taste(S, S) - ref).max() < 1e-15


def corner_site(L, zc, A):
    return lex(L, [2 * zc[m] + ((A >> m) & 1) for m in range(4)])


def test_hypercube_paths():
    L = (4, 4, 2, 4)
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 901)
    I = synth.unit_links(L)
    zc = (1, 0, 0, 1)
    for A in range(16):
        assert np.abs(oracle.hypercube_path(L, I, zc, A, (A * 7 + 3) % 16) - np.eye(3)).max() < 1e-15
        assert np.abs(oracle.hypercube_path(L, U, zc, A, A) - np.eye(3)).max() == 0.0
        for mu in range(4):
            B = A ^ (1 << mu)
            W = oracle.hypercube_path(L, U, zc, A, B)
            ref = U[mu, corner_site(L, zc, A)] if not (A >> mu) & 1 else U[mu, corner_site(L, zc, B)].conj().T
            assert np.abs(W - ref).max() < 1e-15
    g = random_su3(V, 902)
    Ug = np.empty_like(U)
    for mu in range(4):
        for i in range(V):
            x = [i % L[0], i // L[0] % L[1], i // (L[0] * L[1]) % L[2], i // (L[0] * L[1] * L[2])]
            x[mu] = (x[mu] + 1) % L[mu]
            Ug[mu, i] = g[i] @ U[mu, i] @ g[lex(L, x)].conj().T
    for A, D in ((0, 15), (3, 12), (5, 6), (9, 9), (1, 14)):
        W = oracle.hypercube_path(L, U, zc, A, D)
        assert np.abs(oracle.hypercube_path(L, U, zc, D, A) - W.conj().T).max() < 1e-15
        Wg = oracle.hypercube_path(L, Ug, zc, A, D)
        sa, sd = corner_site(L, zc, A), corner_site(L, zc, D)
        assert np.abs(Wg - g[sa] @ W @ g[sd].conj().T).max() < 1e-14


def fields(L, seed):
    V = synth.volume(L)
    return [synth.gaussian_vector(V, seed + k) for k in range(4)]


@pytest.mark.parametrize("st", [(0, 0, 0, 0), (1, 1, 1, 1), (5, 10, 15, 0), (7, 3, 2, 12)])
def test_contraction_gauge_invariance(st):
    L = (4, 2, 4, 4)
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 911)
    cb1, c2, cb3, c4 = fields(L, 912)
    O = oracle.npr_contract(L, U, *st, cb1, c2, cb3, c4)
    g = random_su3(V, 913)
    Ug = np.empty_like(U)
    for mu in range(4):
        for i in range(V):
            x = [i % L[0], i // L[0] % L[1], i // (L[0] * L[1]) % L[2], i // (L[0] * L[1] * L[2])]
            x[mu] = (x[mu] + 1) % L[mu]
            Ug[mu, i] = g[i] @ U[mu, i] @ g[lex(L, x)].conj().T
    chi = lambda v: np.einsum("iab,ib->ia", g, v)           # chi -> g chi
    chib = lambda v: np.einsum("ib,iab->ia", v, g.conj())   # chibar -> chibar g^dag
    Og = oracle.npr_contract(L, Ug, *st, chib(cb1), chi(c2), chib(cb3), chi(c4))
    assert np.abs(Og - O).max() < 1e-12 * np.abs(O).max()


def test_contraction_translation_by_one_hypercube():
    L = (4, 4, 2, 4)
    U = synth.random_links(L, 0.4, 921)
    fs = fields(L, 922)
    st = (3, 6, 9, 12)
    O = oracle.npr_contract(L, U, *st, *fs)
    shape_f = (L[3], L[2], L[1], L[0], 3)
    shape_u = (4, L[3], L[2], L[1], L[0], 3, 3)
    H = [L[m] // 2 for m in range(4)]
    for d in range(4):
        ax = 3 - d
        Ut = np.roll(U.reshape(shape_u), -2, axis=ax + 1).reshape(U.shape)
        ft = [np.roll(f.reshape(shape_f), -2, axis=ax).reshape(f.shape) for f in fs]
        Ot = oracle.npr_contract(L, Ut, *st, *ft)
        ref = np.roll(O.reshape(H[3], H[2], H[1], H[0]), -1, axis=ax).reshape(O.shape)
        assert np.abs(Ot - ref).max() < 1e-12 * np.abs(O).max()


def test_contraction_unit_links_closed_form():
    L = (4, 2, 2, 4)
    U = synth.unit_links(L)
    cb1, c2, cb3, c4 = fields(L, 931)
    O = oracle.npr_contract(L, U, 0, 0, 0, 0, cb1, c2, cb3, c4)
    H = [L[m] // 2 for m in range(4)]
    for h in range(len(O)):
        zc = [h % H[0], h // H[0] % H[1], h // (H[0] * H[1]) % H[2], h // (H[0] * H[1] * H[2])]
        s = [corner_site(L, zc, A) for A in range(16)]
        G14 = cb1[s] @ c4[s].T
        G32 = cb3[s] @ c2[s].T
        assert abs(O[h] - np.trace(G14 @ G32)) < 1e-12 * abs(O[h])
