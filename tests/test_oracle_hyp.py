"""Pins of the oracle's HYP smearing (the smeared one-link field the operator
uses) and of its SU(3) projection, none of them a restatement of the code:

* projection: against the unitary polar factor from numpy's SVD (another
  algorithm) with the determinant phase removed; SU(3)-valued; covariant
  under P(g X h^dag) = g P(X) h^dag for g, h in SU(3);
* HYP: unit links are a fixed point; the output is SU(3); gauge covariance
  V[U^g] = V[U]^g; commutes with lattice translations; (a1, a2, a3) = 0 is the
  identity on SU(3) fields;
* first-order response to one perturbed link U = exp(i eps T) (path counting
  from the three-level definition: a parallel link displaced by the offsets
  of the staples' middle links receives the products of the levels'
  weights): itself (1 - a1); one step in nu != mu: a1 (1 - a2) / 6;
  one step in each of two directions: 2 (a1/6)(a2/4)(1 - a3); one step in
  each of the three: a1 a2 a3 / 8 (3! paths of weight a1/6 a2/4 a3/2).
"""
import numpy as np
import pytest

import oracle
from paper_1511_00088_gb300 import synth

ALPHA = oracle.HYP_ALPHA


def lex(L, x):
    return x[0] + L[0] * (x[1] + L[1] * (x[2] + L[2] * x[3]))


def random_su3(n, seed):
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    q, r = np.linalg.qr(z)
    q = q * (np.diagonal(r, axis1=1, axis2=2) / np.abs(np.diagonal(r, axis1=1, axis2=2)))[:, None, :]
    d = np.linalg.det(q)
    return q / (d ** (1 / 3))[:, None, None]


def svd_project(X):
    W, s, Vh = np.linalg.svd(X)
    Y = W @ Vh
    d = np.linalg.det(Y)
    return Y * np.exp(-1j * np.angle(d) / 3)[..., None, None]


def test_projection_against_svd_polar_factor():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((50, 3, 3)) + 1j * rng.standard_normal((50, 3, 3))
    P = oracle.su3_project(X)
    assert np.abs(P - svd_project(X)).max() < 1e-13
    assert np.abs(P @ np.conj(np.swapaxes(P, 1, 2)) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(P) - 1).max() < 1e-14
    g, h = random_su3(50, 4), random_su3(50, 5)
    gxh = g @ X @ np.conj(np.swapaxes(h, 1, 2))
    assert np.abs(oracle.su3_project(gxh) - g @ P @ np.conj(np.swapaxes(h, 1, 2))).max() < 1e-13


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (2, 4, 2, 4)])
def test_unit_links_fixed_point_and_zero_alpha(L):
    U = synth.unit_links(L)
    assert np.abs(oracle.hyp(L, U) - U).max() < 1e-15
    R = synth.random_links(L, 0.4, 11)
    assert np.abs(oracle.hyp(L, R, (0.0, 0.0, 0.0)) - R).max() < 1e-14


def test_output_is_su3_and_smooths():
    L = (4, 4, 4, 4)
    U = synth.random_links(L, 0.4, 12)
    H = oracle.hyp(L, U)
    assert np.abs(H @ np.conj(np.swapaxes(H, -1, -2)) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(H) - 1).max() < 1e-14

    def plaq(F):
        V = F.shape[1]
        tot = 0.0
        for i in range(V):
            x = [i % L[0], i // L[0] % L[1], i // (L[0] * L[1]) % L[2], i // (L[0] * L[1] * L[2])]
            for mu in range(4):
                for nu in range(mu + 1, 4):
                    xm = list(x); xm[mu] = (xm[mu] + 1) % L[mu]
                    xn = list(x); xn[nu] = (xn[nu] + 1) % L[nu]
                    P = F[mu, i] @ F[nu, lex(L, xm)] @ F[mu, lex(L, xn)].conj().T @ F[nu, i].conj().T
                    tot += np.trace(P).real / 3
        return tot / (6 * V)
    # smearing drives the average plaquette towards 1
    assert plaq(H) > plaq(U) + 0.05


def test_gauge_covariance():
    L = (4, 2, 4, 4)
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 13)
    g = random_su3(V, 14)
    Ug = np.empty_like(U)
    for mu in range(4):
        for i in range(V):
            x = [i % L[0], i // L[0] % L[1], i // (L[0] * L[1]) % L[2], i // (L[0] * L[1] * L[2])]
            x[mu] = (x[mu] + 1) % L[mu]
            Ug[mu, i] = g[i] @ U[mu, i] @ g[lex(L, x)].conj().T
    H, Hg = oracle.hyp(L, U), oracle.hyp(L, Ug)
    for mu in range(4):
        for i in range(V):
            x = [i % L[0], i // L[0] % L[1], i // (L[0] * L[1]) % L[2], i // (L[0] * L[1] * L[2])]
            x[mu] = (x[mu] + 1) % L[mu]
            assert np.abs(Hg[mu, i] - g[i] @ H[mu, i] @ g[lex(L, x)].conj().T).max() < 1e-13


@pytest.mark.parametrize("d", range(4))
def test_translation_invariance(d):
    L = (4, 2, 4, 6)
    U = synth.random_links(L, 0.4, 15)
    shape = (4, L[3], L[2], L[1], L[0], 3, 3)
    axis = 4 - d  # x is the fastest site index
    T = np.roll(U.reshape(shape), -1, axis=axis).reshape(U.shape)
    H, HT = oracle.hyp(L, U), oracle.hyp(L, T)
    assert np.abs(np.roll(H.reshape(shape), -1, axis=axis).reshape(U.shape) - HT).max() < 1e-14


def test_first_order_response_by_path_counting():
    L = (6, 6, 6, 6)
    a1, a2, a3 = 0.7, 0.5, 0.4
    T = np.array([[0.3, 0.1 - 0.2j, 0.05j], [0.1 + 0.2j, -0.1, 0.2], [-0.05j, 0.2, -0.2]])
    eps = 1e-7
    w, Q = np.linalg.eigh(T)
    x0, mu0 = (2, 3, 2, 3), 1
    U = synth.unit_links(L)
    U[mu0, lex(L, x0)] = Q @ np.diag(np.exp(1j * eps * w)) @ Q.conj().T
    H = oracle.hyp(L, U, (a1, a2, a3))

    def coef(*steps):
        y = list(x0)
        for dd, s in steps:
            y[dd] = (y[dd] + s) % L[dd]
        dH = (H[mu0, lex(L, y)] - np.eye(3)) / (1j * eps)
        return np.vdot(T, dH).real / np.vdot(T, T).real

    tol = 1e-6
    assert abs(coef() - (1 - a1)) < tol
    for dd in (0, 2, 3):
        for s in (-1, 1):
            assert abs(coef((dd, s)) - a1 * (1 - a2) / 6) < tol
    assert abs(coef((0, -1), (2, 1)) - 2 * (a1 / 6) * (a2 / 4) * (1 - a3)) < tol
    assert abs(coef((2, -1), (3, -1)) - 2 * (a1 / 6) * (a2 / 4) * (1 - a3)) < tol
    assert abs(coef((0, 1), (2, -1), (3, 1)) - a1 * a2 * a3 / 8) < tol
    assert abs(coef((1, 1))) < tol  # along the link: no staple reaches it at first order
