"""Pins of the FP64 oracle's staggered operator against closed forms and invariants.

The paper (Sec. 3) names the operator (one-link staggered, even-odd
preconditioned, used inside a mixed-precision CG) without writing it down.  The
oracle's reading is pinned here by facts that do not depend on the oracle:

* free field: with unit links, plane waves with p_i = 2 pi n_i / L_i and
  antiperiodic p_t = 2 pi (n_t + 1/2) / L_t are eigenvectors of
  A = 4m^2 - D_eo D_oe with eigenvalue 4m^2 + 4 sum_mu sin^2 p_mu, and on 4^4
  these values are the whole spectrum of the dense A;
* D is anti-Hermitian for any links;
* gauge covariance under a random SU(3) transform;
* translation by two sites commutes with D (antiperiodic twist in t).
A dropped hop, a wrong eta, a U/U^dagger swap, a transposed link, an assigned
instead of accumulated contribution on a length-2 axis, or a wrong boundary
sign fails at least one of them.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1511_00088_gb300 import synth


def coords(L):
    V = synth.volume(L)
    i = np.arange(V)
    x = i % L[0]
    y = (i // L[0]) % L[1]
    z = (i // (L[0] * L[1])) % L[2]
    t = i // (L[0] * L[1] * L[2])
    return np.stack([x, y, z, t], axis=1)


def plane_wave(L, n, colour):
    p = 2 * np.pi * np.asarray(n, float) / np.asarray(L, float)
    p[3] = 2 * np.pi * (n[3] + 0.5) / L[3]
    ph = np.exp(1j * coords(L) @ p)
    return ph[:, None] * np.asarray(colour)[None, :], p


LATTICES = [(2, 2, 2, 2), (4, 4, 4, 4), (4, 2, 6, 8), (6, 4, 2, 4)]


@pytest.mark.parametrize("L", LATTICES)
def test_free_field_plane_waves(L):
    U = synth.unit_links(L)
    rng = np.random.default_rng(7)
    for m in (0.0, 0.05, 0.3):
        for _ in range(6):
            n = [int(rng.integers(0, L[k])) for k in range(4)]
            col = rng.standard_normal(3) + 1j * rng.standard_normal(3)
            psi, p = plane_wave(L, n, col)
            pe = oracle.gather_parity(L, 0, psi)
            lam = 4 * m * m + 4 * np.sum(np.sin(p) ** 2)
            Ape = oracle.mdagm(L, U, m, pe)
            assert np.abs(Ape - lam * pe).max() <= 1e-13 * max(lam, 1.0) * np.abs(pe).max()


def dense_A(L, U, m):
    n = synth.volume(L) // 2 * 3
    A = np.empty((n, n), np.complex128)
    e = np.zeros(n, np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        A[:, j] = oracle.mdagm(L, U, m, e.reshape(-1, 3)).reshape(-1)
    return A


def test_free_field_full_spectrum_4x4():
    L = (4, 4, 4, 4)
    m = 0.1
    A = dense_A(L, synth.unit_links(L), m)
    assert np.abs(A - A.conj().T).max() < 1e-14
    ev = np.sort(np.linalg.eigvalsh(A))
    # even-site plane waves: p and p + (pi,pi,pi,pi) coincide on even sites,
    # so take n_x in {0,1} (half the x momenta), times 3 colours
    vals = []
    for n in itertools.product(range(2), range(4), range(4), range(4)):
        p = 2 * np.pi * np.asarray(n, float) / 4
        p[3] = 2 * np.pi * (n[3] + 0.5) / 4
        vals += [4 * m * m + 4 * np.sum(np.sin(p) ** 2)] * 3
    vals = np.sort(vals)
    assert vals.shape == ev.shape
    assert np.abs(ev - vals).max() < 1e-12


@pytest.mark.parametrize("L", LATTICES)
def test_anti_hermiticity(L):
    U = synth.random_links(L, 0.5, 11)
    V = synth.volume(L)
    x = synth.gaussian_vector(V, 12)
    y = synth.gaussian_vector(V, 13)
    a = np.vdot(x, oracle.dslash_full(L, U, y))
    b = np.vdot(oracle.dslash_full(L, U, x), y)
    assert abs(a + b) <= 1e-13 * abs(a)
    # the even-odd blocks inherit it: D_eo^dag = -D_oe
    xe = oracle.gather_parity(L, 0, x)
    yo = oracle.gather_parity(L, 1, y)
    a = np.vdot(yo, oracle.dslash_oe(L, U, xe))
    b = np.vdot(oracle.dslash_eo(L, U, yo), xe)
    assert abs(a + b) <= 1e-13 * abs(a)


def shift_index(L, mu, d):
    """index map j(i) with x_j = x_i - d mu (periodic)."""
    c = coords(L).copy()
    c[:, mu] = (c[:, mu] - d) % L[mu]
    return c[:, 0] + L[0] * (c[:, 1] + L[1] * (c[:, 2] + L[2] * c[:, 3]))


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (4, 2, 6, 8)])
def test_gauge_covariance(L):
    U = synth.random_links(L, 0.6, 21)
    g = synth.gauge_transform(L, 22)
    V = synth.volume(L)
    psi = synth.gaussian_vector(V, 23)
    Ug = np.empty_like(U)
    for mu in range(4):
        fwd = shift_index(L, mu, -1)  # x + mu
        Ug[mu] = g @ U[mu] @ np.conj(np.transpose(g[fwd], (0, 2, 1)))
    lhs = oracle.dslash_full(L, Ug, np.einsum("nab,nb->na", g, psi))
    rhs = np.einsum("nab,nb->na", g, oracle.dslash_full(L, U, psi))
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(rhs).max()
    # and the solve residual / action are gauge invariant
    m = 0.2
    b = oracle.gather_parity(L, 0, psi)
    ge = np.stack([g[i] for i in range(V) if coords(L)[i].sum() % 2 == 0])
    x, st, _, _ = oracle.cg(L, U, m, b, tol=1e-12)
    xg, st2, _, _ = oracle.cg(L, Ug, m, np.einsum("nab,nb->na", ge, b), tol=1e-12)
    assert st == 0 and st2 == 0
    assert np.abs(np.einsum("nab,nb->na", ge, x) - xg).max() < 1e-9 * np.abs(x).max()


@pytest.mark.parametrize("mu", [0, 1, 2, 3])
def test_translation_by_two(mu):
    L = (4, 6, 4, 8)
    U = synth.random_links(L, 0.5, 31)
    V = synth.volume(L)
    psi = synth.gaussian_vector(V, 32)
    j = shift_index(L, mu, 2)  # (T f)(x) = f(x - 2 mu)
    c = coords(L)
    # antiperiodic twist: a value that crossed the t boundary changes sign
    tw = np.ones(V)
    if mu == 3:
        tw[c[:, 3] < 2] = -1.0
    Tpsi = tw[:, None] * psi[j]
    # links are translated without any sign: the antiperiodic boundary sign
    # belongs to the operator (fields are antiperiodic, links periodic)
    TU = U[:, j]
    lhs = oracle.dslash_full(L, TU, Tpsi)
    rhs = tw[:, None] * oracle.dslash_full(L, U, psi)[j]
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(rhs).max()


def test_mdagm_hermitian_positive_and_L2_accumulation():
    L = (2, 2, 2, 2)
    U = synth.random_links(L, 0.7, 41)
    m = 0.05
    A = dense_A(L, U, m)
    assert np.abs(A - A.conj().T).max() < 1e-14
    ev = np.linalg.eigvalsh(A)
    assert ev.min() >= 4 * m * m - 1e-12
    # D_oe must not be the zero map nor assign (on L=2 both hops land on the same
    # site and must add): compare with the dense -D_eo D_oe built from D itself
    V = 16
    D = np.empty((3 * V, 3 * V), np.complex128)
    e = np.zeros(3 * V, np.complex128)
    for j in range(3 * V):
        e[:] = 0
        e[j] = 1
        D[:, j] = oracle.dslash_full(L, U, e.reshape(-1, 3)).reshape(-1)
    assert np.abs(D + D.conj().T).max() < 1e-14
    c = coords(L)
    ev_idx = np.concatenate([[3 * i, 3 * i + 1, 3 * i + 2] for i in range(V) if c[i].sum() % 2 == 0])
    od_idx = np.concatenate([[3 * i, 3 * i + 1, 3 * i + 2] for i in range(V) if c[i].sum() % 2 == 1])
    Deo = D[np.ix_(ev_idx, od_idx)]
    Doe = D[np.ix_(od_idx, ev_idx)]
    assert np.abs(A - (4 * m * m * np.eye(24) - Deo @ Doe)).max() < 1e-13
