"""Plant plausible mistakes in a copy of the oracle and check that the pins catch each.

Every mutant is a one-line textual change of ``oracle/stag_oracle.c`` compiled
into a temporary library (on the CPU); the pin tests of the operator, CG and
force are then run against it and at least one of them must fail.  This is the
evidence that the pins constrain each term of the oracle, not just its overall
shape.

Not listed: the reversed phase convention eta_mu = (-1)^(x_{mu+1}+...+x_3).  It
is another valid anticommuting choice (unitarily equivalent), so no
convention-free pin can reject it; the GPU-oracle parity tests fix which
convention both sides use.
"""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_hyp as hy
from tests import test_oracle_npr as npr
from tests import test_oracle_operator as op
from tests import test_oracle_solver as sv

SRC = os.path.join(os.path.dirname(oracle.__file__), "stag_oracle.c")

MUTANTS = {
    "backward link not daggered": (
        "c_mul(c_conj(Ub[b * 3 + a]), in[jb * 3 + b])", "c_mul(Ub[a * 3 + b], in[jb * 3 + b])"),
    "backward link conjugated, not transposed": (
        "c_mul(c_conj(Ub[b * 3 + a]), in[jb * 3 + b])", "c_mul(c_conj(Ub[a * 3 + b]), in[jb * 3 + b])"),
    "forward link transposed": (
        "c_mul(Uf[a * 3 + b], in[jf * 3 + b])", "c_mul(Uf[b * 3 + a], in[jf * 3 + b])"),
    "backward link taken at x": (
        "const cplx *Ub = link_at(U, V, mu, jb);", "const cplx *Ub = link_at(U, V, mu, i);"),
    "forward link taken at x+mu": (
        "const cplx *Uf = link_at(U, V, mu, i);", "const cplx *Uf = link_at(U, V, mu, jf);"),
    "eta includes own direction": (
        "for (int nu = 0; nu < mu; ++nu) s += x[nu];", "for (int nu = 0; nu <= mu; ++nu) s += x[nu];"),
    "no antiperiodic sign": (
        "x[3] == L[3] - 1) ? -1 : 1;", "x[3] == L[3]) ? -1 : 1;"),
    "backward hop added": (
        "acc[a] = c_sub(acc[a], c_scale(sb, h));", "acc[a] = c_add(acc[a], c_scale(sb, h));"),
    "backward hop assigned, not accumulated": (
        "acc[a] = c_sub(acc[a], c_scale(sb, h));", "acc[a] = c_scale(-sb, h);"),
    "backward hop dropped in x": (
        "acc[a] = c_sub(acc[a], c_scale(sb, h));", "if (mu) acc[a] = c_sub(acc[a], c_scale(sb, h));"),
    "mass term 2m^2": ("double m4 = 4.0 * mass * mass;", "double m4 = 2.0 * mass * mass;"),
    "mass term added to D_eo D_oe": (
        "out_even[k] = m4 * in_even[k] - out_even[k];", "out_even[k] = m4 * in_even[k] + out_even[k];"),
    "CG beta inverted": ("double beta = rr_new / rr;", "double beta = rr / rr_new;"),
    "CG x update sign": ("x[k] += alpha * p[k];", "x[k] -= alpha * p[k];"),
    "force second term added": (
        "k[a * 3 + b] = c_scale(s, c_sub(t1, t2));", "k[a * 3 + b] = c_scale(s, c_add(t1, t2));"),
    "force without phase": (
        "k[a * 3 + b] = c_scale(s, c_sub(t1, t2));", "k[a * 3 + b] = c_sub(t1, t2);"),
    "force outer product transposed": (
        "cplx t1 = c_mul(P2[j * 3 + a], c_conj(P1[i * 3 + b]));",
        "cplx t1 = c_mul(P2[j * 3 + b], c_conj(P1[i * 3 + a]));"),
    "Lie projection sign": ("f[n * 8 + g] = -0.5 * tr.im;", "f[n * 8 + g] = 0.5 * tr.im;"),
    "full solve: odd source added to the even one": (
        "bt[k] = 2.0 * mass * be[k] - t[k];", "bt[k] = 2.0 * mass * be[k] + t[k];"),
    "full solve: even source without 2m": (
        "bt[k] = 2.0 * mass * be[k] - t[k];", "bt[k] = be[k] - t[k];"),
    "full solve: odd sites without 1/(2m)": (
        "xo[k] = (bo[k] - t[k]) / (2.0 * mass);", "xo[k] = (bo[k] - t[k]) / mass;"),
    "HYP level 3 staple weight a1/4": (
        "c_scale(a1 / 6.0, acc[k])", "c_scale(a1 / 4.0, acc[k])"),
    "HYP level 2 thin weight": (
        "c_scale(1.0 - a2, u[k])", "c_scale(1.0 - a3, u[k])"),
    "HYP staple's last link not daggered": (
        "m_dag(fc(cc, d, xmu), cd);", "for (int k = 0; k < 9; ++k) cd[k] = fc(cc, d, xmu)[k];"),
    "HYP negative staple starts at x+d": (
        "shifted(L, x, d, -1, xmd);", "shifted(L, x, d, 1, xmd);"),
    "HYP level 2 decorated by nu": (
        "int sdir = 6 - mu - nu - rho; /* 0+1+2+3 = 6 */", "int sdir = nu;"),
    "HYP level 3 side links decorated by nu": (
        "fctx side = {Vt, V, L, mu}, mid = {Vt, V, L, nu};", "fctx side = {Vt, V, L, nu}, mid = {Vt, V, L, nu};"),
    "projection keeps the determinant phase": (
        "for (int k = 0; k < 9; ++k) W[k] = c_mul(Y[k], rot);", "for (int k = 0; k < 9; ++k) W[k] = Y[k];"),
    "NPR: g_A not daggered": (
        "for (int j = 0; j < 4; ++j) gAd[i * 4 + j] = c_conj(gA[j * 4 + i]);",
        "for (int j = 0; j < 4; ++j) gAd[i * 4 + j] = gA[i * 4 + j];"),
    "NPR: taste matrix not daggered": (
        "for (int j = 0; j < 4; ++j) gFd[i * 4 + j] = c_conj(gF[j * 4 + i]);",
        "for (int j = 0; j < 4; ++j) gFd[i * 4 + j] = gF[i * 4 + j];"),
    "NPR: backward path step not daggered": (
        "m_dag(U + ((long)mu * V + corner_site(L, zc, nxt)) * 9, step);",
        "for (int q = 0; q < 9; ++q) step[q] = U[((long)mu * V + corner_site(L, zc, nxt)) * 9 + q];"),
    "NPR: colours of the two bilinears not crossed": (
        "t2 = c_add(t2, c_mul(cb3[sC * 3 + a], c_mul(Wcb[a * 3 + b], c2[sB * 3 + b])));",
        "t2 = c_add(t2, c_mul(cb3[sC * 3 + b], c_mul(Wcb[a * 3 + b], c2[sB * 3 + a])));"),
    "NPR: path from D to A": (
        "orc_hypercube_path(L, Ud, zc, A, D, (double *)Wad);", "orc_hypercube_path(L, Ud, zc, D, A, (double *)Wad);"),
    "multi-mass oracle reuses the first mass": (
        "int st = orc_cg(L, antiperiodic, U, masses[k], b, x + k * n, tol, maxiter,",
        "int st = orc_cg(L, antiperiodic, U, masses[0], b, x + k * n, tol, maxiter,"),
}


def _pins():
    yield lambda: op.test_free_field_plane_waves((2, 2, 2, 2))
    yield lambda: op.test_free_field_plane_waves((4, 2, 6, 8))
    yield lambda: op.test_anti_hermiticity((4, 2, 6, 8))
    yield lambda: op.test_gauge_covariance((4, 2, 6, 8))
    for mu in range(4):
        yield lambda mu=mu: op.test_translation_by_two(mu)
    yield lambda: sv.test_cg_matches_dense_solve((2, 2, 2, 2), 0.05, 0.7)
    yield lambda: sv.test_cg_degenerate_cases()
    yield lambda: sv.test_force_central_differences((2, 2, 2, 4))
    yield lambda: sv.test_full_lattice_solve_matches_dense((2, 2, 2, 2), 0.05, 0.7)
    yield lambda: sv.test_cg_masses_matches_dense_solves((2, 2, 2, 2), 0.7)
    yield hy.test_projection_against_svd_polar_factor
    yield hy.test_output_is_su3_and_smooths
    yield hy.test_gauge_covariance
    for d in range(4):
        yield lambda d=d: hy.test_translation_invariance(d)
    yield hy.test_first_order_response_by_path_counting
    yield npr.test_spin_taste_identity_phases_and_orthogonality
    yield npr.test_hypercube_paths
    yield lambda: npr.test_contraction_gauge_invariance((7, 3, 2, 12))
    yield npr.test_contraction_translation_by_one_hypercube
    yield npr.test_contraction_unit_links_closed_form


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, source, tmp_path):
    old, new = MUTANTS[name]
    assert source.count(old) == 1, f"mutation site not unique/found: {old}"
    mutated = source.replace(old, new)
    src = tmp_path / "mutant.c"
    src.write_text(mutated)
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", *oracle.CFLAGS, str(src), "-o", str(lib), "-lm"])
    caught = False
    with oracle.using(str(lib)):
        for pin in _pins():
            try:
                pin()
            except (AssertionError, FloatingPointError, ValueError, ZeroDivisionError,
                    np_linalg_error()):
                caught = True
                break
    assert caught, f"no pin failed for mutant: {name}"


def np_linalg_error():
    import numpy as np
    return np.linalg.LinAlgError
