"""GPU parity of the staggered half operators and M^dag M against the FP64 CPU oracle.

Every call goes through the C ABI (libstag.so via ctypes).  Tolerances:
FP64 relative 1e-13 (norm) against the oracle on the same inputs; FP32/FP16/
BF16 relative 1e-6 against the oracle run on the inputs as the GPU stores them
(links and vectors rounded by the oracle's own storage model; with
reconstruct-12, row 2 rebuilt from the stored rows in FP64); outputs rounded to
FP16/BF16 (STAG_ROUND_OUTPUT) within half a unit of the per-site scale.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1511_00088_gb300 import stag, synth

pytestmark = pytest.mark.gpu

PREC = {"fp64": stag.STAG_FP64, "fp32": stag.STAG_FP32, "fp16": stag.STAG_FP16, "bf16": stag.STAG_BF16}
MANT = {"fp16": 10, "bf16": 7}
# lattices: smallest (L=2 on every axis), cubic, non-cubic, ragged last tile
LATTICES = [(2, 2, 2, 2), (4, 4, 4, 4), (4, 2, 6, 8), (6, 6, 6, 12), (6, 4, 10, 6), (8, 8, 8, 8)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1511_00088_gb300 import build
    build.build()
    stag.load()
    assert torch.cuda.is_available()


def effective_links(U, prec, recon):
    """Links as the GPU holds them: rounded to the storage precision; with
    reconstruct-12 the third row rebuilt (FP64) from the two stored rows."""
    if prec == "fp64":
        return U
    Ur = oracle.round_links(PREC[prec], U)
    if recon:
        Ur = Ur.copy()
        Ur[..., 2, :] = np.conj(np.cross(Ur[..., 0, :], Ur[..., 1, :]))
    return Ur


def effective_vec(v, prec):
    return v if prec == "fp64" else oracle.quantize_vectors(PREC[prec], v)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def tol_for(prec):
    return 1e-13 if prec == "fp64" else 1e-6


@pytest.mark.parametrize("L", LATTICES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
def test_dslash_and_mdagm_parity(L, prec):
    recon_opts = [False] if prec == "fp64" else [False, True]
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 201)
    xe = synth.gaussian_vector(V // 2, 202)
    xo = synth.gaussian_vector(V // 2, 203)
    m = 0.07
    for recon in recon_opts:
        Ue = effective_links(U, prec, recon)
        ref_oe = oracle.dslash_oe(L, Ue, effective_vec(xe, prec))
        ref_eo = oracle.dslash_eo(L, Ue, effective_vec(xo, prec))
        ref_m = oracle.mdagm(L, Ue, m, effective_vec(xe, prec))
        with stag.Context(L, recon12=recon) as ctx:
            ctx.links_upload(U)  # host links
            # host vectors
            g_oe = ctx.dslash_oe(xe, PREC[prec])
            g_eo = ctx.dslash_eo(xo, PREC[prec])
            g_m = ctx.mdagm(xe, m, PREC[prec])
            # device vectors
            d_oe = ctx.dslash_oe(torch.from_numpy(xe).cuda(), PREC[prec]).cpu().numpy()
        t = tol_for(prec)
        assert rel(g_oe, ref_oe) <= t, (recon, rel(g_oe, ref_oe))
        assert rel(g_eo, ref_eo) <= t, (recon, rel(g_eo, ref_eo))
        assert rel(g_m, ref_m) <= t, (recon, rel(g_m, ref_m))
        assert np.array_equal(d_oe, g_oe)
        # element-wise bound as well (no single site far off)
        assert np.abs(g_oe - ref_oe).max() <= 10 * t * np.abs(ref_oe).max()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 6, 6, 12)])
def test_half_storage_output_rounding(prec, L):
    """STAG_ROUND_OUTPUT: the solver's own half-storage kernel; each site's
    output is within half a unit (2^-(mant+1)) of its per-site scale."""
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 211)
    xe = synth.gaussian_vector(V // 2, 212)
    ref = oracle.dslash_oe(L, effective_links(U, prec, False), effective_vec(xe, prec))
    with stag.Context(L) as ctx:
        ctx.links_upload(U)
        g = ctx.dslash_oe(xe, PREC[prec] | stag.STAG_ROUND_OUTPUT)
    re = np.stack([ref.real, ref.imag], -1).reshape(-1, 6)
    ge = np.stack([g.real, g.imag], -1).reshape(-1, 6)
    scale = np.abs(ge).max(axis=1, keepdims=True)
    bound = scale * 2.0 ** -(MANT[prec] + 1) * (1 + 1e-4) + 1e-6 * np.abs(re).max()
    assert np.all(np.abs(ge - re) <= bound)
    assert rel(g, ref) < 2.0 ** -MANT[prec]


@pytest.mark.parametrize("prec,recon", [("fp64", False), ("fp32", False), ("fp32", True), ("fp16", False),
                                        ("fp16", True), ("bf16", False), ("bf16", True)])
def test_full_size_production_lattice(prec, recon):
    """20^3 x 64 (the paper's production shape): whole-field comparison with the
    oracle on the inputs as the GPU stores them, every link format (the
    benchmark's FP32 reconstruct-12 included) and storage precision."""
    L = (20, 20, 20, 64)
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, 1001)
    xe = synth.gaussian_vector(V // 2, 1002)
    m = 0.01
    Ue = effective_links(U, prec, recon)
    ref = oracle.mdagm(L, Ue, m, effective_vec(xe, prec))
    ref_oe = oracle.dslash_oe(L, Ue, effective_vec(xe, prec))
    with stag.Context(L, recon12=recon) as ctx:
        ctx.links_upload(torch.from_numpy(U).cuda())
        xd = torch.from_numpy(xe).cuda()
        g = ctx.mdagm(xd, m, PREC[prec]).cpu().numpy()
        g_oe = ctx.dslash_oe(xd, PREC[prec]).cpu().numpy()
    assert rel(g, ref) <= tol_for(prec)
    assert rel(g_oe, ref_oe) <= tol_for(prec)


def test_recon12_rejects_non_su3_links():
    L = (4, 4, 4, 4)
    U = synth.random_links(L, 0.4, 221)
    U[1, 5] *= 1.01  # not unitary any more
    st, h = stag.stag_create(L, stag.STAG_ANTIPERIODIC_T | stag.STAG_RECON12, 0)
    assert st == stag.STAG_OK
    try:
        assert stag.stag_links_upload(h, U) == stag.STAG_ERR_NOT_SU3
        assert "SU(3)" in stag.stag_last_error(h)
        x = synth.gaussian_vector(128, 1)
        out = np.empty_like(x)
        assert stag.stag_dslash_oe(h, stag.STAG_FP32, x, out) == stag.STAG_ERR_STATE
    finally:
        stag.stag_destroy(h)


def test_operator_before_upload_and_bad_precision():
    L = (4, 4, 4, 4)
    st, h = stag.stag_create(L, stag.STAG_ANTIPERIODIC_T, 0)
    try:
        x = synth.gaussian_vector(128, 1)
        out = np.empty_like(x)
        assert stag.stag_dslash_oe(h, stag.STAG_FP64, x, out) == stag.STAG_ERR_STATE
        assert stag.stag_links_upload(h, synth.random_links(L, 0.3, 2)) == stag.STAG_OK
        assert stag.stag_dslash_oe(h, 7, x, out) == stag.STAG_ERR_ARG
        assert stag.stag_mdagm(h, stag.STAG_FP64, 0.1, x, out) == stag.STAG_OK
    finally:
        stag.stag_destroy(h)


def test_periodic_time_boundary():
    """The antiperiodic flag off: the oracle's periodic operator."""
    L = (4, 4, 2, 6)
    V = synth.volume(L)
    U = synth.random_links(L, 0.5, 231)
    x = synth.gaussian_vector(V // 2, 232)
    ref = oracle.mdagm(L, U, 0.2, x, antiperiodic=False)
    with stag.Context(L, antiperiodic=False) as ctx:
        ctx.links_upload(U)
        g = ctx.mdagm(x, 0.2, stag.STAG_FP64)
    assert rel(g, ref) <= 1e-13
