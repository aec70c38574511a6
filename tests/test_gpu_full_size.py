"""Parity at the full 24^4 size of the benchmark workload (eps 0.25, kappa 0.1565,
antiperiodic time), in every step-kernel form the autotuner can pick there: the
compile-time-block form with one or two rhs per lane and the staged form with one
or two rhs per thread, for the 512-vector batch of the cheapest level (16-rhs
blocks) and the 8-vector batch of the solves (8-rhs blocks).

The oracle cannot apply M to 512 vectors of 4M components in seconds, so it
computes sampled right-hand sides one by one: M eta_j (Sec. 1's Wilson-Dirac
matrix) and the level sample eta_j^H p(M) eta_j (Eq. 2 with the polynomial of
Sec. 3 given by its roots) for noise indices j spread over several rhs blocks,
including the first and the last.

The chains the benchmark itself runs (degree 32 - 8 over 512 noises, 128 - 32 over
128, the 40 x 8 double polynomial of degree 319 - 128 over 32) are checked against
samples the oracle computed once, stored with the command that wrote them
(tests/golden/make_c4_levels.py, oracle only).

Tolerances as in the small-lattice tests: FP32 storage 1e-5 relative (normwise for
M eta, and element-wise against the largest element, so that one wrong site
fails; for the bilinear 1e-5 ||eta|| ||p(M) eta||, Cauchy-Schwarz applied to a
normwise error of p(M) eta), BF16 storage 2^-8 + 1e-6 (Z(4) inputs are exact in
BF16, one rounding of the output)."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import krylov, noise, wilson

pytestmark = pytest.mark.gpu

BF16_BOUND = 2.0 ** -8 + 1e-6
SAMPLED = (0, 5, 300, 511)  # rhs blocks 0, 0, 18, 31 of the 512 batch
LEVEL = 4
THETA = np.array([1.0 + 0.8j, 1.0 - 0.8j, 0.3 + 0.0j])  # p of degree 2 (two matvecs)

# (version, rpt, minb, traversal, store hint) of the forms exercised: v2 lane widths, v3 thread
# widths, v4 register caps, traversals (0 lexicographic, 1 4D blocks, 2 z-halves) and hints
FORMS = [(2, 1, 4, 0, 0), (2, 2, 3, 0, 0), (3, 1, 1, 0, 0), (3, 2, 1, 0, 0),
         (4, 1, 4, 0, 0), (4, 1, 3, 2, 1), (4, 1, 4, 1, 1), (5, 1, 4, 0, 0), (5, 1, 4, 2, 0)]


@pytest.fixture(scope="module")
def mmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_00016_gb300 import mmc as m
    return m


@pytest.fixture(scope="module")
def big(mmc):
    W = synth.WORKLOADS["c4_24x24x24x24"]
    U = synth.random_gauge(W.dims, W.eps, W.gauge_seed)
    ctx = mmc.mmc_create(W.dims, seed=W.noise_seed, device=0)
    mmc.mmc_load_gauge(ctx, U, W.kappa, W.t_antiperiodic)
    shape = (W.dims[3], W.dims[2], W.dims[1], W.dims[0], 4, 3)
    op = lambda v: wilson.apply_M(U, W.kappa, v.reshape(shape), bool(W.t_antiperiodic)).ravel()
    etas = {j: noise.z4_noise(W.dims, W.noise_seed, j, LEVEL).ravel() for j in SAMPLED}
    want_M = {j: op(etas[j]) for j in SAMPLED}
    pe = {j: krylov.apply_poly(op, THETA, etas[j]) for j in SAMPLED}
    want_bil = {j: np.vdot(etas[j], pe[j]) for j in SAMPLED}
    # |eta^H (p~ - p) eta| <= ||eta|| ||p~ eta - p eta||: the bound for a normwise error of p(M) eta
    bil_scale = {j: np.linalg.norm(etas[j]) * np.linalg.norm(pe[j]) for j in SAMPLED}
    yield {"ctx": ctx, "W": W, "V": int(np.prod(W.dims)), "etas": etas, "M": want_M, "bil": want_bil,
           "bil_scale": bil_scale}
    mmc.mmc_destroy(ctx)


def _column(mmc, field, prec, nrhs, V, j):
    """Right-hand side j of a device field in the blocked layout [rb][site][c][R]."""
    import torch
    R = mmc.mmc_rhs_block(nrhs)
    rb, r = divmod(j, R)
    dt = torch.float32 if prec == mmc.MMC_F32 else torch.bfloat16
    t = field.view(dt).view(-1, V, 12, R, 2)[rb, :, :, r, :].float().cpu().numpy().astype(np.float64)
    return (t[..., 0] + 1j * t[..., 1]).ravel()


def _set_form(mmc, ctx, prec, form):
    ver, rpt, minb, order, hint = form
    v = {"version": ver, "rpt": rpt, "minb": minb, "spc": 64, "blocked": order, "ns": 0}
    for rc in (0, 1):
        mmc.mmc_set_step_variant_class(ctx, prec, rc, v)
    mmc.mmc_set_step_variant(ctx, prec, 0, 400 + hint, 0)


def test_column_extraction_matches_unpack(mmc, big):
    """The test's own reading of the device layout agrees with mmc_unpack."""
    ctx, V = big["ctx"], big["V"]
    x = mmc.new_field(ctx, 8, mmc.MMC_F32)
    mmc.mmc_noise(ctx, LEVEL, 0, mmc.MMC_TAG_NOISE, 8, mmc.MMC_F32, x)
    un = mmc.mmc_unpack(ctx, x, 8, mmc.MMC_F32, V)
    for j in (0, 5, 7):
        assert np.array_equal(_column(mmc, x, mmc.MMC_F32, 8, V, j), un[j])
    assert np.array_equal(un[5], big["etas"][5])


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("form", FORMS)
def test_apply_M_full_size(mmc, big, prec, form):
    ctx, V = big["ctx"], big["V"]
    tol = 1e-5 if prec == mmc.MMC_F32 else BF16_BOUND
    _set_form(mmc, ctx, prec, form)
    for nrhs, cols in ((512, SAMPLED), (8, (0, 5))):
        x = mmc.new_field(ctx, nrhs, prec)
        y = mmc.new_field(ctx, nrhs, prec)
        mmc.mmc_noise(ctx, LEVEL, 0, mmc.MMC_TAG_NOISE, nrhs, prec, x)
        mmc.mmc_apply_M(ctx, x, y, nrhs, prec, 0)
        for j in cols:
            got = _column(mmc, y, prec, nrhs, V, j)
            want = big["M"][j]
            assert np.linalg.norm(got - want) / np.linalg.norm(want) < tol, (nrhs, j)
            # element-wise: a single wrong element (an indexing error at one site) must fail too
            assert np.abs(got - want).max() <= tol * np.abs(want).max(), (nrhs, j)
        del x, y


@pytest.mark.parametrize("form", FORMS)
def test_level_samples_full_size(mmc, big, form):
    """Samples eta_j^H p(M) eta_j of a 512-noise level (bilinear epilogue of the chain)."""
    ctx, V = big["ctx"], big["V"]
    _set_form(mmc, ctx, mmc.MMC_F32, form)
    h = mmc.mmc_poly_from_roots(ctx, THETA)
    st = mmc.mmc_trace_level(ctx, h, mmc.MMC_ZERO, mmc.MMC_THETA_ONE, 0, 512, 0, LEVEL, mmc.MMC_F32)
    for j in SAMPLED:
        assert abs(st["samples"][j] - big["bil"][j]) < 1e-5 * big["bil_scale"][j], j


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c4_24x24x24x24_levels.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.slow
@pytest.mark.parametrize("form", [FORMS[0], FORMS[4], FORMS[5], FORMS[7]])
def test_benchmark_levels_full_size(mmc, big, form):
    """The level chains the benchmark runs at 24^4, in FP32 storage, against samples the
    oracle computed once (tests/golden/make_c4_levels.py): p_32 - p_8 over 512 noises,
    p_128 - p_32 over 128 and p_dbl(40 x 8, degree 319) - p_128 over 32, with the oracle's
    roots fed to the library.  Bound per sample: 1e-5 of ||eta|| (||p_hi eta|| + ||p_lo eta||)
    (FP32 storage, Cauchy-Schwarz on a normwise error of the chains' vectors)."""
    ctx = big["ctx"]
    gold = _golden()
    cx = lambda a: np.array([complex(r, i) for r, i in a])
    _set_form(mmc, ctx, mmc.MMC_F32, form)
    h = {name: mmc.mmc_poly_from_roots(ctx, cx(gold["roots"][name])) for name in ("p8", "p32", "p128")}
    h_in = mmc.mmc_poly_from_roots(ctx, cx(gold["roots"]["in"]))
    h_out = mmc.mmc_poly_from_roots(ctx, cx(gold["roots"]["out"]))
    h["dbl"] = mmc.mmc_poly_double(ctx, h_in, h_out)
    assert mmc.mmc_poly_degree(ctx, h["dbl"]) == 319
    for lv in gold["levels"]:
        st = mmc.mmc_trace_level(ctx, h[lv["hi"]], h[lv["lo"]], mmc.MMC_THETA_ONE, 0, lv["n_noise"], 0, lv["level"],
                                 mmc.MMC_F32)
        for smp in lv["samples"]:
            want = complex(*smp["sample"])
            got = st["samples"][smp["j"]]
            assert abs(got - want) <= 1e-5 * smp["scale"], (lv["level"], smp["j"], got, want, smp["scale"])
