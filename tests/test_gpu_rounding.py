"""Stochastic rounding of BF16 chain storage (mmc_set_rounding).

1. Element level: M applied to the same BF16 field K times, each application with a
   fresh salt.  With stochastic rounding the mean of the K stored results converges to
   the FP32 result (each element's rounding error has mean zero and variance at most
   ulp^2 / 4, so the mean's error is at most ulp / (2 sqrt K) in RMS); round to nearest
   keeps its error (RMS about ulp / sqrt(12)) however many times it is repeated.
2. Estimator level: a degree-32 chain's samples eta^H p(M) eta over 256 noises at
   16^4 with BF16 storage, against the FP64 chain on the same noises: with stochastic
   rounding the mean difference is zero within 3 standard errors of the differences
   (the bias that round to nearest can carry is what this guards against).  Round to
   nearest is run on the same noises and its mean shift is reported.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_00016_gb300 import mmc as m
    return m


def _bf16_ulp(x):
    """Spacing of BF16 numbers at |x| (8 significant bits)."""
    a = np.maximum(np.abs(x), 1e-30)
    return 2.0 ** (np.floor(np.log2(a)) - 7)


@pytest.mark.parametrize("ver", [1, 2, 4, 5])
def test_stochastic_rounding_is_unbiased_per_element(mmc, ver):
    import torch
    dims = (6, 4, 2, 6)
    V = int(np.prod(dims))
    U = synth.random_gauge(dims, 0.5, 3)
    ctx = mmc.mmc_create(dims, seed=9, device=0)
    try:
        mmc.mmc_load_gauge(ctx, U, 0.13, 1)
        mmc.mmc_set_step_variant(ctx, mmc.MMC_BF16, 1, 100 + ver, 0)
        nrhs = 16
        x = mmc.new_field(ctx, nrhs, mmc.MMC_BF16)
        y = mmc.new_field(ctx, nrhs, mmc.MMC_BF16)
        x32 = mmc.new_field(ctx, nrhs, mmc.MMC_F32)
        y32 = mmc.new_field(ctx, nrhs, mmc.MMC_F32)
        mmc.mmc_noise(ctx, 1, 0, mmc.MMC_TAG_NOISE, nrhs, mmc.MMC_BF16, x)
        mmc.mmc_noise(ctx, 1, 0, mmc.MMC_TAG_NOISE, nrhs, mmc.MMC_F32, x32)  # the same (exact) noise
        mmc.mmc_apply_M(ctx, x32, y32, nrhs, mmc.MMC_F32, 0)
        ref = mmc.mmc_unpack(ctx, y32, nrhs, mmc.MMC_F32, V)
        ulp = np.sqrt(np.mean(_bf16_ulp(ref.real) ** 2 + _bf16_ulp(ref.imag) ** 2) / 2)
        K = 64
        rms = {}
        for mode in (mmc.MMC_ROUND_NEAREST, mmc.MMC_ROUND_STOCHASTIC):
            mmc.mmc_set_rounding(ctx, mode, seed=17)
            acc = np.zeros_like(ref)
            for _ in range(K):
                mmc.mmc_apply_M(ctx, x, y, nrhs, mmc.MMC_BF16, 0)
                torch.cuda.synchronize()
                acc += mmc.mmc_unpack(ctx, y, nrhs, mmc.MMC_BF16, V)
            d = acc / K - ref
            rms[mode] = np.sqrt(np.mean(d.real ** 2 + d.imag ** 2) / 2)
        assert rms[mmc.MMC_ROUND_STOCHASTIC] <= 1.2 * ulp / (2 * np.sqrt(K)), (rms, ulp)
        assert rms[mmc.MMC_ROUND_NEAREST] >= 0.2 * ulp, (rms, ulp)
    finally:
        mmc.mmc_destroy(ctx)


@pytest.mark.slow
def test_stochastic_rounding_keeps_level_unbiased(mmc):
    dims = (16, 16, 16, 16)
    W = synth.WORKLOADS["c3_16x16x16x16"]
    U = synth.random_gauge(dims, W.eps, W.gauge_seed)
    ctx = mmc.mmc_create(dims, seed=W.noise_seed, device=0)
    try:
        mmc.mmc_load_gauge(ctx, U, W.kappa, 1)
        h, _ = mmc.mmc_gmres_poly(ctx, 33)  # degree 32
        n = 256
        ref = mmc.mmc_trace_level(ctx, h, mmc.MMC_ZERO, mmc.MMC_THETA_ONE, 0, n, 0, 5, mmc.MMC_F64)["samples"]
        t = {}
        for mode in (mmc.MMC_ROUND_NEAREST, mmc.MMC_ROUND_STOCHASTIC):
            mmc.mmc_set_rounding(ctx, mode, seed=23)
            got = mmc.mmc_trace_level(ctx, h, mmc.MMC_ZERO, mmc.MMC_THETA_ONE, 0, n, 0, 5, mmc.MMC_BF16)["samples"]
            d = (got - ref).real
            t[mode] = d.mean() / (d.std(ddof=1) / np.sqrt(n))
        print("mean shift of BF16 samples against FP64, in standard errors:", t)
        assert abs(t[mmc.MMC_ROUND_STOCHASTIC]) < 3.0, t
    finally:
        mmc.mmc_destroy(ctx)
