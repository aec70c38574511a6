"""Failure detection through the C ABI, with every fault made on the host side or by
a bounded device wait that is allowed to run out -- nothing traps, faults or hangs
the GPU:

* calls out of order or with a bad handle return MMC_ERR_STATE / MMC_ERR_ARG;
* a NaN planted in a solve's right-hand side returns MMC_ERR_NAN;
* a solve capped at one outer cycle returns MMC_ERR_NOCONV;
* the staged step kernel with its producer told to copy nothing: every wait of its
  compute warps gives up after a short poll bound, the kernel raises its error flag,
  and the next synchronising call returns MMC_ERR_TIMEOUT;
and after each fault the context still gives correct results."""
import numpy as np
import pytest

import synth
from oracle import noise, wilson

pytestmark = pytest.mark.gpu

DIMS = (6, 4, 2, 6)


@pytest.fixture(scope="module")
def mmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_00016_gb300 import mmc as m
    return m


def _ctx(mmc, load=True):
    ctx = mmc.mmc_create(DIMS, seed=5, device=0)
    if load:
        mmc.mmc_load_gauge(ctx, synth.random_gauge(DIMS, 0.5, 11), 0.13, 1)
    return ctx


def _check_M(mmc, ctx, prec=1, nrhs=5):
    """The context still applies M correctly (FP32 storage, 1e-5)."""
    V = int(np.prod(DIMS))
    U = synth.random_gauge(DIMS, 0.5, 11)
    x = mmc.new_field(ctx, nrhs, prec)
    y = mmc.new_field(ctx, nrhs, prec)
    mmc.mmc_noise(ctx, 2, 0, mmc.MMC_TAG_NOISE, nrhs, prec, x)
    mmc.mmc_apply_M(ctx, x, y, nrhs, prec, 0)
    got = mmc.mmc_unpack(ctx, y, nrhs, prec, V)
    shape = (DIMS[3], DIMS[2], DIMS[1], DIMS[0], 4, 3)
    for j in range(nrhs):
        eta = noise.z4_noise(DIMS, 5, j, 2).ravel()
        want = wilson.apply_M(U, 0.13, eta.reshape(shape), True).ravel()
        assert np.linalg.norm(got[j] - want) / np.linalg.norm(want) < 1e-5


def test_state_and_argument_errors(mmc):
    ctx = _ctx(mmc, load=False)
    try:
        with pytest.raises(mmc.MMCError) as e:
            mmc.mmc_gmres_poly(ctx, 8)
        assert e.value.code == mmc.MMC_ERR_STATE
        mmc.mmc_load_gauge(ctx, synth.random_gauge(DIMS, 0.5, 11), 0.13, 1)
        x = mmc.new_field(ctx, 3, 1)
        y = mmc.new_field(ctx, 3, 1)
        with pytest.raises(mmc.MMCError) as e:
            mmc.mmc_apply_poly(ctx, 999, x, y, 3, 1)
        assert e.value.code == mmc.MMC_ERR_ARG
        _check_M(mmc, ctx)
    finally:
        mmc.mmc_destroy(ctx)


def test_nan_and_noconv_in_solves(mmc):
    import torch
    ctx = _ctx(mmc)
    try:
        nrhs = 3
        b = mmc.new_field(ctx, nrhs, mmc.MMC_F64)
        x = mmc.new_field(ctx, nrhs, mmc.MMC_F64)
        mmc.mmc_noise(ctx, 1, 0, mmc.MMC_TAG_NOISE, nrhs, mmc.MMC_F64, b)
        b.view(torch.float64)[123] = float("nan")
        with pytest.raises(mmc.MMCError) as e:
            mmc.mmc_solve(ctx, b, x, nrhs, 1e-10, mmc.MMC_ZERO, mmc.MMC_F32, 8, 50)
        assert e.value.code == mmc.MMC_ERR_NAN
        mmc.mmc_noise(ctx, 1, 0, mmc.MMC_TAG_NOISE, nrhs, mmc.MMC_F64, b)
        x.zero_()
        with pytest.raises(mmc.MMCError) as e:
            mmc.mmc_solve(ctx, b, x, nrhs, 1e-14, mmc.MMC_ZERO, mmc.MMC_F32, 2, 1)
        assert e.value.code == mmc.MMC_ERR_NOCONV
        x.zero_()
        its, rel = mmc.mmc_solve(ctx, b, x, nrhs, 1e-10, mmc.MMC_ZERO, mmc.MMC_F32, 16, 400)
        assert (rel <= 1e-10).all()
        _check_M(mmc, ctx)
    finally:
        mmc.mmc_destroy(ctx)


@pytest.mark.parametrize("prec", [1, 2])
def test_staged_kernel_bounded_wait_gives_up(mmc, prec):
    ctx = _ctx(mmc)
    try:
        mmc.mmc_set_step_variant(ctx, prec, 1, 103, 0)
        theta = np.array([1.0 + 0.5j, 1.0 - 0.5j, 0.6 + 0.0j])
        h = mmc.mmc_poly_from_roots(ctx, theta)
        ok = mmc.mmc_trace_level(ctx, h, mmc.MMC_ZERO, mmc.MMC_THETA_ONE, 0, 19, 0, 3, prec)
        mmc.mmc_test_stall_staged(ctx, 1, 1 << 14)
        with pytest.raises(mmc.MMCError) as e:
            mmc.mmc_trace_level(ctx, h, mmc.MMC_ZERO, mmc.MMC_THETA_ONE, 0, 19, 0, 3, prec)
        assert e.value.code == mmc.MMC_ERR_TIMEOUT
        mmc.mmc_test_stall_staged(ctx, 0, 0)
        again = mmc.mmc_trace_level(ctx, h, mmc.MMC_ZERO, mmc.MMC_THETA_ONE, 0, 19, 0, 3, prec)
        assert np.array_equal(ok["samples"], again["samples"])
        _check_M(mmc, ctx)
    finally:
        mmc.mmc_destroy(ctx)
