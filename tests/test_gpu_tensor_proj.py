"""Tensor-core (tcgen05) deflation projections of BF16 levels (Sec. 7) against
the CUDA-core path.  The deflation vectors are given BF16-exact entries
(multiples of 1/16 in [-1, 1]) and the noise is exact too, so the BF16 GEMM
with FP32 accumulation is exact (every partial sum is a dyadic number far
below 2^24 / 16): both paths must give the same deflated samples and the same
correction up to the rounding of the FP64 bookkeeping.  Several M tiles and a
ragged tail (70 noises), both insertions Theta = 1 and gamma_4."""
import numpy as np
import pytest

import synth
from oracle import krylov, noise, wilson

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 2, 6)


@pytest.fixture(scope="module")
def mmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_00016_gb300 import mmc as m
    return m


@pytest.mark.parametrize("theta", [0, 1])
def test_tensor_core_projections_match_cuda_cores(mmc, theta):
    U = synth.random_gauge(DIMS, 0.5, 1)
    V = int(np.prod(DIMS))
    ctx = mmc.mmc_create(DIMS, seed=6, device=0)
    try:
        mmc.mmc_load_gauge(ctx, U, 0.13, 1)
        shape = (6, 2, 4, 4, 4, 3)
        op = lambda v: wilson.apply_M(U, 0.13, v.reshape(shape)).ravel()
        b = noise.z4_noise(DIMS, 6, 0, 0, noise.TAG_GMRES).ravel()
        h1 = mmc.mmc_poly_from_roots(ctx, krylov.gmres_poly_roots(op, b, 8))
        h2 = mmc.mmc_poly_from_roots(ctx, krylov.gmres_poly_roots(op, b, 3))
        rng = np.random.default_rng(3)
        k = 5
        q = lambda: rng.integers(-16, 17, size=(k, 12 * V)) / 16.0
        Z = q() + 1j * q()
        W = q() + 1j * q()
        lam = np.array([0.3 + 0.1j, 0.3 - 0.1j, 0.5, 0.7 + 0.2j, 0.7 - 0.2j])
        mmc.mmc_set_deflation(ctx, lam, Z, W)
        n = 70
        mmc.mmc_set_tensor_projections(ctx, 1)
        a = mmc.mmc_trace_level(ctx, h1, h2, theta, 1, n, 0, 5, mmc.MMC_BF16)
        mmc.mmc_set_tensor_projections(ctx, 0)
        r = mmc.mmc_trace_level(ctx, h1, h2, theta, 1, n, 0, 5, mmc.MMC_BF16)
        assert a["k_deflated"] == k and r["k_deflated"] == k
        scale = np.abs(r["samples"]).max() + 1.0
        assert np.abs(a["samples"] - r["samples"]).max() < 1e-9 * scale
        corr_a = a["corr_re"] + 1j * a["corr_im"]
        corr_r = r["corr_re"] + 1j * r["corr_im"]
        assert abs(corr_a - corr_r) < 1e-9 * (abs(corr_r) + 1.0)
        # the correction is sum_i c_i u_i^H Theta z_i with the exact vectors
        G = {0: np.eye(4), 1: np.array([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]])}[theta]
        th_z = np.stack([np.einsum("su,xua->xsa", G, z.reshape(V, 4, 3)).ravel() for z in Z])
        c = mmc.mmc_poly_eval(ctx, h1, lam) - mmc.mmc_poly_eval(ctx, h2, lam)
        want = np.sum(c * np.einsum("ij,ij->i", W.conj(), th_z))
        assert abs(corr_a - want) < 1e-9 * (abs(want) + 1.0)
    finally:
        mmc.mmc_destroy(ctx)
