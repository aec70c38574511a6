"""The relative-variance scan over the polynomial degree (Sec. 4, Eq. 3, Eq. 4, Fig. 1)
through the library against the oracle on 4^4 lattices (eps 0.3, kappa 0.155, three
configurations): the per-noise samples of the unsubtracted estimator (from the
refined solves) and of each subtraction level agree to the solves' tolerance, and the
relative and log-averaged relative variances computed from them agree with the
oracle's formulas applied to the oracle's samples."""
import numpy as np
import pytest

import synth
from oracle import estimator, krylov, noise, wilson

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)
SHAPE = (4, 4, 4, 4, 4, 3)
DEGREES = (2, 5, 10, 20)
SEEDS = (1, 2, 3)
N_NOISE = 12
LEVEL = 7


@pytest.fixture(scope="module")
def mmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_00016_gb300 import mmc as m
    return m


def _oracle_config(seed):
    U = synth.random_gauge(DIMS, 0.3, seed)
    op = lambda v: wilson.apply_M(U, 0.155, v.reshape(SHAPE + v.shape[1:])).reshape(v.shape)
    A = wilson.dense_M(U, 0.155)
    Ainv = np.linalg.inv(A)
    b = noise.z4_noise(DIMS, seed, 0, 0, noise.TAG_GMRES).ravel()
    roots = {d: krylov.gmres_poly_roots(op, b, d + 1) for d in DEGREES}
    etas = [noise.z4_noise(DIMS, seed, j, LEVEL).ravel() for j in range(N_NOISE)]
    ns = np.array([np.vdot(e, Ainv @ e) for e in etas])
    levels = {d: ns - np.array([np.vdot(e, krylov.apply_poly(op, roots[d], e)) for e in etas]) for d in DEGREES}
    return U, roots, ns, levels, np.linalg.norm(Ainv, 2)


def test_degree_scan_matches_oracle(mmc):
    from paper_2402_00016_gb300 import degree_scan
    gpu, orc = [], []
    for seed in SEEDS:
        U, roots, ns, levels, inv_norm = _oracle_config(seed)
        ctx = mmc.mmc_create(DIMS, seed=seed, device=0)
        try:
            mmc.mmc_load_gauge(ctx, U, 0.155, 1)
            res = degree_scan.config_variances(mmc, ctx, DEGREES, N_NOISE, level=LEVEL, roots=roots)
        finally:
            mmc.mmc_destroy(ctx)
        # solves to 1e-10 relative residual: |dx| <= ||M^-1|| 1e-10 ||eta||, so each sample
        # moves by at most ||eta||^2 ||M^-1|| 1e-10
        bound = 12 * 256 * inv_norm * 1.1e-10
        assert np.abs(res["ns"]["samples"] - ns).max() <= bound
        for d in DEGREES:
            assert np.abs(res["levels"][d]["samples"] - levels[d]).max() <= bound, d
        gpu.append(res)
        orc.append({"ns": estimator.stats(ns)["var"], **{d: estimator.stats(levels[d])["var"] for d in DEGREES}})
    rv = degree_scan.relative_variances(gpu, DEGREES)
    vns = [o["ns"] for o in orc]
    for d in DEGREES:
        va = [o[d] for o in orc]
        assert np.isclose(rv[d]["relative"], estimator.relative_variance(va, vns), rtol=1e-6, atol=0)
        assert np.isclose(rv[d]["log_averaged"], estimator.log_averaged_relative_variance(va, vns), rtol=1e-6,
                          atol=0)
    # subtraction with a higher-degree polynomial removes more variance (Fig. 1's falloff)
    assert rv[DEGREES[-1]]["log_averaged"] < rv[DEGREES[0]]["log_averaged"]
