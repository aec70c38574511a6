"""GPU parity of the adaptive multilevel estimate (Sec. 8 stopping by standard
error, Sec. 9 cost-optimal counts) against the oracle's stopping rules applied
to the oracle's own FP64 sample streams, through the C ABI.

Noise counts are integers decided from FP64 variances: they must agree
exactly; means and variances to 1e-10 relative (FP64 chains)."""
import numpy as np
import pytest

import synth
from oracle import estimator, krylov, noise, wilson

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_00016_gb300 import mmc as m
    return m


@pytest.fixture(scope="module")
def setup(mmc):
    dims, kappa, seed = (4, 4, 4, 4), 0.12, 7
    U = synth.random_gauge(dims, 0.5, 1)
    shape = (dims[3], dims[2], dims[1], dims[0], 4, 3)
    op = lambda v: wilson.apply_M(U, kappa, v.reshape(shape + v.shape[1:])).reshape(v.shape)
    ctx = mmc.mmc_create(dims, seed=seed, device=0)
    mmc.mmc_load_gauge(ctx, U, kappa, 1)
    b = noise.z4_noise(dims, seed, 0, 0, noise.TAG_GMRES).ravel()
    roots = {m: krylov.gmres_poly_roots(op, b, m) for m in (12, 6, 3)}
    handles = {m: mmc.mmc_poly_from_roots(ctx, t) for m, t in roots.items()}
    # three levels: p12 - p6, p6 - p3, p3 (most to least accurate)
    pairs = [(12, 6), (6, 3), (3, None)]
    n_max = 60
    streams = []
    for lvl, (hi, lo) in enumerate(pairs, start=1):
        etas = [noise.z4_noise(dims, seed, j, lvl).ravel() for j in range(n_max)]
        A = lambda v, m=hi: krylov.apply_poly(op, roots[m], v)
        B = (lambda v, m=lo: krylov.apply_poly(op, roots[m], v)) if lo else None
        xs, _ = estimator.level_samples(A, B, lambda v: v, etas)
        streams.append(xs)
    levels = [{"hi": handles[hi], "lo": handles[lo] if lo else mmc.MMC_ZERO, "deflate": 0, "level": lvl,
               "n_first": 3 if lvl < 3 else 6, "n_check": 3, "n_max": n_max}
              for lvl, (hi, lo) in enumerate(pairs, start=1)]
    yield mmc, ctx, levels, streams
    mmc.mmc_destroy(ctx)


def _check(stats, streams, counts):
    for st, x, n in zip(stats, streams, counts):
        assert st["n"] == n
        o = estimator.stats(x[:n])
        assert abs(st["mean_re"] - o["mean"].real) <= 1e-10 * max(1.0, abs(o["mean"]))
        assert abs(st["var_re"] - o["var"]) <= 1e-10 * max(1.0, o["var"])


@pytest.mark.parametrize("eps_scale", [0.5, 2.0])
def test_equal_split_counts_match_oracle(setup, eps_scale):
    mmc, ctx, levels, streams = setup
    # a target between the levels' pilot standard errors, so some levels stop early
    se = [estimator.stats(x[:l["n_first"]])["stderr"] for x, l in zip(streams, levels)]
    eps = eps_scale * float(np.median(se)) * np.sqrt(3)
    counts = estimator.equal_split_counts(streams, eps, [l["n_first"] for l in levels],
                                          [l["n_check"] for l in levels], [l["n_max"] for l in levels])
    stats, tot, tse = mmc.mmc_estimate(ctx, levels, mmc.MMC_THETA_ONE, mmc.MMC_F64, mmc.MMC_ZERO, eps,
                                       mmc.MMC_ALLOC_EQUAL)
    _check(stats, streams, counts)
    ref_tot = sum(x[:n].mean().real for x, n in zip(streams, counts))
    assert abs(tot - ref_tot) <= 1e-10 * max(1.0, abs(ref_tot))
    ref_se = np.sqrt(sum(estimator.stats(x[:n])["var"] / n for x, n in zip(streams, counts)))
    assert abs(tse - ref_se) <= 1e-10 * ref_se


def test_cost_optimal_counts_match_oracle(setup):
    mmc, ctx, levels, streams = setup
    costs = [16.0, 7.0, 2.0]  # matvecs per sample: deg p12 + deg p6 = 11 + 5, 5 + 2, 2
    se = [estimator.stats(x[:l["n_first"]])["stderr"] for x, l in zip(streams, levels)]
    eps = float(np.median(se))
    counts = estimator.cost_optimal_counts(streams, costs, eps, [l["n_first"] for l in levels],
                                           [l["n_check"] for l in levels], [l["n_max"] for l in levels])
    stats, _, _ = mmc.mmc_estimate(ctx, levels, mmc.MMC_THETA_ONE, mmc.MMC_F64, mmc.MMC_ZERO, eps,
                                   mmc.MMC_ALLOC_COST, cost=costs)
    _check(stats, streams, counts)


def test_estimate_rejects_bad_arguments(setup):
    mmc, ctx, levels, _ = setup
    bad = [dict(levels[0], n_first=1)]
    with pytest.raises(Exception):
        mmc.mmc_estimate(ctx, bad, mmc.MMC_THETA_ONE, mmc.MMC_F64, mmc.MMC_ZERO, 1.0)
    with pytest.raises(Exception):
        mmc.mmc_estimate(ctx, levels, mmc.MMC_THETA_ONE, mmc.MMC_F64, mmc.MMC_ZERO, 0.0)
    with pytest.raises(Exception):
        mmc.mmc_estimate(ctx, levels, mmc.MMC_THETA_ONE, mmc.MMC_F64, mmc.MMC_ZERO, 1.0, mmc.MMC_ALLOC_COST,
                         cost=[1.0, 0.0, 1.0])
