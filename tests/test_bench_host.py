"""Host-side arithmetic of the benchmark line, on CPU: the time to a target standard
error at the measured noise proportions and with cost-optimal noise counts (Sec. 9,
multilevel cost function), pinned against a direct root find and a brute-force
constrained minimisation, and the DRAM-traffic table covering every variant of the
fourth step-kernel form the autotuner can pick for the level chains."""
import numpy as np
import pytest
from scipy import optimize

import bench

# three measured steps of a 4-level estimate: sample variances, seconds for the step's
# samples of each level, noises per level (the 8/32/128/512 mix)
VAR = [8.2e4, 3.0e4, 2.5e5, 3.2e5]
SEC = [0.898, 0.349, 0.511, 0.519]
NOISES = [8, 32, 128, 512]
EPS = 165.888


def test_time_at_measured_proportions_by_root_find():
    """Scaling every N_l by one factor k until sum_l var_l / (k N_l) = eps^2 takes k times the
    step's seconds; k found by a root finder, not by the closed form."""
    fixed, _ = bench.time_to_error(VAR, SEC, NOISES, EPS)
    err2 = lambda k: sum(v / (k * n) for v, n in zip(VAR, NOISES)) - EPS ** 2
    k = optimize.brentq(err2, 1e-6, 1e6, xtol=1e-14, rtol=1e-14)
    assert fixed == pytest.approx(k * sum(SEC), rel=1e-10)


def test_cost_optimal_time_by_constrained_minimisation():
    """The cost-optimal time equals the minimum of sum_l N_l c_l (c_l = seconds per sample)
    subject to sum_l var_l / N_l = eps^2 over real N_l > 0, found numerically (SLSQP in
    log N), and never exceeds the time at the measured proportions."""
    fixed, opt = bench.time_to_error(VAR, SEC, NOISES, EPS)
    c = np.array(SEC) / np.array(NOISES)
    v = np.array(VAR)
    cost = lambda z: float(np.sum(np.exp(z) * c))
    con = {"type": "eq", "fun": lambda z: float(np.sum(v * np.exp(-z)) / EPS ** 2 - 1.0)}
    z0 = np.log(np.array(NOISES, dtype=float))
    res = optimize.minimize(cost, z0, constraints=[con], method="SLSQP",
                            options={"ftol": 1e-14, "maxiter": 500})
    assert res.success, res.message
    assert opt == pytest.approx(res.fun, rel=1e-6)
    assert opt <= fixed * (1 + 1e-12)


def test_cost_optimal_equals_fixed_at_optimal_proportions():
    """With the noise counts already in the proportions sqrt(var_l / c_l) (and the seconds
    scaled with the counts), the two times coincide; a level with zero variance adds no
    time to the optimum."""
    c = np.array(SEC) / np.array(NOISES)
    n_opt = np.sqrt(np.array(VAR) / c)
    sec_opt = list(c * n_opt)
    fixed, opt = bench.time_to_error(VAR, sec_opt, list(n_opt), EPS)
    assert opt == pytest.approx(fixed, rel=1e-12)
    _, opt0 = bench.time_to_error(VAR[:3] + [0.0], SEC, NOISES, EPS)
    _, opt3 = bench.time_to_error(VAR[:3], SEC[:3], NOISES[:3], EPS)
    assert opt0 == pytest.approx(opt3, rel=1e-12)


def test_traffic_table_covers_fourth_form_variants():
    """Every register cap (minb 3..6) and site traversal (0..2) of the fourth form the
    autotuner searches for the FP32 level chains has a measured DRAM-traffic entry, each
    between the algorithmic bytes of a site and rhs (96 in + 96 out + links) and twice that."""
    for minb in (3, 4, 5, 6):
        for order in (0, 1, 2):
            tps = bench.TRAFFIC_PER_SITE_RHS.get((4, minb, order, "bilinear", 1))
            assert tps is not None, (minb, order)
            assert 192.0 < tps < 2 * 196.5, (minb, order, tps)
