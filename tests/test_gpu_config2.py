"""The full multilevel workload on the 8^4 lattice (eps 0.3, kappa 0.155, FP64),
end to end through the C ABI against the oracle (Sec. 5, Sec. 6, Sec. 7, Sec. 8):

  Tr(Theta (M^-1 - p_dbl))   p_dbl: 20 inner x 10 outer (degree 199), deflated solves
  Tr(Theta (p_dbl - p_50))   deflated by k = 10 eigenpairs
  Tr(Theta (p_50 - p_10))    deflated
  Tr(Theta p_10)             exact (probing; on 8^4 the colouring for reach 10 is the
                             unit-vector sweep, compared with the unit sweep itself)

for Theta = 1 and gamma_4, a few noise vectors per level (the configured 64 would
make the oracle's share of the test minutes long; the samples are per noise).
The polynomials are the oracle's (Leja-ordered harmonic Ritz values of MGS
Arnoldi, fed to the library as roots, since the library's CGS2 Arnoldi agrees
with MGS only to the conditioning of the Ritz problem), and so are the deflation
eigenpairs (the oracle's PP-Arnoldi with the library's kept-set rules, loaded
with mmc_set_deflation).  Polynomial levels agree to 1e-12 of the sample scale;
the M^-1 level to the solves' 1e-10 residual.
"""
import numpy as np
import pytest

import synth
from oracle import deflation, estimator, gamma, krylov, noise, wilson

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

W = synth.WORKLOADS["c2_8x8x8x8"]
SHAPE = (W.dims[3], W.dims[2], W.dims[1], W.dims[0], 4, 3)
N_NOISE = {1: 2, 2: 3, 3: 6}  # per level id


@pytest.fixture(scope="module")
def mmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_00016_gb300 import mmc as m
    return m


@pytest.fixture(scope="module")
def setup(mmc):
    U = synth.random_gauge(W.dims, W.eps, W.gauge_seed)
    op = lambda v: wilson.apply_M(U, W.kappa, v.reshape(SHAPE + v.shape[1:]), True).reshape(v.shape)
    g5 = lambda v: wilson.apply_gamma5(v.reshape(SHAPE + v.shape[1:])).reshape(v.shape)
    b = noise.z4_noise(W.dims, W.noise_seed, 0, 0, noise.TAG_GMRES).ravel()
    tin, tout = krylov.double_poly_roots(op, b, 20, 10)
    t50 = krylov.gmres_poly_roots(op, b, 51)
    t10 = krylov.gmres_poly_roots(op, b, 11)
    start = noise.z4_noise(W.dims, W.noise_seed, 0, 0, noise.TAG_ARNOLDI).ravel()
    lam, Z, Ul, _ = deflation.pp_arnoldi_eigenpairs(op, g5, tin, start, 60, W.deflate_k)
    assert len(lam) >= 6
    ctx = mmc.mmc_create(W.dims, seed=W.noise_seed, device=0)
    mmc.mmc_load_gauge(ctx, U, W.kappa, 1)
    h_in = mmc.mmc_poly_from_roots(ctx, tin)
    h_out = mmc.mmc_poly_from_roots(ctx, tout)
    h = {"dbl": mmc.mmc_poly_double(ctx, h_in, h_out), "p50": mmc.mmc_poly_from_roots(ctx, t50),
         "p10": mmc.mmc_poly_from_roots(ctx, t10)}
    mmc.mmc_set_deflation(ctx, lam, Z.T, Ul.T)
    maps = {"dbl": lambda v: krylov.apply_double(op, tin, tout, v),
            "p50": lambda v: krylov.apply_poly(op, t50, v),
            "p10": lambda v: krylov.apply_poly(op, t10, v)}
    scal = {"dbl": lambda a: krylov.double_scalar(tin, tout, a), "p50": lambda a: krylov.poly_scalar(t50, a),
            "p10": lambda a: krylov.poly_scalar(t10, a)}
    yield {"ctx": ctx, "op": op, "h": h, "maps": maps, "scal": scal, "lam": lam, "Z": Z, "U": Ul, "t10": t10}
    mmc.mmc_destroy(ctx)


def _theta(name):
    G = {"1": np.eye(4), "g4": gamma.GAMMA[3]}[name]
    return lambda v: wilson.apply_gamma(G, v.reshape(SHAPE + v.shape[1:])).reshape(v.shape)


@pytest.mark.parametrize("theta_name", ["1", "g4"])
@pytest.mark.parametrize("hi,lo,level", [("dbl", "p50", 2), ("p50", "p10", 3)])
def test_deflated_polynomial_levels(mmc, setup, theta_name, hi, lo, level):
    s = setup
    n = N_NOISE[level]
    st = mmc.mmc_trace_level(s["ctx"], s["h"][hi], s["h"][lo], mmc.THETA[theta_name], 1, n, 0, level,
                             mmc.MMC_F64)
    th = _theta(theta_name)
    etas = [noise.z4_noise(W.dims, W.noise_seed, j, level).ravel() for j in range(n)]
    c = s["scal"][hi](s["lam"]) - s["scal"][lo](s["lam"])
    want, corr = estimator.level_samples(s["maps"][hi], s["maps"][lo], th, etas, defl=(s["Z"], s["U"]), c=c)
    scale = np.array([np.linalg.norm(e) * (np.linalg.norm(s["maps"][hi](e)) + np.linalg.norm(s["maps"][lo](e)))
                      for e in etas])
    assert st["k_deflated"] == len(s["lam"])
    assert np.all(np.abs(st["samples"] - want) <= 1e-12 * scale), np.abs(st["samples"] - want) / scale
    cscale = np.sum(np.abs(c) * np.linalg.norm(s["U"], axis=0) * np.linalg.norm(s["Z"], axis=0))
    assert abs(st["corr_re"] + 1j * st["corr_im"] - corr) <= 1e-12 * cscale


@pytest.mark.parametrize("theta_name", ["1", "g4"])
def test_inverse_level(mmc, setup, theta_name):
    """Tr(Theta (M^-1 - p_dbl)) samples: the library's deflated, refined FP64 solves against
    the oracle's deflated GMRES to 1e-12; both solves end within their tolerance of
    M^-1 eta, so the samples agree to ||eta|| ||M^-1|| 1e-10 ||eta||.  ||M^-1|| is taken
    as at most 100 (the smallest |lambda| of M here is about 0.18; the bound leaves a
    factor 18 for the non-normality of M)."""
    s = setup
    n = N_NOISE[1]
    hp = s["h"]["p10"]
    st = mmc.mmc_trace_level(s["ctx"], mmc.MMC_INV, s["h"]["dbl"], mmc.THETA[theta_name], 0, n, 0, 1,
                             mmc.MMC_F64, precond=hp)
    th = _theta(theta_name)
    guess = deflation.deflated_guess(s["Z"], s["U"], s["lam"])
    inv_norm = 100.0
    assert np.abs(s["lam"]).min() > 0.1
    for j in range(n):
        e = noise.z4_noise(W.dims, W.noise_seed, j, 1).ravel()
        x, _, _ = krylov.gmres_solve(s["op"], e, tol=1e-12, m=60, deflate=guess)
        want = np.vdot(e, th(x - s["maps"]["dbl"](e)))
        bound = np.linalg.norm(e) ** 2 * inv_norm * 1.1e-10
        assert abs(st["samples"][j] - want) <= bound, (j, abs(st["samples"][j] - want), bound)


def test_exact_last_level(mmc, setup):
    """Tr(p_10) by the library's probing equals its unit-vector sweep (the oracle's own
    unit sweep is checked on 4^4), and the scalar p_10 on the deflation eigenvalues,
    which the level corrections use, equals the oracle's recurrence."""
    s = setup
    probe = mmc.mmc_trace_exact(s["ctx"], s["h"]["p10"], mmc.MMC_THETA_ONE, mmc.MMC_EXACT_PROBE, mmc.MMC_F64)
    unit = mmc.mmc_trace_exact(s["ctx"], s["h"]["p10"], mmc.MMC_THETA_ONE, mmc.MMC_EXACT_UNIT, mmc.MMC_F64)
    assert abs(probe - unit) <= 1e-12 * abs(unit)
    # the scalar recurrence on the deflated eigenvalues is part of the same polynomial
    assert np.allclose(mmc.mmc_poly_eval(s["ctx"], s["h"]["p10"], s["lam"]), krylov.poly_scalar(s["t10"], s["lam"]),
                       rtol=1e-12, atol=0)
