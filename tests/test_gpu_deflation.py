"""GPU parity of deflation (Sec. 7, Sec. 8) against the oracle, through the C ABI.

* mmc_deflate against the oracle's PP-Arnoldi with the same kept-set rules
  (Sec. 8 acceptance, gamma_5 partners, the overlap drop rules), both from the
  oracle's polynomial roots, on a near-critical 2x2x2x4 lattice where the Arnoldi
  run of 150 steps converges the smallest eigenpairs to rounding: eigenvalues to
  1e-10, the rank-one maps z_i u_i^H (independent of the phase of z_i) to 1e-9,
  with the default bound on the left vectors and with a bound of 2 that makes the
  column-norm rule drop two pairs.
* Deflated Monte Carlo levels with the oracle's eigenpairs loaded by
  mmc_set_deflation: FP64 samples and exact correction to 1e-12; FP32 chains with
  the tensor-core (tcgen05, BF16 operands) projections to 1e-5 of the sample
  scale plus the BF16 rounding bound of the projections.
* Deflated solves: the first deflated iterate Z Lambda^-1 U^H b against the
  oracle's deflated_guess (1e-12 from the FP64 vectors, 1e-5 from the FP32
  copies), and the refined solve's residual 1e-10 checked with the oracle's M.
* Probing against the unit-vector sweep on the 8^4 lattice (Sec. 6).
"""
import numpy as np
import pytest

import synth
from oracle import deflation, estimator, gamma, krylov, noise, wilson

pytestmark = pytest.mark.gpu

DIMS = (2, 2, 2, 4)
SHAPE = (4, 2, 2, 2, 4, 3)
EPS, KAPPA, SEED = 0.3, 0.155, 1
M_ARN, K = 150, 16
BF16_UNIT = 2.0 ** -8


@pytest.fixture(scope="module")
def mmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_00016_gb300 import mmc as m
    return m


class Small:
    def __init__(self):
        self.U = synth.random_gauge(DIMS, EPS, 1)
        self.V = int(np.prod(DIMS))
        self.n = 12 * self.V

    def op(self, v):
        return wilson.apply_M(self.U, KAPPA, v.reshape(SHAPE + v.shape[1:])).reshape(v.shape)

    def g5(self, v):
        return wilson.apply_gamma5(v.reshape(SHAPE + v.shape[1:])).reshape(v.shape)

    def theta(self, name):
        G = {"1": np.eye(4), "g4": gamma.GAMMA[3]}[name]
        return lambda v: wilson.apply_gamma(G, v.reshape(SHAPE + v.shape[1:])).reshape(v.shape)


@pytest.fixture(scope="module")
def small():
    s = Small()
    b = noise.z4_noise(DIMS, SEED, 0, 0, noise.TAG_GMRES).ravel()
    s.th = krylov.gmres_poly_roots(s.op, b, 3)  # the PP-Arnoldi polynomial, degree 2
    s.start = noise.z4_noise(DIMS, SEED, 0, 0, noise.TAG_ARNOLDI).ravel()
    s.eig = {mu: deflation.pp_arnoldi_eigenpairs(s.op, s.g5, s.th, s.start, M_ARN, K, max_u=mu)
             for mu in (100.0, 2.0)}
    return s


@pytest.fixture
def ctx(mmc, small):
    c = mmc.mmc_create(DIMS, seed=SEED, device=0)
    mmc.mmc_load_gauge(c, small.U, KAPPA, 1)
    yield c
    mmc.mmc_destroy(c)


def _match(a, b, tol):
    """Indices j(i) with |a_i - b_j(i)| < tol, a bijection (eigenvalue sets in any order)."""
    left = list(range(len(b)))
    out = []
    for x in a:
        d = [abs(x - b[j]) for j in left]
        k = int(np.argmin(d))
        assert d[k] < tol * max(1.0, abs(x)), (x, b[left[k]])
        out.append(left.pop(k))
    return out


@pytest.mark.parametrize("max_u", [100.0, 2.0])
def test_deflate_matches_oracle(mmc, small, ctx, max_u):
    lam_o, Z_o, U_o, res_o = small.eig[max_u]
    assert res_o.max() < 1e-12  # converged: the comparison below is not limited by the Arnoldi variant
    assert len(lam_o) == (16 if max_u == 100.0 else 12)  # the bound of 2 drops two gamma_5 pairs
    h = mmc.mmc_poly_from_roots(ctx, small.th)
    mmc.mmc_set_deflation_bound(ctx, max_u)
    lam = mmc.mmc_deflate(ctx, K, h, M_ARN, 1e-3)
    assert len(lam) == len(lam_o)
    idx = _match(lam, lam_o, 1e-10)
    lam2, Z, U = mmc.mmc_get_deflation(ctx, small.V)
    assert np.array_equal(lam2, lam)
    assert np.abs(U.conj() @ Z.T - np.eye(len(lam))).max() < 1e-10
    rng = np.random.default_rng(4)
    R = rng.standard_normal((small.n, 3)) + 1j * rng.standard_normal((small.n, 3))
    for i, j in enumerate(idx):
        got = np.outer(Z[i], U[i].conj()) @ R
        want = np.outer(Z_o[:, j], U_o[:, j].conj()) @ R
        assert np.abs(got - want).max() < 1e-9 * np.abs(want).max(), i
        assert np.linalg.norm(small.op(Z[i]) - lam[i] * Z[i]) < 1e-10


def _level(mmc, small, ctx, theta_name, prec, eig):
    lam_o, Z_o, U_o, _ = eig
    mmc.mmc_set_deflation(ctx, lam_o, Z_o.T, U_o.T)
    b = noise.z4_noise(DIMS, SEED, 0, 0, noise.TAG_GMRES).ravel()
    t_hi = krylov.gmres_poly_roots(small.op, b, 9)
    h_hi = mmc.mmc_poly_from_roots(ctx, t_hi)
    h_lo = mmc.mmc_poly_from_roots(ctx, small.th)
    n = 21  # two rhs blocks and a ragged tail
    st = mmc.mmc_trace_level(ctx, h_hi, h_lo, mmc.THETA[theta_name], 1, n, 0, 4, prec)
    c = krylov.poly_scalar(t_hi, lam_o) - krylov.poly_scalar(small.th, lam_o)
    etas = [noise.z4_noise(DIMS, SEED, j, 4).ravel() for j in range(n)]
    th = small.theta(theta_name)
    hi = lambda v: krylov.apply_poly(small.op, t_hi, v)
    lo = lambda v: krylov.apply_poly(small.op, small.th, v)
    want, corr = estimator.level_samples(hi, lo, th, etas, defl=(Z_o, U_o), c=c)
    # scales: Cauchy-Schwarz bounds of the undeflated bilinears, and of the deflated part
    scale = np.array([np.linalg.norm(e) * (np.linalg.norm(hi(e)) + np.linalg.norm(lo(e))) for e in etas])
    dscale = np.array([np.sum(np.abs(c) * np.abs([np.vdot(e, th(z)) for z in Z_o.T]) * np.abs(U_o.conj().T @ e))
                       for e in etas])
    cscale = np.sum(np.abs(c) * np.linalg.norm(U_o, axis=0) * np.linalg.norm(Z_o, axis=0))
    return st, want, corr, scale, dscale, cscale


@pytest.mark.parametrize("theta_name", ["1", "g4"])
def test_deflated_level_fp64_with_oracle_pairs(mmc, small, ctx, theta_name):
    st, want, corr, scale, dscale, cscale = _level(mmc, small, ctx, theta_name, mmc.MMC_F64, small.eig[100.0])
    assert st["k_deflated"] == len(small.eig[100.0][0])
    assert np.all(np.abs(st["samples"] - want) <= 1e-12 * (scale + dscale))
    assert abs(st["corr_re"] + 1j * st["corr_im"] - corr) <= 1e-12 * cscale


@pytest.mark.parametrize("theta_name", ["1", "g4"])
def test_deflated_level_tensor_core_projections_vs_oracle(mmc, small, ctx, theta_name):
    """FP32 chains, deflation projections a_i = eta^H Theta z_i and b_i = u_i^H eta as one
    BF16 GEMM on the tensor cores: z_i and u_i are rounded once to BF16 (relative 2^-8 per
    element, the Z(4) noise is exact), so each deflated term c_i a_i b_i moves by at most
    about 2 * 2^-8 |c_i| |a|_1-bound |b|_1-bound; the chain adds 1e-5 of the sample scale."""
    mmc.mmc_set_tensor_projections(ctx, 1)
    st, want, corr, scale, dscale, cscale = _level(mmc, small, ctx, theta_name, mmc.MMC_F32, small.eig[100.0])
    # |a_i| and |b_i| are bounded elementwise by sums of |entries|: the BF16 bound per term
    lam_o, Z_o, U_o, _ = small.eig[100.0]
    b = noise.z4_noise(DIMS, SEED, 0, 0, noise.TAG_GMRES).ravel()
    t_hi = krylov.gmres_poly_roots(small.op, b, 9)
    c = krylov.poly_scalar(t_hi, lam_o) - krylov.poly_scalar(small.th, lam_o)
    l1 = np.sum(np.abs(c) * np.sum(np.abs(Z_o), axis=0) * np.sum(np.abs(U_o), axis=0))
    bound = 1e-5 * scale + 2.5 * BF16_UNIT * l1
    err = np.abs(st["samples"] - want)
    assert np.all(err <= bound), (err.max(), bound.min())
    cbound = 2.5 * BF16_UNIT * np.sum(np.abs(c) * np.sum(np.abs(U_o) * np.abs(Z_o), axis=0))
    assert abs(st["corr_re"] + 1j * st["corr_im"] - corr) <= cbound + 1e-12 * cscale


@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_deflated_solve(mmc, small, ctx, inner):
    """mmc_solve with deflation data: its first iterate x = Z Lambda^-1 U^H b (oblique
    projection of Sec. 8's deflated solves) against the oracle, then the refined solve."""
    import torch
    lam_o, Z_o, U_o, _ = small.eig[100.0]
    mmc.mmc_set_deflation(ctx, lam_o, Z_o.T, U_o.T)
    prec_inner = mmc.PREC[inner]
    nrhs = 3
    b = mmc.new_field(ctx, nrhs, mmc.MMC_F64)
    x = mmc.new_field(ctx, nrhs, mmc.MMC_F64)
    mmc.mmc_noise(ctx, 6, 0, mmc.MMC_TAG_NOISE, nrhs, mmc.MMC_F64, b)
    x.zero_()
    with pytest.raises(mmc.MMCError) as e:  # no outer cycle allowed: the deflated guess alone
        mmc.mmc_solve(ctx, b, x, nrhs, 1e-10, mmc.MMC_ZERO, prec_inner, 8, 0)
    assert e.value.code == mmc.MMC_ERR_NOCONV
    torch.cuda.synchronize()
    xs = mmc.mmc_unpack(ctx, x, nrhs, mmc.MMC_F64, small.V)
    guess = deflation.deflated_guess(Z_o, U_o, lam_o)
    tol = 1e-12 if inner == "f64" else 1e-5
    for j in range(nrhs):
        want = guess(noise.z4_noise(DIMS, SEED, j, 6).ravel())
        assert np.linalg.norm(xs[j] - want) <= tol * np.linalg.norm(want), j
        assert np.abs(xs[j] - want).max() <= tol * np.abs(want).max(), j
    x.zero_()
    its, rel = mmc.mmc_solve(ctx, b, x, nrhs, 1e-10, mmc.MMC_ZERO, prec_inner, 16, 200)
    xs = mmc.mmc_unpack(ctx, x, nrhs, mmc.MMC_F64, small.V)
    for j in range(nrhs):
        e = noise.z4_noise(DIMS, SEED, j, 6).ravel()
        assert np.linalg.norm(e - small.op(xs[j])) <= 1.05e-10 * np.linalg.norm(e), j


def test_probing_equals_unit_sweep_8x4(mmc):
    """Tr(Theta p(M)) by probing (256 colours for the degree-6 polynomial) equals the sum
    over all 12 V unit vectors on the 8^4 lattice (eps 0.3, kappa 0.155), FP64, 1e-12."""
    dims = (8, 8, 8, 8)
    U = synth.random_gauge(dims, 0.3, 1)
    c = mmc.mmc_create(dims, seed=1, device=0)
    try:
        mmc.mmc_load_gauge(c, U, 0.155, 1)
        theta = mmc.mmc_leja_order(1.0 + 0.6 * np.exp(2j * np.pi * (np.arange(7) + 0.5) / 7))
        h = mmc.mmc_poly_from_roots(c, theta)
        assert mmc.mmc_probe_colours(c, 6) == 256
        scale = None
        for th in (mmc.MMC_THETA_ONE, mmc.MMC_THETA_G4):
            unit = mmc.mmc_trace_exact(c, h, th, mmc.MMC_EXACT_UNIT, mmc.MMC_F64)
            probe = mmc.mmc_trace_exact(c, h, th, mmc.MMC_EXACT_PROBE, mmc.MMC_F64)
            scale = abs(unit) if scale is None else scale  # |Tr p(M)|: the scale of both traces
            assert abs(probe - unit) <= 1e-12 * scale, (th, probe, unit)
    finally:
        mmc.mmc_destroy(c)


def test_deflated_double_polynomial_matches_oracle(mmc, small, ctx):
    """The deflated double polynomial (reading of Sec. 7 / Sec. 9): the outer GMRES cycle
    on phi_in(M) from the start vector without the deflated components gives the oracle's
    harmonic Ritz values (1e-9, m_out = 4), and the deflated top level
    Tr(M^-1 - p_dbl) samples with c_i = 1/lambda_i - p_dbl(lambda_i) match the oracle's
    (dense inverse) within the solves' 1e-10 residual, with the exact correction to 1e-12."""
    lam_o, Z_o, U_o, _ = small.eig[100.0]
    mmc.mmc_set_deflation(ctx, lam_o, Z_o.T, U_o.T)
    b = noise.z4_noise(DIMS, SEED, 0, 0, noise.TAG_GMRES).ravel()
    t_in, t_out = deflation.deflated_double_poly_roots(small.op, b, 5, 4, Z_o, U_o)
    h_in = mmc.mmc_poly_from_roots(ctx, t_in)
    h_out, got_out = mmc.mmc_gmres_poly_deflated(ctx, 4, h_in)
    assert np.abs(got_out - t_out).max() < 1e-9 * np.abs(t_out).max(), (got_out, t_out)
    h_dbl = mmc.mmc_poly_double(ctx, h_in, mmc.mmc_poly_from_roots(ctx, t_out))
    h_pre = mmc.mmc_poly_from_roots(ctx, small.th)
    n = 5
    st = mmc.mmc_trace_level(ctx, mmc.MMC_INV, h_dbl, mmc.MMC_THETA_ONE, 1, n, 0, 8, mmc.MMC_F64, precond=h_pre)
    A = wilson.dense_M(small.U, KAPPA)
    Ainv = np.linalg.inv(A)
    c = 1.0 / lam_o - krylov.double_scalar(t_in, t_out, lam_o)
    etas = [noise.z4_noise(DIMS, SEED, j, 8).ravel() for j in range(n)]
    want, corr = estimator.level_samples(lambda v: Ainv @ v, lambda v: krylov.apply_double(small.op, t_in, t_out, v),
                                         lambda v: v, etas, defl=(Z_o, U_o), c=c)
    inv_norm = np.linalg.norm(Ainv, 2)
    bound = small.n * inv_norm * 1.1e-10 + 1e-12 * np.abs(want).max()
    assert st["k_deflated"] == len(lam_o)
    assert np.abs(st["samples"] - want).max() <= bound, (np.abs(st["samples"] - want).max(), bound)
    cscale = np.sum(np.abs(c) * np.linalg.norm(U_o, axis=0) * np.linalg.norm(Z_o, axis=0))
    assert abs(st["corr_re"] + 1j * st["corr_im"] - corr) <= 1e-12 * cscale
