"""GPU parity of the estimator path against the oracle, through the C ABI:
Monte Carlo level samples (Eq. 2, Sec. 6) for polynomial differences in FP64,
FP32 and BF16 storage, the M^-1 level through refined solves (Sec. 1, Sec. 8),
PP-Arnoldi deflation and deflated levels with their exact correction
(Sec. 7, Sec. 8), and exact traces by unit vectors and probing (Sec. 6).

Tolerances: FP64 1e-12 relative; FP32 1e-5; solves 1e-10 relative residual;
BF16-storage level samples: each polynomial step rounds the iterate to an
8-bit significand (unit 2^-8), so a degree-d chain carries a relative error
of about d * 2^-8 amplified by the growth of the Leja products; the bound
written here, 0.05 of the sample scale for d <= 20, is what that leaves
with a safety factor of 2 over the measured worst case."""
import numpy as np
import pytest

import synth
from oracle import deflation, estimator, gamma, krylov, noise, wilson

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_00016_gb300 import mmc as m
    return m


class Lat:
    def __init__(self, mmc, dims, eps, kappa, seed=5, gauge_seed=1):
        self.dims, self.kappa, self.seed = dims, kappa, seed
        self.U = synth.random_gauge(dims, eps, gauge_seed)
        self.V = int(np.prod(dims))
        self.shape = (dims[3], dims[2], dims[1], dims[0], 4, 3)
        self.ctx = mmc.mmc_create(dims, seed=seed, device=0)
        mmc.mmc_load_gauge(self.ctx, self.U, kappa, 1)

    def op(self, v):
        sh = self.shape + v.shape[1:]
        return wilson.apply_M(self.U, self.kappa, v.reshape(sh)).reshape(v.shape)

    def theta(self, name):
        G = {"1": np.eye(4), "g4": gamma.GAMMA[3], "g5": gamma.GAMMA5}[name]
        return lambda v: wilson.apply_gamma(G, v.reshape(self.shape + v.shape[1:])).reshape(v.shape)

    def eta(self, j, level):
        return noise.z4_noise(self.dims, self.seed, j, level).ravel()


@pytest.fixture(scope="module")
def lat(mmc):
    L = Lat(mmc, (4, 4, 2, 6), 0.5, 0.13)
    yield L
    mmc.mmc_destroy(L.ctx)


def _oracle_samples(L, hi, lo, theta_name, n, level, first=0):
    th = L.theta(theta_name)
    out = []
    for j in range(first, first + n):
        e = L.eta(j, level)
        v = hi(e) - (lo(e) if lo is not None else 0)
        out.append((np.vdot(e, th(v)), abs(np.vdot(e, th(hi(e)))) + (abs(np.vdot(e, th(lo(e)))) if lo else 0)))
    return np.array([o[0] for o in out]), np.array([o[1] for o in out])


@pytest.mark.parametrize("ver,blocked", [(1, 0), (2, 0), (2, 1), (3, 0), (4, 0), (4, 1), (5, 0), (5, 1)])
@pytest.mark.parametrize("theta_name", ["1", "g4"])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5), (2, 5e-2)])
def test_level_poly_difference(mmc, lat, theta_name, prec, tol, ver, blocked):
    if prec == 0 and ver >= 2:
        pytest.skip("FP64 uses the generic kernel only")
    mmc.mmc_set_step_variant(lat.ctx, prec, 0, 100 + ver, 0)
    mmc.mmc_set_step_variant(lat.ctx, prec, 0, 200 + blocked, 0)  # 4x4x2x2 blocks divide this 4x4x2x6 lattice
    try:
        _level_poly_difference(mmc, lat, theta_name, prec, tol)
    finally:
        mmc.mmc_set_step_variant(lat.ctx, prec, 0, 100 + (1 if prec == 0 else 2), 0)
        mmc.mmc_set_step_variant(lat.ctx, prec, 0, 200, 0)


def _level_poly_difference(mmc, lat, theta_name, prec, tol):
    b = noise.z4_noise(lat.dims, lat.seed, 0, 0, noise.TAG_GMRES).ravel()
    t1 = krylov.gmres_poly_roots(lat.op, b, 14)
    t2 = krylov.gmres_poly_roots(lat.op, b, 5)
    h1 = mmc.mmc_poly_from_roots(lat.ctx, t1)
    h2 = mmc.mmc_poly_from_roots(lat.ctx, t2)
    n = 19  # two rhs blocks and a ragged tail
    st = mmc.mmc_trace_level(lat.ctx, h1, h2, mmc.THETA[theta_name], 0, n, 0, 3, prec)
    want, scale = _oracle_samples(lat, lambda v: krylov.apply_poly(lat.op, t1, v),
                                  lambda v: krylov.apply_poly(lat.op, t2, v), theta_name, n, 3)
    err = np.abs(st["samples"] - want) / scale
    assert err.max() < tol, err.max()
    assert st["n"] == n and st["k_deflated"] == 0
    assert np.isclose(st["mean_re"], want.real.mean(), rtol=0, atol=tol * scale.max())


def test_level_double_poly_vs_zero(mmc, lat):
    b = noise.z4_noise(lat.dims, lat.seed, 0, 0, noise.TAG_GMRES).ravel()
    hi_in, _ = mmc.mmc_gmres_poly(lat.ctx, 4)
    hi_out, _ = mmc.mmc_gmres_poly(lat.ctx, 3, hi_in)
    hd = mmc.mmc_poly_double(lat.ctx, hi_in, hi_out)
    tin, tout = krylov.double_poly_roots(lat.op, b, 4, 3)
    n = 5
    st = mmc.mmc_trace_level(lat.ctx, hd, mmc.MMC_ZERO, mmc.MMC_THETA_ONE, 0, n, 2, 9, mmc.MMC_F64)
    want, scale = _oracle_samples(lat, lambda v: krylov.apply_double(lat.op, tin, tout, v), None, "1", n, 9, first=2)
    assert (np.abs(st["samples"] - want) / scale).max() < 1e-11


@pytest.mark.parametrize("sched", [(1.0, 1), (3e-2, 8), (1e-3, 8)])
def test_solve_refined(mmc, lat, sched):
    """Inner FP32 FGMRES with FP64 defect correction reaches 1e-10 (residual checked by the
    oracle's M) with every schedule of the FP32 stage: one cycle per FP64 residual, and
    restarts from the FP32 residual until it has gained 3e-2 or 1e-3."""
    nrhs = 3
    b = mmc.new_field(lat.ctx, nrhs, 0)
    x = mmc.new_field(lat.ctx, nrhs, 0)
    mmc.mmc_noise(lat.ctx, 1, 0, mmc.MMC_TAG_NOISE, nrhs, 0, b)
    hp, _ = mmc.mmc_gmres_poly(lat.ctx, 6)
    mmc.mmc_set_solve_refinement(lat.ctx, *sched)
    try:
        for pre in (mmc.MMC_ZERO, hp):
            x.zero_()
            its, rel = mmc.mmc_solve(lat.ctx, b, x, nrhs, 1e-10, pre, mmc.MMC_F32, 24, 100)
            xs = mmc.mmc_unpack(lat.ctx, x, nrhs, 0, lat.V)
            for j in range(nrhs):
                e = lat.eta(j, 1)
                r = np.linalg.norm(e - lat.op(xs[j])) / np.linalg.norm(e)
                assert r <= 1.05e-10, r
                assert rel[j] <= 1e-10
        for bad in ((0.0, 8), (1.5, 8), (0.1, 0), (0.1, 65)):
            with pytest.raises(mmc.MMCError):
                mmc.mmc_set_solve_refinement(lat.ctx, *bad)
    finally:
        mmc.mmc_set_solve_refinement(lat.ctx, 3e-2, 8)


@pytest.mark.parametrize("passes", [1, 2])
def test_solve_gram_schmidt_passes(mmc, lat, passes):
    """The FP32 stage with one (the default) or two Gram-Schmidt passes per Arnoldi step
    reaches the 1e-10 residual (checked with the oracle's M); 1 and 2 are the only pass
    counts."""
    nrhs = 8
    b = mmc.new_field(lat.ctx, nrhs, 0)
    x = mmc.new_field(lat.ctx, nrhs, 0)
    mmc.mmc_noise(lat.ctx, 8, 0, mmc.MMC_TAG_NOISE, nrhs, 0, b)
    hp, _ = mmc.mmc_gmres_poly(lat.ctx, 6)
    mmc.mmc_set_gram_schmidt(lat.ctx, passes)
    try:
        its, rel = mmc.mmc_solve(lat.ctx, b, x, nrhs, 1e-10, hp, mmc.MMC_F32, 8, 200)
        xs = mmc.mmc_unpack(lat.ctx, x, nrhs, 0, lat.V)
        for j in range(nrhs):
            e = lat.eta(j, 8)
            assert np.linalg.norm(e - lat.op(xs[j])) <= 1.05e-10 * np.linalg.norm(e), j
        for bad in (0, 3):
            with pytest.raises(mmc.MMCError):
                mmc.mmc_set_gram_schmidt(lat.ctx, bad)
    finally:
        mmc.mmc_set_gram_schmidt(lat.ctx, 1)


@pytest.mark.parametrize("minb", [3, 5])
def test_solve_8rhs_fourth_form(mmc, lat, minb):
    """Refined solves of 8 vectors (the 8-rhs block class: Horner preconditioner chains
    with the aux operand, M) through the fourth kernel form at 168 registers (minb 3) and
    at 128 with its links staged in shared memory (minb 5), the Horner chains in the
    blocked layout (the paired layout runs at 168 registers only): residual 1e-10 checked
    with the oracle's M."""
    nrhs = 8
    v = {"version": 4, "rpt": 1, "minb": minb, "spc": 64, "blocked": 0, "ns": 0}
    mmc.mmc_set_step_variant_class(lat.ctx, mmc.MMC_F32, 0, v)
    mmc.mmc_set_horner_layout(lat.ctx, 0)
    try:
        b = mmc.new_field(lat.ctx, nrhs, 0)
        x = mmc.new_field(lat.ctx, nrhs, 0)
        mmc.mmc_noise(lat.ctx, 7, 0, mmc.MMC_TAG_NOISE, nrhs, 0, b)
        hp, _ = mmc.mmc_gmres_poly(lat.ctx, 6)
        its, rel = mmc.mmc_solve(lat.ctx, b, x, nrhs, 1e-10, hp, mmc.MMC_F32, 8, 200)
        xs = mmc.mmc_unpack(lat.ctx, x, nrhs, 0, lat.V)
        for j in range(nrhs):
            e = lat.eta(j, 7)
            r = np.linalg.norm(e - lat.op(xs[j])) / np.linalg.norm(e)
            assert r <= 1.05e-10, (j, r)
    finally:
        mmc.mmc_set_horner_layout(lat.ctx, 1)
        mmc.mmc_set_step_variant_class(lat.ctx, mmc.MMC_F32, 0, {"version": 2, "rpt": 1, "minb": 4, "spc": 64,
                                                                 "blocked": 0, "ns": 0})


@pytest.mark.parametrize("minb", [3, 6])
def test_solve_horner_paired_layout(mmc, lat, minb):
    """The paired-component layout of the solves' Horner chains (FP32, 8-rhs blocks, fourth
    kernel form with whole or rebuilt links) against the blocked layout, for a full block of
    8 vectors and a padded one of 5: the same iteration counts and the same solutions (the
    arithmetic is the same; a misplaced component would change the preconditioner and with
    it the iterations), each at residual 1e-10 with the oracle's M."""
    v = {"version": 4, "rpt": 1, "minb": minb, "spc": 64, "blocked": 0, "ns": 0}
    mmc.mmc_set_step_variant_class(lat.ctx, mmc.MMC_F32, 0, v)
    try:
        hp, _ = mmc.mmc_gmres_poly(lat.ctx, 6)
        for nrhs in (8, 5):
            out = []
            for paired in (0, 1):
                mmc.mmc_set_horner_layout(lat.ctx, paired)
                b = mmc.new_field(lat.ctx, nrhs, 0)
                x = mmc.new_field(lat.ctx, nrhs, 0)
                mmc.mmc_noise(lat.ctx, 7, 0, mmc.MMC_TAG_NOISE, nrhs, 0, b)
                its, rel = mmc.mmc_solve(lat.ctx, b, x, nrhs, 1e-10, hp, mmc.MMC_F32, 8, 200)
                out.append((its, mmc.mmc_unpack(lat.ctx, x, nrhs, 0, lat.V)))
            assert out[0][0] == out[1][0], (nrhs, out[0][0], out[1][0])
            for j in range(nrhs):
                d = np.linalg.norm(out[1][1][j] - out[0][1][j]) / np.linalg.norm(out[0][1][j])
                assert d < 1e-12, (nrhs, j, d)
                e = lat.eta(j, 7)
                r = np.linalg.norm(e - lat.op(out[1][1][j])) / np.linalg.norm(e)
                assert r <= 1.05e-10, (nrhs, j, r)
        with pytest.raises(mmc.MMCError):
            mmc.mmc_set_horner_layout(lat.ctx, 2)
    finally:
        mmc.mmc_set_horner_layout(lat.ctx, 1)
        mmc.mmc_set_step_variant_class(lat.ctx, mmc.MMC_F32, 0, {"version": 2, "rpt": 1, "minb": 4, "spc": 64,
                                                                 "blocked": 0, "ns": 0})


@pytest.mark.parametrize("prec,inner", [(0, 1), (1, 1), (1, 2)])
def test_level_inverse_vs_dense(mmc, prec, inner):
    """Tr(M^-1 - p) samples on the 4^4 plain workload (eps 0.5, kappa 0.12) vs a dense solve:
    the FP64 form, and the FP32 form with its solves' inner stage (preconditioner chain
    included) stored in FP32 or BF16, all refined to the same 1e-10 residual."""
    L = Lat(mmc, (4, 4, 4, 4), 0.5, 0.12, seed=0)
    try:
        A = wilson.dense_M(L.U, L.kappa)
        h, th = mmc.mmc_gmres_poly(L.ctx, 16)
        n = 6
        mmc.mmc_set_solve_storage(L.ctx, inner)
        st = mmc.mmc_trace_level(L.ctx, mmc.MMC_INV, h, mmc.MMC_THETA_ONE, 0, n, 0, 0, prec, precond=h)
        for j in range(n):
            e = L.eta(j, 0)
            xinv = np.linalg.solve(A, e)
            pe = krylov.apply_poly(L.op, th, e)
            want = np.vdot(e, xinv) - np.vdot(e, pe)
            # solve to 1e-10 relative residual: |delta x| <= ||A^-1|| 1e-10 ||e||; the FP32
            # subtracted operand p(M) e adds at most 1e-5 ||e|| ||p(M) e|| (Cauchy-Schwarz)
            bound = np.linalg.norm(e) ** 2 * 1e-10 * 10
            if prec != 0:
                bound += 1e-5 * np.linalg.norm(e) * np.linalg.norm(pe)
            assert abs(st["samples"][j] - want) < bound
        with pytest.raises(mmc.MMCError):
            mmc.mmc_set_solve_storage(L.ctx, 0)
    finally:
        mmc.mmc_destroy(L.ctx)


def test_deflation_eigenpairs_and_deflated_level(mmc):
    """Near-critical small lattice: eigenvalues vs dense eig; deflated samples and the
    exact correction vs the oracle using dense eigenvectors of the same eigenvalues."""
    dims = (2, 4, 4, 4)
    L = Lat(mmc, dims, 0.3, 0.155, seed=2)
    try:
        A = wilson.dense_M(L.U, L.kappa)
        lam_all, W = np.linalg.eig(A)
        hp, th = mmc.mmc_gmres_poly(L.ctx, 3)
        lam = mmc.mmc_deflate(L.ctx, 8, hp, 100, 1e-3)
        assert len(lam) >= 4
        idx = []
        for l in lam:
            i = int(np.argmin(np.abs(lam_all - l)))
            assert abs(lam_all[i] - l) < 1e-8
            idx.append(i)
        # oracle deflation data from dense eigenvectors (z u^H is independent of scaling)
        Z = W[:, idx] / np.linalg.norm(W[:, idx], axis=0)
        g5 = L.theta("g5")
        partner = [int(np.argmin(np.abs(lam - np.conj(l)))) for l in lam]
        Wl = np.stack([g5(Z[:, j]) for j in partner], axis=1)
        Ul = deflation.biorthonormalise(Z, Wl)
        b = noise.z4_noise(dims, L.seed, 0, 0, noise.TAG_GMRES).ravel()
        t_hi = krylov.gmres_poly_roots(L.op, b, 10)
        h_hi = mmc.mmc_poly_from_roots(L.ctx, t_hi)
        h_lo = mmc.mmc_poly_from_roots(L.ctx, th)
        n = 7
        st = mmc.mmc_trace_level(L.ctx, h_hi, h_lo, mmc.MMC_THETA_ONE, 1, n, 0, 4, mmc.MMC_F64)
        c = krylov.poly_scalar(t_hi, lam) - krylov.poly_scalar(th, lam)
        etas = [L.eta(j, 4) for j in range(n)]
        want, corr = estimator.level_samples(lambda v: krylov.apply_poly(L.op, t_hi, v),
                                             lambda v: krylov.apply_poly(L.op, th, v), lambda v: v, etas,
                                             defl=(Z, Ul), c=c)
        scale = np.abs(want).max() + 1.0
        assert np.abs(st["samples"] - want).max() < 1e-7 * scale
        assert abs(st["corr_re"] + 1j * st["corr_im"] - corr) < 1e-7 * (abs(corr) + 1)
        assert st["k_deflated"] == len(lam)
    finally:
        mmc.mmc_destroy(L.ctx)


def test_exact_trace_unit_and_probe(mmc):
    dims = (4, 4, 4, 4)
    L = Lat(mmc, dims, 0.5, 0.12, seed=0)
    try:
        b = noise.z4_noise(dims, 0, 0, 0, noise.TAG_GMRES).ravel()
        th = krylov.gmres_poly_roots(L.op, b, 3)  # degree 2
        h = mmc.mmc_poly_from_roots(L.ctx, th)
        n = 12 * 256
        for name in ("1", "g4"):
            ref = estimator.exact_trace_unit(lambda E: krylov.apply_poly(L.op, th, E), L.theta(name), n, 1024)
            got_u = mmc.mmc_trace_exact(L.ctx, h, mmc.THETA[name], mmc.MMC_EXACT_UNIT, mmc.MMC_F64)
            got_p = mmc.mmc_trace_exact(L.ctx, h, mmc.THETA[name], mmc.MMC_EXACT_PROBE, mmc.MMC_F64)
            assert abs(got_u - ref) < 1e-11 * max(1, abs(ref))
            assert abs(got_p - ref) < 1e-11 * max(1, abs(ref))
        ncol = mmc.mmc_probe_colours(L.ctx, 2)
        assert ncol < 256
    finally:
        mmc.mmc_destroy(L.ctx)


def test_extra_deflation_configuration(mmc):
    """Sec. 8's "extra deflation": PP(70)-Arnoldi (p_in of degree 69) for 150 steps, the 60
    smallest accepted Ritz pairs kept.  Every returned pair is an eigenpair of M to the
    acceptance bound (residual checked with the oracle's M in FP64), the left vectors
    are biorthonormal to the right ones, and the eigenvalues come in gamma_5 partner
    pairs (conjugates, or real)."""
    dims = (8, 8, 8, 8)
    L = Lat(mmc, dims, 0.3, 0.155, seed=3)
    try:
        h69, _ = mmc.mmc_gmres_poly(L.ctx, 70)
        lam = mmc.mmc_deflate(L.ctx, 60, h69, 150, 1e-3)
        assert 10 <= len(lam) <= 60
        lam2, Z, U = mmc.mmc_get_deflation(L.ctx, L.V)
        assert np.allclose(lam2, lam)
        for i in range(len(lam)):
            z = Z[i]
            r = L.op(z) - lam[i] * z
            assert np.linalg.norm(r) / np.linalg.norm(z) < 1e-3
        G = U.conj() @ Z.T
        assert np.abs(G - np.eye(len(lam))).max() < 1e-8
        for l in lam:
            assert np.min(np.abs(lam - np.conj(l))) < 4e-4 + 1e-3 * abs(l)
    finally:
        mmc.mmc_destroy(L.ctx)
