"""Pins for the oracle's estimators: Hutchinson with subtraction (Eq. 2),
multipolynomial levels (Sec. 6), level deflation and its exact correction
(Sec. 7), exact traces by unit vectors and by probing (Sec. 6)."""
import itertools

import numpy as np
import pytest

import synth
from oracle import deflation, estimator, gamma, krylov, noise, wilson


def _all_z4(n):
    vals = np.array([1, 1j, -1, -1j])
    for codes in itertools.product(range(4), repeat=n):
        yield vals[list(codes)]


def test_z4_hutchinson_exact_moments():
    """Averaged over every Z(4) vector: E[x] = Tr A and E|x - Tr A|^2 = sum_{i != j} |A_ij|^2."""
    n = 5
    rng = np.random.default_rng(0)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    etas = list(_all_z4(n))
    xs, corr = estimator.level_samples(lambda v: A @ v, None, lambda v: v, etas)
    assert corr == 0
    assert abs(xs.mean() - np.trace(A)) < 1e-12 * abs(np.trace(A))
    off = np.sum(np.abs(A) ** 2) - np.sum(np.abs(np.diag(A)) ** 2)
    assert abs(np.mean(np.abs(xs - np.trace(A)) ** 2) - off) < 1e-10 * off


def test_deflated_level_is_unbiased_exactly():
    """mean over every Z(4) vector of the deflated samples + correction = Tr(Theta (A - B))."""
    n = 5
    rng = np.random.default_rng(1)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    B = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    T = np.diag([1.0, -1.0, 1.0, 1j, 2.0])
    Z = rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))
    W = rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))
    U = deflation.biorthonormalise(Z, W)
    assert np.abs(U.conj().T @ Z - np.eye(2)).max() < 1e-12
    c = np.array([0.7 - 0.2j, -1.3 + 0.5j])
    etas = list(_all_z4(n))
    xs, corr = estimator.level_samples(lambda v: A @ v, lambda v: B @ v, lambda v: T @ v, etas,
                                       defl=(Z, U), c=c)
    exact = np.trace(T @ (A - B))
    assert abs(xs.mean() + corr - exact) < 1e-12 * abs(exact)
    # the correction is the trace of the deflated part
    D = sum(c[i] * np.outer(Z[:, i], U[:, i].conj()) for i in range(2))
    assert abs(corr - np.trace(T @ D)) < 1e-12


DIMS = (2, 2, 4, 4)
SHAPE = (4, 4, 2, 2, 4, 3)


@pytest.fixture(scope="module")
def lattice():
    U = synth.random_gauge(DIMS, 0.5, 1)
    kappa = 0.12
    op = lambda v: wilson.apply_M(U, kappa, v.reshape(SHAPE + v.shape[1:])).reshape(v.shape)
    g5 = lambda v: wilson.apply_gamma5(v.reshape(SHAPE + v.shape[1:])).reshape(v.shape)
    A = wilson.dense_M(U, kappa)
    lam, W = np.linalg.eig(A)
    return U, kappa, op, g5, A, lam, W


def test_deflated_difference_annihilates_eigenvectors(lattice):
    """(p1 - p2 - sum_i c_i z_i u_i^H) z_j = 0 and u_j^H (...) = 0 for exact eigenpairs (Sec. 7)."""
    U, kappa, op, g5, A, lam, W = lattice
    b = noise.z4_noise(DIMS, 0, 0, 0, noise.TAG_GMRES).ravel()
    th1 = krylov.gmres_poly_roots(op, b, 12)
    th2 = krylov.gmres_poly_roots(op, b, 4)
    idx = np.argsort(np.abs(lam))[:6]
    Z = W[:, idx] / np.linalg.norm(W[:, idx], axis=0)
    # left vectors from gamma5-hermiticity: gamma5 z_j is left for conj(lambda_j)
    partner = [int(np.argmin(np.abs(lam[idx] - np.conj(l)))) for l in lam[idx]]
    Wl = np.stack([g5(Z[:, j]) for j in partner], axis=1)
    Ul = deflation.biorthonormalise(Z, Wl)
    for i in range(6):
        assert np.linalg.norm(Ul[:, i].conj() @ A - lam[idx][i] * Ul[:, i].conj()) < 1e-9 * np.linalg.norm(Ul[:, i])
    c = krylov.poly_scalar(th1, lam[idx]) - krylov.poly_scalar(th2, lam[idx])
    n = A.shape[0]
    P1 = np.stack([krylov.apply_poly(op, th1, e) for e in np.eye(n)], axis=1)
    P2 = np.stack([krylov.apply_poly(op, th2, e) for e in np.eye(n)], axis=1)
    D = P1 - P2 - (Z * c) @ Ul.conj().T
    assert np.linalg.norm(D @ Z) < 1e-9 * np.linalg.norm(P1 - P2)
    assert np.linalg.norm(Ul.conj().T @ D) < 1e-9 * np.linalg.norm(P1 - P2)


@pytest.mark.parametrize("m_poly", [3, 6])
def test_pp_arnoldi_eigenpairs_match_dense(m_poly):
    """Near-critical lattice (spectrum around the origin): eigenpairs vs dense eig."""
    dims, shape = (2, 4, 4, 4), (4, 4, 4, 2, 4, 3)
    U = synth.random_gauge(dims, 0.3, 1)
    op = lambda v: wilson.apply_M(U, 0.155, v.reshape(shape + v.shape[1:])).reshape(v.shape)
    g5 = lambda v: wilson.apply_gamma5(v.reshape(shape + v.shape[1:])).reshape(v.shape)
    A = wilson.dense_M(U, 0.155)
    lam = np.linalg.eigvals(A)
    b = noise.z4_noise(dims, 0, 0, 0, noise.TAG_GMRES).ravel()
    th = krylov.gmres_poly_roots(op, b, m_poly)
    start = noise.z4_noise(dims, 0, 0, 0, noise.TAG_ARNOLDI).ravel()
    lam_d, Z, Ul, res = deflation.pp_arnoldi_eigenpairs(op, g5, th, start, 100, 8)
    assert len(lam_d) >= 4
    assert np.abs(Ul.conj().T @ Z - np.eye(len(lam_d))).max() < 1e-10
    for l, z in zip(lam_d, Z.T):
        assert np.min(np.abs(lam - l)) < 1e-6
        assert np.linalg.norm(A @ z - l * z) < 1e-3
    # they are the smallest in modulus
    smallest = np.sort(np.abs(lam))[: len(lam_d)]
    assert np.max(np.abs(lam_d)) <= smallest[-1] * 1.5


def test_exact_trace_unit_vectors_vs_eigenvalues(lattice):
    """Tr(p(M)) = sum_i p(lambda_i), Tr(gamma4 p(M)) against the dense matrix polynomial."""
    U, kappa, op, g5, A, lam, W = lattice
    b = noise.z4_noise(DIMS, 0, 0, 0, noise.TAG_GMRES).ravel()
    th = krylov.gmres_poly_roots(op, b, 6)
    n = A.shape[0]
    tr = estimator.exact_trace_unit(lambda E: krylov.apply_poly(op, th, E), lambda v: v, n)
    assert abs(tr - np.sum(krylov.poly_scalar(th, lam))) < 1e-9 * abs(tr)
    G4 = np.kron(np.eye(n // 12), np.kron(gamma.GAMMA[3], np.eye(3)))
    pA = (W * krylov.poly_scalar(th, lam)) @ np.linalg.inv(W)
    tr4 = estimator.exact_trace_unit(lambda E: krylov.apply_poly(op, th, E), lambda v: G4 @ v, n)
    assert abs(tr4 - np.trace(G4 @ pA)) < 1e-9 * max(1, abs(tr4))


def _greedy_colouring(dims, reach):
    lx, ly, lz, lt = dims
    coords = np.array([(x, y, z, t) for t in range(lt) for z in range(lz) for y in range(ly) for x in range(lx)])
    L = np.array(dims)
    col = -np.ones(len(coords), dtype=int)
    for s, c in enumerate(coords):
        d = np.abs(coords - c)
        d = np.minimum(d, L - d).sum(axis=1)
        used = set(col[(d <= reach) & (col >= 0)])
        k = 0
        while k in used:
            k += 1
        col[s] = k
    return col


def test_probing_equals_unit_sweep():
    dims = (4, 4, 4, 4)
    shape = (4, 4, 4, 4, 4, 3)
    U = synth.random_gauge(dims, 0.5, 1)
    op = lambda v: wilson.apply_M(U, 0.12, v.reshape(shape + v.shape[1:])).reshape(v.shape)
    b = noise.z4_noise(dims, 0, 0, 0, noise.TAG_GMRES).ravel()
    th = krylov.gmres_poly_roots(op, b, 3)          # degree 2: couples sites within L1 distance 2
    g4 = lambda v: wilson.apply_gamma(gamma.GAMMA[3], v.reshape(shape + v.shape[1:])).reshape(v.shape)
    col = _greedy_colouring(dims, 2)
    ncol = col.max() + 1
    assert ncol < 256
    pmap = lambda E: krylov.apply_poly(op, th, E)
    n = 12 * 256
    for theta in (lambda v: v, g4):
        ref = estimator.exact_trace_unit(pmap, theta, n, batch=512)
        pr = estimator.exact_trace_probing(pmap, theta, col, ncol)
        assert abs(pr - ref) < 1e-10 * max(1.0, abs(ref))
    # a colouring that separates only distance 1 is not exact for degree 2
    bad = _greedy_colouring(dims, 1)
    pr_bad = estimator.exact_trace_probing(pmap, lambda v: v, bad, bad.max() + 1)
    ref = estimator.exact_trace_unit(pmap, lambda v: v, n, batch=512)
    assert abs(pr_bad - ref) > 1e-6


def test_c1_plain_mmc_vs_dense_lu():
    """4^4, eps 0.5, kappa 0.12: Tr(M^-1 - p) by 32 noises + exact Tr(p) within 5 sigma of dense LU."""
    dims = (4, 4, 4, 4)
    shape = (4, 4, 4, 4, 4, 3)
    U = synth.random_gauge(dims, 0.5, 1)
    kappa = 0.12
    op = lambda v: wilson.apply_M(U, kappa, v.reshape(shape + v.shape[1:])).reshape(v.shape)
    A = wilson.dense_M(U, kappa)
    Ainv = np.linalg.inv(A)
    exact = np.trace(Ainv)
    b = noise.z4_noise(dims, 0, 0, 0, noise.TAG_GMRES).ravel()
    th = krylov.gmres_poly_roots(op, b, 16)
    etas = [noise.z4_noise(dims, 0, j, 0).ravel() for j in range(32)]
    xs, _ = estimator.level_samples(lambda v: Ainv @ v, lambda v: krylov.apply_poly(op, th, v),
                                    lambda v: v, etas)
    st = estimator.stats(xs)
    trp = estimator.exact_trace_unit(lambda E: krylov.apply_poly(op, th, E), lambda v: v, A.shape[0], 1024)
    total = st["mean"] + trp
    assert abs(total.real - exact.real) < 5 * st["stderr"] + 1e-9
    # the subtraction reduces the variance against plain Hutchinson on the same noises
    xs_ns, _ = estimator.level_samples(lambda v: Ainv @ v, None, lambda v: v, etas)
    assert st["var"] < 0.5 * estimator.stats(xs_ns)["var"]


def test_stats_and_relative_variance():
    x = np.array([1.0 + 2j, 3.0 - 1j, -2.0 + 0.5j, 4.0 + 0j])
    s = estimator.stats(x)
    assert np.isclose(s["var"], np.var(x.real, ddof=1))
    assert np.isclose(estimator.stats(x, "im")["var"], np.var(x.imag, ddof=1))
    assert np.isclose(s["stderr"], np.sqrt(np.var(x.real, ddof=1) / 4))
    assert np.isclose(estimator.log_averaged_relative_variance([1e-2, 1e-4], [1.0, 1.0]), 1e-3)
    assert np.isclose(estimator.relative_variance([2.0, 4.0], [6.0, 6.0]), 0.5)


def test_equal_split_stops_at_hand_computed_count():
    # alternating +-1 samples: even n gives stderr 1/sqrt(n-1), odd n gives sqrt(n+1)/n.
    # Target eps / sqrt(L) = 0.25 (L = 1): checks at 3, 6, 9, 12, 15 give 0.667, 0.447,
    # 0.351, 0.302, 0.267; n = 18 gives 0.2425, the first below 0.25.
    x = np.array([(-1.0) ** j for j in range(100)], dtype=np.complex128)
    assert estimator.equal_split_counts([x], 0.25, [3], [3], [100]) == [18]
    # the cap wins, and a zero-variance level stops at its first batch
    assert estimator.equal_split_counts([x], 0.25, [3], [3], [10]) == [10]
    c = np.full(50, 7.0 + 1j)
    assert estimator.equal_split_counts([c, x], 0.25 * np.sqrt(2), [6, 3], [3, 3], [50, 100]) == [6, 18]
    # the imaginary part for gamma_4 levels
    assert estimator.equal_split_counts([1j * x], 0.25, [3], [3], [100], part="im") == [18]
    assert estimator.equal_split_counts([1j * x], 0.25, [3], [3], [100], part="re") == [3]


def test_giles_allocation_minimises_cost():
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(4)
    var = rng.uniform(0.5, 50.0, 4)
    cost = rng.uniform(1.0, 300.0, 4)
    eps = 0.3
    N = estimator.giles_allocation(var, cost, eps)
    assert np.isclose(np.sum(var / N), eps**2, rtol=1e-12)
    # independent check: constrained minimisation of the total cost
    res = scipy_opt.minimize(lambda n: float(np.dot(cost, n)), x0=np.full(4, 500.0),
                             constraints=[{"type": "eq", "fun": lambda n: float(np.sum(var / n) - eps**2)}],
                             bounds=[(1e-3, None)] * 4, method="SLSQP", options={"ftol": 1e-12, "maxiter": 500})
    assert res.success
    assert np.allclose(res.x, N, rtol=1e-3)
    assert np.dot(cost, N) <= np.dot(cost, res.x) * (1 + 1e-9)


def test_cost_optimal_counts_meet_targets():
    # two levels of alternating samples with amplitudes 1 and 3, costs 100 and 1, eps 0.1
    x1 = np.array([(-1.0) ** j for j in range(6000)], dtype=np.complex128)
    x2 = 3.0 * x1
    costs = [100.0, 1.0]
    eps = 0.1
    n = estimator.cost_optimal_counts([x1, x2], costs, eps, [3, 6], [3, 3], [6000, 6000])
    # by hand: pilot variances 4/3 (3 samples) and 9 * 6/5 = 10.8 (6 samples);
    # s = sqrt(400/3) + sqrt(10.8) = 14.83; targets ceil(sqrt(4/300) s / eps^2) = 172 and
    # ceil(sqrt(10.8) s / eps^2) = 4875; shortfalls 169 -> 171 and 4869 (multiples of 3)
    # give 174 and 4875; the second round (variances 174/173 and 9 * 4875/4874) asks for
    # 131 and 3909, below both, so the counts stay
    assert n == [174, 4875]
    var = [estimator.stats(x1[:n[0]])["var"], estimator.stats(x2[:n[1]])["var"]]
    target = np.ceil(estimator.giles_allocation(var, costs, eps))
    assert all(nl >= t for nl, t in zip(n, target))
    assert sum(v / nl for v, nl in zip(var, n)) <= eps**2
