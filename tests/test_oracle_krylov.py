"""Pins for the oracle's GMRES polynomials (Sec. 3), double polynomials
(Sec. 5) and GMRES solves, against dense linear algebra, the GMRES
least-squares residual and brute force."""
import itertools

import numpy as np
import pytest

import synth
from oracle import krylov, noise, wilson

DIMS = (2, 2, 2, 4)
SHAPE = (4, 2, 2, 2, 4, 3)


@pytest.fixture(scope="module")
def system():
    U = synth.random_gauge(DIMS, 0.5, 1)
    kappa = 0.12
    op = lambda v: wilson.apply_M(U, kappa, v.reshape(SHAPE + v.shape[1:])).reshape(v.shape)
    A = wilson.dense_M(U, kappa)
    b = noise.z4_noise(DIMS, 0, 0, 0, noise.TAG_GMRES).ravel()
    return op, A, b


def test_arnoldi_relation(system):
    op, A, b = system
    V, H, beta = krylov.arnoldi(op, b, 12)
    assert np.abs(V.conj().T @ V - np.eye(13)).max() < 1e-12
    assert np.abs(A @ V[:, :12] - V @ H).max() < 1e-13
    assert np.allclose(np.tril(H, -2), 0)


def test_harmonic_ritz_are_gmres_residual_roots(system):
    """GMRES(m) residual b - M x_m (x_m from the Hessenberg least squares) equals pi(M) b."""
    op, A, b = system
    m = 10
    V, H, beta = krylov.arnoldi(op, b, m)
    e1 = np.zeros(m + 1, dtype=complex)
    e1[0] = beta
    y, *_ = np.linalg.lstsq(H, e1, rcond=None)
    r = b - A @ (V[:, :m] @ y)
    theta = krylov.leja_order(krylov.harmonic_ritz(H))
    assert np.linalg.norm(r - krylov.apply_pi(op, theta, b)) < 1e-10 * np.linalg.norm(r)


def test_gmres_poly_is_optimal(system):
    """||pi(M) b|| is minimal over residual polynomials (q(0) = 1) of the same degree."""
    op, A, b = system
    m = 6
    theta = krylov.gmres_poly_roots(op, b, m)
    best = np.linalg.norm(krylov.apply_pi(op, theta, b))
    rng = np.random.default_rng(0)
    for _ in range(20):
        roots = theta * (1 + 0.05 * (rng.standard_normal(m) + 1j * rng.standard_normal(m)))
        assert np.linalg.norm(krylov.apply_pi(op, roots, b)) >= best * (1 - 1e-12)


def test_poly_identities(system):
    op, A, b = system
    theta = krylov.gmres_poly_roots(op, b, 14)
    # p(theta_k) = 1/theta_k and pi(theta_k) = 0
    assert np.abs(krylov.pi_scalar(theta, theta)).max() < 1e-12
    assert np.abs(krylov.poly_scalar(theta, theta) - 1 / theta).max() < 1e-12 * np.abs(1 / theta).max()
    # pi(M) = 1 - M p(M)
    x = synth.random_spinor(DIMS, 3).ravel()
    lhs = x - A @ krylov.apply_poly(op, theta, x)
    assert np.linalg.norm(lhs - krylov.apply_pi(op, theta, x)) < 1e-12 * np.linalg.norm(x)
    # p(M) = W diag(p(lambda)) W^-1 from a dense eigendecomposition
    lam, W = np.linalg.eig(A)
    pA = W @ np.diag(krylov.poly_scalar(theta, lam)) @ np.linalg.inv(W)
    assert np.linalg.norm(pA @ x - krylov.apply_poly(op, theta, x)) < 1e-9 * np.linalg.norm(x)
    # p(M) approximates M^-1 better than the identity does
    assert np.linalg.norm(A @ krylov.apply_poly(op, theta, x) - x) < np.linalg.norm(A @ x - x)


def test_leja_order_brute_force():
    rng = np.random.default_rng(4)
    pts = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    out = krylov.leja_order(pts)
    assert np.allclose(np.sort_complex(out), np.sort_complex(pts))
    assert np.isclose(abs(out[0]), np.abs(pts).max(), rtol=1e-15)
    for k in range(1, 9):
        chosen = out[:k]
        cand = [p for p in pts if not np.any(np.isclose(p, chosen))]
        prods = [np.prod(np.abs(p - chosen)) for p in cand]
        assert np.isclose(np.prod(np.abs(out[k] - chosen)), max(prods))
    # tie rule: lowest original index first
    tie = np.array([1.0, -1.0, 1j, -1j])
    assert krylov.leja_order(tie)[0] == 1.0


def test_double_poly(system):
    op, A, b = system
    m_in, m_out = 5, 4
    th_in, th_out = krylov.double_poly_roots(op, b, m_in, m_out)
    a = np.linspace(0.3, 1.7, 7) + 0.2j
    pin = krylov.poly_scalar(th_in, a)
    # 1 - a p_double(a) = pi_out(a p_in(a))
    lhs = 1 - a * krylov.double_scalar(th_in, th_out, a)
    assert np.abs(lhs - krylov.pi_scalar(th_out, a * pin)).max() < 1e-12
    # matrix form against the dense eigendecomposition; count M applications
    calls = []

    def counted(v):
        calls.append(1)
        return op(v)

    x = synth.random_spinor(DIMS, 6).ravel()
    y = krylov.apply_double(counted, th_in, th_out, x)
    lam, W = np.linalg.eig(A)
    pd = W @ np.diag(krylov.double_scalar(th_in, th_out, lam)) @ np.linalg.inv(W)
    assert np.linalg.norm(pd @ x - y) < 1e-9 * np.linalg.norm(x)
    # p_double has degree (d_in + 1)(d_out + 1) - 1 = m_in*m_out - 1 (Sec. 5): one M per degree
    assert len(calls) == m_in * m_out - 1


def test_gmres_solve_matches_dense(system):
    op, A, b = system
    x, its, rel = krylov.gmres_solve(op, b, tol=1e-12, m=40)
    xd = np.linalg.solve(A, b)
    assert rel <= 1e-12
    assert np.linalg.norm(x - xd) < 1e-9 * np.linalg.norm(xd)
