"""Pins for the oracle's Wilson-Dirac matrix (Sec. 1, Eq. 1; kappa in Sec. 4).

Nothing here retypes the stencil: it is checked through gamma-matrix algebra,
gamma_5-hermiticity, gauge covariance and the free-field spectrum in closed
form (plane waves, antiperiodic time)."""
import itertools

import numpy as np
import pytest

import synth
from oracle import gamma, wilson


def test_gamma_algebra():
    g = gamma.GAMMA
    for m, n in itertools.product(range(4), range(4)):
        assert np.allclose(g[m] @ g[n] + g[n] @ g[m], 2.0 * (m == n) * np.eye(4))
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
    g5 = gamma.GAMMA5
    assert np.allclose(g5, g5.conj().T) and np.allclose(g5 @ g5, np.eye(4))
    for m in range(4):
        assert np.allclose(g5 @ g[m], -g[m] @ g5)


def test_gauge_is_su3():
    U = synth.random_gauge((4, 4, 4, 4), 0.5, 1)
    uu = np.einsum("...ij,...kj->...ik", U, U.conj())
    assert np.abs(uu - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14


@pytest.mark.parametrize("tap", [True, False])
def test_gamma5_hermiticity(tap):
    dims = (4, 4, 2, 6)
    U = synth.random_gauge(dims, 0.5, 3)
    a = synth.random_spinor(dims, 4)
    b = synth.random_spinor(dims, 5)
    k = 0.13
    lhs = np.vdot(wilson.apply_gamma5(a), wilson.apply_M(U, k, wilson.apply_gamma5(b), tap))
    rhs = np.vdot(wilson.apply_M(U, k, a, tap), b)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    # the separately written M^+ is the adjoint of M
    lhs = np.vdot(a, wilson.apply_Mdag(U, k, b, tap))
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_gauge_covariance():
    """M[U^g] (g psi) = g M[U] psi with U^g_mu(x) = g(x) U_mu(x) g(x+mu)^+."""
    dims = (4, 2, 4, 4)
    U = synth.random_gauge(dims, 0.7, 8)
    g = synth.gauge_transform_matrices(dims, 9)
    axes = (3, 2, 1, 0)
    Ug = np.empty_like(U)
    for mu in range(4):
        gfwd = np.roll(g, -1, axis=axes[mu])
        Ug[mu] = np.einsum("...ab,...bc,...dc->...ad", g, U[mu], gfwd.conj())
    psi = synth.random_spinor(dims, 10)
    gpsi = np.einsum("tzyxab,tzyxsb->tzyxsa", g, psi)
    lhs = wilson.apply_M(Ug, 0.14, gpsi)
    rhs = np.einsum("tzyxab,tzyxsb->tzyxsa", g, wilson.apply_M(U, 0.14, psi))
    assert np.abs(lhs - rhs).max() < 1e-13


def _free_eigs(dims, kappa, tap=True):
    lx, ly, lz, lt = dims
    out = []
    for n in itertools.product(range(lx), range(ly), range(lz), range(lt)):
        p = [2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz,
             2 * np.pi * (n[3] + (0.5 if tap else 0.0)) / lt]
        a = 1 - 2 * kappa * sum(np.cos(q) for q in p)
        b = 2 * kappa * np.sqrt(sum(np.sin(q) ** 2 for q in p))
        out += [a + 1j * b] * 6 + [a - 1j * b] * 6
    return np.array(out)


def test_free_field_plane_waves():
    """A plane wave e^{ip.x} chi is an eigenvector with lambda = 1 - 2k sum cos p +- 2ik sqrt(sum sin^2 p)."""
    dims = (4, 6, 2, 8)
    kappa = 0.12
    U = synth.unit_gauge(dims)
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    for n in [(1, 2, 0, 3), (0, 0, 0, 0), (3, 5, 1, 7)]:
        p = [2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz,
             2 * np.pi * (n[3] + 0.5) / lt]
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        S = sum(gamma.GAMMA[m] * np.sin(p[m]) for m in range(4))
        a = 1 - 2 * kappa * sum(np.cos(q) for q in p)
        w, chis = np.linalg.eigh(S)
        for i in range(4):
            chi = chis[:, i]
            colour = np.array([0.3, -0.5j, 0.8])
            psi = phase[..., None, None] * chi[:, None] * colour[None, :]
            lam = a + 2j * kappa * w[i]
            assert np.abs(wilson.apply_M(U, kappa, psi) - lam * psi).max() < 1e-13


def test_free_field_dense_spectrum_and_trace():
    dims = (2, 2, 2, 4)
    kappa = 0.11
    A = wilson.dense_M(synth.unit_gauge(dims), kappa)
    ev = np.linalg.eigvals(A)
    ref = _free_eigs(dims, kappa)
    key = lambda v: np.round(v.real, 8) + 1e-3 * np.round(v.imag, 8)
    assert np.allclose(np.sort_complex(np.round(ev, 9)), np.sort_complex(np.round(ref, 9)), atol=1e-8)
    tr = np.trace(np.linalg.inv(A))
    assert abs(tr - np.sum(1.0 / ref)) < 1e-10 * abs(tr)
    assert abs(np.trace(A) - A.shape[0]) < 1e-12


def test_theta_insertions_trace_symmetry():
    """Tr(M^-1) real, Tr(gamma4 M^-1) imaginary (gamma5 gamma4 gamma5 = -gamma4), dense."""
    dims = (2, 2, 2, 4)
    U = synth.random_gauge(dims, 0.5, 1)
    A = wilson.dense_M(U, 0.12)
    Ainv = np.linalg.inv(A)
    n = A.shape[0]
    G4 = np.kron(np.eye(n // 12), np.kron(gamma.GAMMA[3], np.eye(3)))
    t1 = np.trace(Ainv)
    t4 = np.trace(G4 @ Ainv)
    assert abs(t1.imag) < 1e-12 * abs(t1)
    assert abs(t4.real) < 1e-12 * max(1.0, abs(t4))
