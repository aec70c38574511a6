"""Pins of the oracle's deflation selection rules (Sec. 7, Sec. 8 and the reading for
the left eigenvectors): the acceptance test, the order by |lambda|, the gamma_5
partners (distinct for equal eigenvalues), and the drop rules on the overlap W^H Z.
Each case is small enough to be worked out by hand; the expected lists below are
those hand results."""
import numpy as np

from oracle import deflation


def test_acceptance_and_order():
    lam = np.array([0.5, 0.2, 0.9, 0.1, 0.3])
    res = np.array([1e-4, 2e-3, 1e-5, 1e-6, 5e-4])  # 0.2 is rejected (residual above 1e-3)
    keep, partner = deflation.select_pairs(lam, res, k=3)
    assert keep == [3, 4, 0]  # |lambda| 0.1, 0.3, 0.5: the three smallest accepted
    assert partner == keep  # real eigenvalues are their own partners


def test_stable_order_for_equal_moduli():
    lam = np.array([0.3, -0.3, 0.3j, -0.3j])  # all |lambda| = 0.3
    res = np.zeros(4)
    keep, partner = deflation.select_pairs(lam, res, k=4)
    # the real ones keep their order; 0.3i pairs with -0.3i and back
    assert keep == [0, 1, 2, 3]
    assert partner == [0, 1, 3, 2]


def test_real_threshold():
    lam = np.array([0.2 + 1.9e-4j, 0.4 + 3e-4j])  # the first counts as real, the second has no partner
    keep, partner = deflation.select_pairs(lam, np.zeros(2), k=2)
    assert keep == [0] and partner == [0]


def test_conjugate_partner_window():
    a = 0.25 + 0.1j
    # partner within 10 max(2e-4, 1e-6 |a|) = 2e-3 of conj(a), an impostor outside it
    lam = np.array([a, np.conj(a) + 1.5e-3, 0.5 + 0.3j, 0.5 - 0.3j + 3e-3])
    keep, partner = deflation.select_pairs(lam, np.zeros(4), k=4)
    assert keep == [0, 1] and partner == [1, 0]


def test_equal_eigenvalues_take_distinct_partners():
    a = 0.2 + 0.05j
    lam = np.array([a, a, np.conj(a), np.conj(a)])
    keep, partner = deflation.select_pairs(lam, np.zeros(4), k=4)
    assert keep == [0, 1, 2, 3]
    assert partner == [2, 3, 0, 1]
    # three copies of a with two of conj(a): the third copy of a finds no free partner
    lam = np.array([a, a, a, np.conj(a), np.conj(a)])
    keep, partner = deflation.select_pairs(lam, np.zeros(5), k=5)
    assert keep == [0, 1, 3, 4] and partner == [3, 4, 0, 1]


def test_k_limit_applies_before_pairing():
    a = 0.2 + 0.05j
    lam = np.array([0.1, a, 0.3, np.conj(a) * 1.5])
    # the k = 2 smallest are 0.1 and a; a's partner is not among them, so a is dropped
    keep, partner = deflation.select_pairs(lam, np.zeros(4), k=2)
    assert keep == [0] and partner == [0]


def test_condition_well_conditioned_keeps_all():
    S = np.array([[1.0, 0.5], [0.0, 1.0]], dtype=complex)
    sel, Inv = deflation.condition_selection(S, [0, 1])
    assert sel == [0, 1]
    # (S^H)^{-1} = [[1, 0], [-0.5, 1]]
    assert np.allclose(Inv, [[1, 0], [-0.5, 1]])


def test_condition_norm_bound_drops_pair_with_partner():
    S = np.diag([1.0, 1e-3, 1.0, 0.5]).astype(complex)
    # column norms of S^{-H}: 1, 1000, 1, 2; position 1 exceeds 100
    sel, _ = deflation.condition_selection(S, [0, 1, 2, 3])
    assert sel == [0, 2, 3]
    sel, _ = deflation.condition_selection(S, [0, 2, 1, 3])  # 1 and 2 are gamma_5 partners
    assert sel == [0, 3]
    # the bound itself: 1000 is kept under a bound of 1000
    sel, _ = deflation.condition_selection(S, [0, 1, 2, 3], max_u=1000.0)
    assert sel == [0, 1, 2, 3]


def test_condition_singular_drops_largest_with_partner():
    S = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 0.0]], dtype=complex)
    sel, _ = deflation.condition_selection(S, [0, 1, 2])
    assert sel == [0, 1]
    sel, _ = deflation.condition_selection(S, [0, 2, 1])  # the last position takes 1 along
    assert sel == [0]
    sel, Inv = deflation.condition_selection(np.zeros((2, 2), dtype=complex), [0, 1])
    assert sel == [] and Inv.shape == (0, 0)


def test_condition_repeats_until_bounded():
    # two nearly dependent columns: after the first drop the rest is well conditioned
    S = np.array([[1.0, 1.0], [1.0, 1.0 + 1e-4]], dtype=complex)
    sel, Inv = deflation.condition_selection(S, [0, 1])
    assert len(sel) == 1
    assert np.allclose(Inv, 1.0 / np.conj(S[sel[0], sel[0]]))


def _tiny():
    import synth
    from oracle import wilson
    dims, shape = (2, 2, 2, 4), (4, 2, 2, 2, 4, 3)
    U = synth.random_gauge(dims, 0.3, 1)
    op = lambda v: wilson.apply_M(U, 0.155, v.reshape(shape + v.shape[1:])).reshape(v.shape)
    A = wilson.dense_M(U, 0.155)
    return dims, op, A


def test_deflated_start_vector_keeps_krylov_space_in_complement():
    """With exact eigenvectors the deflated start vector has no component along them
    (U^H b' = 0) and neither has any phi_in^j b': the space GMRES builds for p_out."""
    from oracle import krylov, noise
    dims, op, A = _tiny()
    lam, R = np.linalg.eig(A)
    Lf = np.linalg.inv(R).conj().T  # left eigenvectors, Lf^H R = I
    idx = np.argsort(np.abs(lam))[:6]
    Z, U = R[:, idx], Lf[:, idx]
    b = noise.z4_noise(dims, 1, 0, 0, noise.TAG_GMRES).ravel()
    bp = deflation.deflate_vector(Z, U, b)
    assert np.abs(U.conj().T @ bp).max() < 1e-10 * np.linalg.norm(b)
    # the removed part is exactly the spectral component: b = b' + Z U^H b
    assert np.allclose(bp + Z @ (U.conj().T @ b), b, atol=1e-12)
    th_in = krylov.gmres_poly_roots(op, b, 4)
    v = bp
    for j in range(5):
        v = op(krylov.apply_poly(op, th_in, v))
        assert np.abs(U.conj().T @ v).max() < 1e-9 * np.linalg.norm(v), j
    t_in, t_out = deflation.deflated_double_poly_roots(op, b, 4, 3, Z, U)
    assert np.allclose(t_in, th_in)
    phi = lambda x: op(krylov.apply_poly(op, th_in, x))
    assert np.allclose(t_out, krylov.gmres_poly_roots(phi, bp, 3))


def test_deflated_inverse_level_is_unbiased():
    """Tr(M^-1 - p_dbl) = E[eta^H (A - sum_i c_i z_i u_i^H) eta] + sum_i c_i u_i^H z_i with
    c_i = 1/lambda_i - p_dbl(lambda_i), for Z(4) noise (E[eta^H B eta] = Tr B), with the
    double polynomial built from the deflated start vector; exact with dense matrices."""
    from oracle import krylov, noise
    dims, op, A = _tiny()
    lam, R = np.linalg.eig(A)
    Lf = np.linalg.inv(R).conj().T
    idx = np.argsort(np.abs(lam))[:6]
    Z, U, lz = R[:, idx], Lf[:, idx], lam[idx]
    b = noise.z4_noise(dims, 1, 0, 0, noise.TAG_GMRES).ravel()
    t_in, t_out = deflation.deflated_double_poly_roots(op, b, 4, 3, Z, U)
    n = A.shape[0]
    P = krylov.apply_double(lambda X: A @ X, t_in, t_out, np.eye(n))
    Ainv = np.linalg.inv(A)
    c = 1.0 / lz - krylov.double_scalar(t_in, t_out, lz)
    B = Ainv - P - (Z * c) @ U.conj().T
    corr = np.sum(c * np.einsum("ij,ij->j", U.conj(), Z))
    assert abs(np.trace(B) + corr - np.trace(Ainv - P)) < 1e-9 * abs(np.trace(Ainv))
    # the deflated operator annihilates the deflated eigenvectors: B z_i = 0
    assert np.abs(B @ Z).max() < 1e-8 * np.abs(Ainv).max()
