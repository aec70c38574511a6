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
