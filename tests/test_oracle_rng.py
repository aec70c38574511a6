"""Pins for the oracle's counter-based generator and Z(4) noise (Sec. 1)."""
import os

import numpy as np

from oracle.philox import philox4x32_10
from oracle import noise

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([int(w, 16) for w in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        out = philox4x32_10(*r[:6])
        assert [int(w) for w in out] == r[6:]


def test_philox_vectorised_matches_scalar():
    c = np.arange(17, dtype=np.uint64) * 7919
    w = philox4x32_10(c, 3, 5, 7, 11, 13)
    for i in range(17):
        s = philox4x32_10(int(c[i]), 3, 5, 7, 11, 13)
        assert all(int(w[k][i]) == int(s[k]) for k in range(4))


def test_z4_values_and_frequencies():
    dims = (4, 4, 4, 8)
    codes = noise.z4_codes(dims, seed=12345, noise_index=3, level_id=1)
    eta = noise.z4_noise(dims, seed=12345, noise_index=3, level_id=1)
    assert set(np.unique(codes)) <= {0, 1, 2, 3}
    assert np.allclose(np.abs(eta), 1.0)
    assert np.allclose(eta, 1j ** codes)
    counts = np.bincount(codes.ravel(), minlength=4)
    expected = codes.size / 4
    chi2 = np.sum((counts - expected) ** 2 / expected)
    assert chi2 < 16.27  # 3 dof, p = 0.001


def test_z4_streams_independent():
    dims = (4, 4, 4, 4)
    a = noise.z4_codes(dims, 1, 0, 0)
    b = noise.z4_codes(dims, 1, 1, 0)
    c = noise.z4_codes(dims, 1, 0, 1)
    d = noise.z4_codes(dims, 2, 0, 0)
    for other in (b, c, d):
        assert np.mean(a == other) < 0.3
    # second moment identity of Z(4): E[conj(eta_i) eta_j] = delta_ij
    etas = np.stack([noise.z4_noise(dims, 7, j, 0).ravel() for j in range(200)])
    g = (etas.conj().T @ etas[:, :50]) / 200
    off = g[:50] - np.eye(50)
    assert np.abs(off).max() < 0.35
