"""CPU tests of the C ABI: the library loads, exports every symbol the header
declares, and its host-only FP64 steps (harmonic Ritz values, Leja order,
small eigenproblems; Sec. 3, Sec. 7) agree with the oracle."""
import os
import re

import numpy as np
import pytest

import synth
from oracle import krylov, noise, wilson

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_00016_gb300 import mmc as m
    return m


def test_exports_every_declared_symbol(mmc):
    header = open(os.path.join(ROOT, "include", "mmc.h")).read()
    declared = set(re.findall(r"^(?:int|size_t|const char\*)\s+(mmc_\w+)\(", header, re.M))
    assert len(declared) >= 25
    for name in declared:
        assert hasattr(mmc.lib, name), name


def test_eig_against_numpy(mmc):
    rng = np.random.default_rng(0)
    for n in (1, 2, 7, 40):
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        ev, V = mmc.mmc_eig(A, vectors=True)
        ref = np.linalg.eigvals(A)
        for e in ref:
            assert np.min(np.abs(ev - e)) < 1e-10 * max(1, abs(e))
        assert np.linalg.norm(A @ V - V * ev) < 1e-10 * np.linalg.norm(A)


def test_harmonic_ritz_and_leja_vs_oracle(mmc):
    dims, shape = (2, 2, 2, 4), (4, 2, 2, 2, 4, 3)
    U = synth.random_gauge(dims, 0.5, 1)
    op = lambda v: wilson.apply_M(U, 0.12, v.reshape(shape)).ravel()
    b = noise.z4_noise(dims, 0, 0, 0, noise.TAG_GMRES).ravel()
    for m in (1, 5, 16, 40):
        _, H, _ = krylov.arnoldi(op, b, m)
        ref = krylov.leja_order(krylov.harmonic_ritz(H))
        got = mmc.mmc_harmonic_ritz(H)
        assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max()


def test_leja_tie_rule(mmc):
    pts = np.array([1.0, -1.0, 1j, -1j, 0.5 + 0.5j])
    assert np.allclose(mmc.mmc_leja_order(pts), krylov.leja_order(pts))
