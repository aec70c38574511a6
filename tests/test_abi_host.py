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


def _random_candidates(rng, m):
    """Candidate eigenvalues with conjugate pairs, near-real values, duplicates and unpaired ones."""
    base = rng.uniform(0.05, 1.0, m // 3) * np.exp(1j * rng.uniform(-np.pi, np.pi, m // 3))
    lam = list(base) + list(np.conj(base) + rng.normal(0, 3e-4, base.size))
    lam += list(rng.uniform(-1, 1, m // 6) + 1j * rng.uniform(-1.5e-4, 1.5e-4, m // 6))
    lam += [base[0]] * 2 + [np.conj(base[0])]
    lam = np.array(lam)
    rng.shuffle(lam)
    res = 10.0 ** rng.uniform(-8, -2, lam.size)
    return lam, res


def test_deflation_pairs_match_oracle(mmc):
    """The library's kept set and gamma_5 partners equal the oracle's, index for index."""
    from oracle import deflation
    rng = np.random.default_rng(11)
    for trial in range(40):
        lam, res = _random_candidates(rng, 30 + trial)
        for k in (1, 5, 17, 100):
            want = deflation.select_pairs(lam, res, k)
            got = mmc.mmc_deflation_pairs(lam, res, 1e-3, k)
            assert got == (list(want[0]), list(want[1])), (trial, k)


def test_deflation_condition_matches_oracle(mmc):
    """The overlap drop rules (singular, column norm above the bound, partner dropped
    along) give the oracle's kept positions."""
    from oracle import deflation
    rng = np.random.default_rng(12)
    for trial in range(60):
        q = int(rng.integers(1, 12))
        S = np.eye(q) + 0.3 * (rng.standard_normal((q, q)) + 1j * rng.standard_normal((q, q)))
        if trial % 3 == 0 and q > 1:  # nearly dependent columns
            i, j = rng.choice(q, 2, replace=False)
            S[:, j] = S[:, i] + 10.0 ** -rng.uniform(1, 6) * rng.standard_normal(q)
        if trial % 5 == 0:  # a zero column: exactly singular
            S[:, q - 1] = 0
        mates = np.arange(q)
        for a in range(0, q - 1, 2):
            if rng.random() < 0.6:
                mates[a], mates[a + 1] = a + 1, a
        for bound in (100.0, 3.0):
            want, _ = deflation.condition_selection(S, list(mates), bound)
            got = mmc.mmc_deflation_condition(S, mates, bound)
            assert got == list(want), (trial, bound)


@pytest.mark.parametrize("dims,reach", [((24, 24, 24, 24), 8), ((8, 8, 8, 8), 6), ((16, 16, 16, 16), 10),
                                        ((4, 4, 4, 4), 2)])
def test_probing_colouring_separates_reach(mmc, dims, reach):
    """Probing is exact (Sec. 6) only if no two distinct sites within the polynomial's
    reach share a colour.  Brute force on the library's colouring: for every
    displacement d with 1 <= periodic L1 norm <= reach, the colour array shifted by d
    differs from itself at every site.  (24^4, reach 8: the benchmark's Tr p_8.)"""
    colour, n = mmc.mmc_probe_colouring(dims, reach)
    lx, ly, lz, lt = dims
    c = colour.reshape(lt, lz, ly, lx)
    assert n == len(np.unique(colour)) and colour.min() == 0 and colour.max() == n - 1
    rng = [range(-min(reach, L // 2), min(reach, L // 2) + 1) for L in dims]
    seen = set()
    checked = 0
    for dx in rng[0]:
        for dy in rng[1]:
            for dz in rng[2]:
                for dt in rng[3]:
                    d = tuple(((v % L) for v, L in zip((dx, dy, dz, dt), dims)))
                    l1 = sum(min(v, L - v) for v, L in zip(d, dims))
                    if l1 == 0 or l1 > reach or d in seen:
                        continue
                    seen.add(d)
                    shifted = np.roll(c, shift=(-d[3], -d[2], -d[1], -d[0]), axis=(0, 1, 2, 3))
                    assert not np.any(shifted == c), d
                    checked += 1
    assert checked > 0


def test_every_context_call_rejects_a_null_context(mmc):
    """Every entry point that takes a context returns MMC_ERR_ARG for a NULL one (all other
    arguments zero or NULL) before it touches the device, so none of these calls needs a
    GPU; mmc_destroy accepts NULL and returns MMC_OK, as its header comment states."""
    import ctypes
    checked = 0
    for name, (res, args) in mmc._SIGS.items():
        if not args or args[0] is not mmc._vp or res is not mmc._i:
            continue
        vals = [0.0 if a is mmc._d else 0 if a in (mmc._i, mmc._u32, mmc._u64, ctypes.c_longlong) else None
                for a in args]
        rc = getattr(mmc.lib, name)(*vals)
        assert rc == (mmc.MMC_OK if name == "mmc_destroy" else mmc.MMC_ERR_ARG), (name, rc)
        checked += 1
    assert checked >= 45, checked


def test_host_routines_reject_bad_sizes_and_null_buffers(mmc):
    """The context-free routines (harmonic Ritz values, Leja order, eigenpairs, deflation
    pairs and condition, probing colouring, context creation) return MMC_ERR_ARG for
    negative sizes and for NULL buffers with positive sizes, without dereferencing them."""
    import ctypes
    checked = 0
    for name, (res, args) in mmc._SIGS.items():
        if not args or args[0] is mmc._vp or res is not mmc._i or name == "mmc_rhs_block":
            continue
        for size in (-1, 2):
            vals = [1e-3 if a is mmc._d else size if a in (mmc._i, mmc._u32, mmc._u64, ctypes.c_longlong) else None
                    for a in args]
            assert getattr(mmc.lib, name)(*vals) == mmc.MMC_ERR_ARG, (name, size)
        checked += 1
    assert checked >= 7, checked
