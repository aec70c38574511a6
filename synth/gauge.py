"""Synthetic SU(3) gauge fields and generic complex test vectors.

Canonical host layouts (complex128, C order):
  gauge  U[mu][t][z][y][x][row][col],  mu = 0:x, 1:y, 2:z, 3:t
  spinor psi[t][z][y][x][spin][colour] (optionally a trailing batch axis)

The paper measures on quenched beta = 6.0 ensembles, which are not
available here; these fields stand in for them.  Each link is
U = exp(i*eps*H) with H = sum_a h_a lambda_a / 2 (Gell-Mann matrices,
h_a ~ N(0, 1)), followed by a reunitarisation: Gram-Schmidt on the first two
rows and the third row set to conj(row1 x row2), which puts det U = 1 to
rounding.  The generator is numpy's PCG64 seeded with ``seed``, identical on
x86_64 and aarch64.
"""
import numpy as np

_GELL_MANN = np.zeros((8, 3, 3), dtype=np.complex128)
_GELL_MANN[0][0, 1] = _GELL_MANN[0][1, 0] = 1
_GELL_MANN[1][0, 1] = -1j
_GELL_MANN[1][1, 0] = 1j
_GELL_MANN[2][0, 0] = 1
_GELL_MANN[2][1, 1] = -1
_GELL_MANN[3][0, 2] = _GELL_MANN[3][2, 0] = 1
_GELL_MANN[4][0, 2] = -1j
_GELL_MANN[4][2, 0] = 1j
_GELL_MANN[5][1, 2] = _GELL_MANN[5][2, 1] = 1
_GELL_MANN[6][1, 2] = -1j
_GELL_MANN[6][2, 1] = 1j
_GELL_MANN[7][0, 0] = _GELL_MANN[7][1, 1] = 1 / np.sqrt(3)
_GELL_MANN[7][2, 2] = -2 / np.sqrt(3)


def _reunitarise(u):
    """Project a batch of 3x3 matrices onto SU(3) (rows 1-2 Gram-Schmidt, row 3 = conj(r1 x r2))."""
    r1 = u[..., 0, :]
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = u[..., 1, :]
    r2 = r2 - np.sum(np.conj(r1) * r2, axis=-1, keepdims=True) * r1
    r2 = r2 / np.linalg.norm(r2, axis=-1, keepdims=True)
    r3 = np.conj(np.cross(r1, r2))
    return np.stack([r1, r2, r3], axis=-2)


def _random_su3(rng, shape, eps):
    h = rng.standard_normal(shape + (8,))
    H = np.einsum("...a,aij->...ij", h, _GELL_MANN) / 2.0
    w, q = np.linalg.eigh(H)
    u = np.einsum("...ik,...k,...jk->...ij", q, np.exp(1j * eps * w), np.conj(q))
    return _reunitarise(u)


def random_gauge(dims, eps, seed):
    """Random gauge field of lattice ``dims`` = (Lx, Ly, Lz, Lt), spread ``eps``, numpy seed ``seed``."""
    lx, ly, lz, lt = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    u = _random_su3(rng, (4, lt, lz, ly, lx), float(eps))
    return np.ascontiguousarray(u)


def unit_gauge(dims):
    """Free field: every link is the 3x3 identity."""
    lx, ly, lz, lt = (int(d) for d in dims)
    u = np.zeros((4, lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1
    return u


def gauge_transform_matrices(dims, seed):
    """Random site-local SU(3) matrices g(x), shape [t][z][y][x][3][3], for covariance tests."""
    lx, ly, lz, lt = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    return _random_su3(rng, (lt, lz, ly, lx), 1.0)


def random_spinor(dims, seed, nrhs=None):
    """Complex Gaussian spinor field(s) in canonical layout; trailing batch axis if ``nrhs``."""
    lx, ly, lz, lt = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    shape = (lt, lz, ly, lx, 4, 3) + ((int(nrhs),) if nrhs is not None else ())
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
