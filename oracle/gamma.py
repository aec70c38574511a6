"""Euclidean Dirac matrices in a chiral basis (Hermitian, gamma_mu^2 = 1).

The paper names the Wilson-Dirac matrix (Sec. 2) without fixing a basis; the
trace Tr(Theta M^-1) for Theta in {1, gamma_4} does not depend on the choice.
Basis used on both sides of the library:
  gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = 1, 2, 3 -> x, y, z)
  gamma_4 = [[0, 1], [1, 0]]                   (t)
  gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4
Index mu = 0, 1, 2, 3 stands for x, y, z, t.
"""
import numpy as np

SIGMA = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = np.stack([_block(_Z2, -1j * SIGMA[k], 1j * SIGMA[k], _Z2) for k in range(3)]
                 + [_block(_Z2, _I2, _I2, _Z2)])
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
IDENTITY4 = np.eye(4, dtype=np.complex128)

THETA = {"1": IDENTITY4, "g4": GAMMA[3], "g5": GAMMA5}
