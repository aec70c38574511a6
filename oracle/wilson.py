"""Wilson-Dirac matrix M(U, kappa) (Sec. 1, Eq. 1; kappa and beta in Sec. 4).

The paper names the Wilson-Dirac matrix and the hopping parameter kappa but
does not write M out.  Reading taken (kappa normalisation, Wilson r = 1):

  (M psi)(x) = psi(x) - kappa * sum_mu [ (1 - gamma_mu) U_mu(x)        psi(x + mu)
                                        + (1 + gamma_mu) U_mu(x - mu)^+ psi(x - mu) ]

periodic in x, y, z and, when ``t_antiperiodic``, antiperiodic in t (a factor
-1 on every hop across the t = Lt-1 <-> 0 boundary).

Layouts are the canonical host ones: U[mu][t][z][y][x][3][3],
psi[t][z][y][x][spin][colour] with an optional trailing batch axis.
"""
import numpy as np

from .gamma import GAMMA, GAMMA5

# array axis of psi that moves with direction mu (x, y, z, t)
_AXIS = (3, 2, 1, 0)


def _shift(psi, mu, forward, t_antiperiodic):
    """psi(x + mu) when ``forward`` else psi(x - mu), with the time boundary sign."""
    ax = _AXIS[mu]
    out = np.roll(psi, -1 if forward else 1, axis=ax)
    if mu == 3 and t_antiperiodic:
        out = out.copy()
        if forward:
            out[-1] *= -1.0
        else:
            out[0] *= -1.0
    return out


def _colour(Umat, psi, batch):
    """U psi on colour indices: (U psi)_{s a} = sum_b U_{ab} psi_{s b}."""
    if batch:
        return np.matmul(Umat[:, :, :, :, None, :, :], psi)
    return np.matmul(Umat[:, :, :, :, None, :, :], psi[..., None])[..., 0]


def _spin(G, psi):
    """G psi on spin indices: (G psi)_{s a} = sum_u G_{su} psi_{u a}."""
    sh = psi.shape
    flat = psi.reshape(sh[:4] + (4, -1))
    return np.matmul(G, flat).reshape(sh)


def hop(U, psi, t_antiperiodic=True, dagger_sign=1):
    """D psi = sum_mu [(1 - s gamma_mu) U_mu(x) psi(x+mu) + (1 + s gamma_mu) U_mu(x-mu)^+ psi(x-mu)], s = dagger_sign."""
    batch = psi.ndim == 7
    out = np.zeros_like(psi)
    eye = np.eye(4)
    for mu in range(4):
        Um = U[mu]
        Ub = np.conj(np.swapaxes(np.roll(Um, 1, axis=_AXIS[mu]), -1, -2))  # U_mu(x - mu)^+
        colour_f = _colour(Um, _shift(psi, mu, True, t_antiperiodic), batch)
        colour_b = _colour(Ub, _shift(psi, mu, False, t_antiperiodic), batch)
        out += _spin(eye - dagger_sign * GAMMA[mu], colour_f)
        out += _spin(eye + dagger_sign * GAMMA[mu], colour_b)
    return out


def apply_M(U, kappa, psi, t_antiperiodic=True):
    """M psi (Eq. 1's matrix M, Wilson form above)."""
    return psi - kappa * hop(U, psi, t_antiperiodic)


def apply_Mdag(U, kappa, psi, t_antiperiodic=True):
    """M^+ psi, written out directly: the hop with (1 + gamma_mu) forward and (1 - gamma_mu) backward."""
    return psi - kappa * hop(U, psi, t_antiperiodic, dagger_sign=-1)


def apply_gamma(G, psi):
    """Site-local spin matrix G applied to psi (Theta of Eq. 1, gamma_5)."""
    return _spin(np.asarray(G, dtype=np.complex128), psi)


def apply_gamma5(psi):
    return apply_gamma(GAMMA5, psi)


def dense_M(U, kappa, t_antiperiodic=True):
    """Dense n x n matrix of M (n = 12V) in canonical ordering, built column by column."""
    lt, lz, ly, lx = U.shape[1:5]
    n = 12 * lx * ly * lz * lt
    eye = np.eye(n, dtype=np.complex128).reshape(lt, lz, ly, lx, 4, 3, n)
    cols = apply_M(U, kappa, eye, t_antiperiodic)
    return cols.reshape(n, n)
