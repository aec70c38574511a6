"""Eigenpairs for Monte Carlo level deflation (Sec. 7, Sec. 8).

PP-Arnoldi (Sec. 7): an Arnoldi run of ``m_arnoldi`` steps on
phi(M) = M p(M) from a start vector; Ritz vectors of phi(M) are
approximate eigenvectors z_i of M (same eigenvectors).  lambda_i is the Rayleigh quotient
z_i^H M z_i (||z_i|| = 1).  A pair is accepted when ||M z_i - lambda_i z_i||
is below ``tol_accept`` (1e-3 in Sec. 8); values with |Im lambda| below
``real_tol`` (2e-4 in Sec. 8) count as real.

The paper says only that the left eigenvectors "are found".  Reading taken:
gamma_5-hermiticity (gamma5 M gamma5 = M^+) makes gamma5 z a left eigenvector
for conj(lambda); so u_i = gamma5 z_j with lambda_j the conjugate partner of
lambda_i (j = i for real lambda_i).  Eigenvalues whose partner is not among
the accepted ones are dropped.  Finally U is rescaled so that U^H Z = I
(biorthonormal), U = W (W^H Z)^{-H}.
"""
import numpy as np

from . import krylov


def pp_arnoldi_eigenpairs(op, gamma5, theta_poly, b, m_arnoldi, k, tol_accept=1e-3, real_tol=2e-4,
                          n_candidates=None):
    """Return (lambda, Z, U, residuals) for up to k smallest eigenpairs, U^H Z = I.

    ``op`` applies M to a flat vector, ``gamma5`` applies gamma_5 to a flat vector,
    ``theta_poly`` are the Leja-ordered roots of the preconditioning polynomial p.
    Reading taken for "the smallest Ritz vectors" (Sec. 8): the Ritz vectors of
    the ``n_candidates`` (default: all m) Ritz values of phi(M) smallest in
    modulus are each tested against M (Rayleigh quotient, residual); the
    accepted ones are ordered by |lambda| and the first k kept.  When the
    spectrum of M surrounds the origin, phi(lambda) for the smallest lambda
    need not be the smallest |phi|, so selecting on phi alone would miss them.
    """
    phi = lambda v: op(krylov.apply_poly(op, theta_poly, v))
    V, H, _ = krylov.arnoldi(phi, b, m_arnoldi)
    mu, G = np.linalg.eig(H[:m_arnoldi, :m_arnoldi])
    ncand = min(m_arnoldi, n_candidates if n_candidates is not None else m_arnoldi)
    order = np.argsort(np.abs(mu), kind="stable")[:ncand]
    lam, Zs, res = [], [], []
    for i in order:
        z = V[:, :m_arnoldi] @ G[:, i]
        z = z / np.linalg.norm(z)
        Mz = op(z)
        l = np.vdot(z, Mz)
        r = np.linalg.norm(Mz - l * z)
        if r < tol_accept:
            lam.append(l)
            Zs.append(z)
            res.append(r)
    by_size = np.argsort(np.abs(np.array(lam)), kind="stable")[:k]
    lam = np.array(lam, dtype=np.complex128)[by_size]
    Zs = [Zs[i] for i in by_size]
    res = [res[i] for i in by_size]
    keep, partner = [], []
    for i, l in enumerate(lam):
        if abs(l.imag) < real_tol:
            keep.append(i)
            partner.append(i)
            continue
        d = np.abs(lam - np.conj(l))
        d[i] = np.inf
        j = int(np.argmin(d))
        if d[j] < max(real_tol, 1e-6 * abs(l)) * 10:
            keep.append(i)
            partner.append(j)
    if not keep:
        n = b.size
        return (np.zeros(0, complex), np.zeros((n, 0), complex), np.zeros((n, 0), complex),
                np.zeros(0))
    Z = np.stack([Zs[i] for i in keep], axis=1)
    W = np.stack([gamma5(Zs[j]) for j in partner], axis=1)
    U = biorthonormalise(Z, W)
    return lam[keep], Z, U, np.array(res)[keep]


def biorthonormalise(Z, W):
    """U = W (W^H Z)^{-H}, so that U^H Z = I."""
    S = W.conj().T @ Z
    return W @ np.linalg.inv(S).conj().T


def deflated_guess(Z, U, lam):
    """Oblique eigen-projection used to deflate solves: r -> Z Lambda^{-1} U^H r."""
    def apply(r):
        return Z @ ((U.conj().T @ r) / lam)
    return apply
