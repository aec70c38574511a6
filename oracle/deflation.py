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
lambda_i (j = i for real lambda_i); equal eigenvalues take distinct partners.
Eigenvalues whose partner is not among the kept ones are dropped.  U is
rescaled so that U^H Z = I (biorthonormal), U = W (W^H Z)^{-H}.  Two further
rules bound the variance that the deflated samples carry through
(eta^H Theta z_i)(u_i^H eta): while W^H Z is singular the pair of largest
|lambda| is dropped, and while a column of (W^H Z)^{-H} (whose norm is the
norm of u_i for unit w) exceeds ``max_u`` = 100 in norm the pair with the
largest one is dropped; a dropped pair takes its gamma_5 partner with it, so
the kept eigenvalues stay closed under conjugation.  Any kept set keeps the
estimator unbiased (Eq. 2 with an exactly traced deflated part, Sec. 7).
"""
import numpy as np

from . import krylov


def select_pairs(lam, res, k, tol_accept=1e-3, real_tol=2e-4):
    """Kept candidates and their gamma_5 partners (Sec. 8 acceptance, reading above).

    ``lam``, ``res``: Rayleigh quotients and residual norms of the candidate
    Ritz vectors.  Accepted: res < tol_accept (finite).  The accepted ones are
    ordered by |lambda| (stable) and the first k considered.  In that order a
    real lambda (|Im| < real_tol) is its own partner; a complex one takes the
    nearest considered candidate to conj(lambda), other than itself and not
    already taken as a partner, if it lies within 10 max(real_tol, 1e-6
    |lambda|); otherwise it is dropped.  Returns (keep, partner): lists of
    candidate indices, partner[i] belonging to keep[i].
    """
    lam = np.asarray(lam, dtype=np.complex128)
    res = np.asarray(res, dtype=np.float64)
    acc = [i for i in range(lam.size) if np.isfinite(res[i]) and res[i] < tol_accept]
    acc = sorted(acc, key=lambda i: abs(lam[i]))[:k]  # sorted() is stable
    taken = set()
    keep, partner = [], []
    for a in acc:
        l = lam[a]
        if abs(l.imag) < real_tol:
            keep.append(a)
            partner.append(a)
            continue
        best, bd = None, np.inf
        for b in acc:
            if b == a or b in taken:
                continue
            d = abs(lam[b] - np.conj(l))
            if d < bd:
                best, bd = b, d
        if best is not None and bd < 10 * max(real_tol, 1e-6 * abs(l)):
            keep.append(a)
            partner.append(best)
            taken.add(best)
    return keep, partner


def condition_selection(S, mates, max_u=100.0):
    """Drop rules on the overlap S = W^H Z of the kept pairs (reading above).

    ``S``: q x q complex, S[i, j] = w_i^H z_j; ``mates[i]``: position of pair
    i's gamma_5 partner among the q (i itself for a real eigenvalue).  Starting
    from all positions in order: if S restricted to the selection is singular,
    drop the last selected position (the largest |lambda|) and its partner;
    else form Inv = (S_sel)^{-H}; if the largest column norm of Inv exceeds
    max_u, drop that column's position and its partner; else stop.
    Returns (sel, Inv): the kept positions (increasing) and the inverse.
    """
    S = np.asarray(S, dtype=np.complex128)
    sel = list(range(S.shape[0]))
    while sel:
        Ssel = S[np.ix_(sel, sel)]
        try:
            Inv = np.linalg.inv(Ssel.conj().T)
        except np.linalg.LinAlgError:
            victim = len(sel) - 1
        else:
            norms = np.sqrt(np.sum(np.abs(Inv) ** 2, axis=0))
            victim = int(np.argmax(norms))  # first maximum
            if np.isfinite(norms[victim]) and norms[victim] <= max_u:
                return sel, Inv
        v = sel[victim]
        drop = {v, mates[v]}
        sel = [s for s in sel if s not in drop]
    return [], np.zeros((0, 0), dtype=np.complex128)


def pp_arnoldi_eigenpairs(op, gamma5, theta_poly, b, m_arnoldi, k, tol_accept=1e-3, real_tol=2e-4,
                          max_u=100.0):
    """Return (lambda, Z, U, residuals) for up to k smallest eigenpairs, U^H Z = I.

    ``op`` applies M to a flat vector, ``gamma5`` applies gamma_5 to a flat vector,
    ``theta_poly`` are the Leja-ordered roots of the preconditioning polynomial p
    (an empty list: phi = M itself).  Reading taken for "the smallest Ritz
    vectors" (Sec. 8): every Ritz vector of phi(M) is tested against M (Rayleigh
    quotient, residual), and the accepted ones of smallest |lambda| are kept
    (select_pairs, condition_selection).  When the spectrum of M surrounds the
    origin, phi(lambda) for the smallest lambda need not be the smallest |phi|,
    so selecting on phi alone would miss them.
    """
    if len(theta_poly):
        phi = lambda v: op(krylov.apply_poly(op, theta_poly, v))
    else:
        phi = op
    V, H, _ = krylov.arnoldi(phi, b, m_arnoldi)
    mu, G = np.linalg.eig(H[:m_arnoldi, :m_arnoldi])
    lam = np.zeros(m_arnoldi, dtype=np.complex128)
    res = np.zeros(m_arnoldi)
    Zc = []
    for i in range(m_arnoldi):
        z = V[:, :m_arnoldi] @ G[:, i]
        z = z / np.linalg.norm(z)
        Mz = op(z)
        lam[i] = np.vdot(z, Mz)
        res[i] = np.linalg.norm(Mz - lam[i] * z)
        Zc.append(z)
    keep, partner = select_pairs(lam, res, k, tol_accept, real_tol)
    n = b.size
    if not keep:
        return (np.zeros(0, complex), np.zeros((n, 0), complex), np.zeros((n, 0), complex), np.zeros(0))
    Z = np.stack([Zc[i] for i in keep], axis=1)
    W = np.stack([gamma5(Zc[j]) for j in partner], axis=1)
    pos = {c: i for i, c in enumerate(keep)}
    mates = [pos.get(partner[i], i) for i in range(len(keep))]
    sel, Inv = condition_selection(W.conj().T @ Z, mates, max_u)
    if not sel:
        return (np.zeros(0, complex), np.zeros((n, 0), complex), np.zeros((n, 0), complex), np.zeros(0))
    Z = Z[:, sel]
    U = W[:, sel] @ Inv
    kept = [keep[i] for i in sel]
    return lam[kept], Z, U, res[kept]


def deflate_vector(Z, U, b):
    """b - Z (U^H b): b without its components along the right eigenvectors z_i (U^H Z = I)."""
    return b - Z @ (U.conj().T @ b)


def deflated_double_poly_roots(op, b, m_in, m_out, Z, U):
    """Deflated double polynomial.  The paper names it (abstract, Sec. 7, Sec. 9: a deflated
    polynomial lowers the degree of the highest-degree polynomial) without giving its
    construction.  Reading taken: theta_in from GMRES(m_in) on M from b as in Sec. 5;
    theta_out from GMRES(m_out) on phi_in(M) = M p_in(M) from the start vector with the
    deflated eigenvector components removed, b - Z U^H b.  The Krylov space then avoids
    those components (exactly so for exact eigenvectors), so pi_out spends no roots on
    phi_in at the deflated eigenvalues, whose part of every level is traced exactly."""
    theta_in = krylov.gmres_poly_roots(op, b, m_in)
    phi_in = lambda v: op(krylov.apply_poly(op, theta_in, v))
    theta_out = krylov.gmres_poly_roots(phi_in, deflate_vector(Z, U, b), m_out)
    return theta_in, theta_out


def biorthonormalise(Z, W):
    """U = W (W^H Z)^{-H}, so that U^H Z = I."""
    S = W.conj().T @ Z
    return W @ np.linalg.inv(S).conj().T


def deflated_guess(Z, U, lam):
    """Oblique eigen-projection used to deflate solves: r -> Z Lambda^{-1} U^H r."""
    def apply(r):
        return Z @ ((U.conj().T @ r) / lam)
    return apply
