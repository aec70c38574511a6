"""GMRES polynomials (Sec. 3), double polynomials (Sec. 5) and GMRES solves,
in FP64 on flat complex vectors.

Conventions (readings of the paper, stated once here):
* A GMRES cycle of length m (GMRES(m), Sec. 3) gives m harmonic Ritz values
  theta_1..theta_m, the roots of the residual polynomial
  pi(a) = prod_i (1 - a/theta_i), of degree m; p has degree m - 1 and
  pi(a) = 1 - a p(a).
* The paper prints u_k with a leading factor M; summed, those terms give
  M p(M) = 1 - pi(M), not p(M).  The reading used here is
  u_k = (1/theta_k) prod_{j<k} (1 - M/theta_j), which is the one that
  satisfies pi(M) = 1 - M p(M) (the identity the paper states first).
* Arnoldi uses modified Gram-Schmidt from b/||b||.
* Leja order: first the value of largest modulus; then repeatedly the value
  maximising the product of distances to those already chosen (compared as
  a sum of logs); ties go to the lowest original index.
"""
import numpy as np


def arnoldi(op, b, m):
    """Arnoldi with modified Gram-Schmidt (the single GMRES(m) cycle of Sec. 3).

    Returns (V, H, beta): V is n x (m+1) orthonormal, H is the (m+1) x m
    upper Hessenberg matrix with op V[:, :m] = V H, beta = ||b||.
    """
    n = b.size
    V = np.zeros((n, m + 1), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    beta = np.linalg.norm(b)
    V[:, 0] = b.ravel() / beta
    for j in range(m):
        w = np.asarray(op(V[:, j])).ravel().astype(np.complex128)
        for i in range(j + 1):
            H[i, j] = np.vdot(V[:, i], w)
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] == 0:
            raise ArithmeticError("Arnoldi breakdown at step %d" % j)
        V[:, j + 1] = w / H[j + 1, j]
    return V, H, beta


def harmonic_ritz(H):
    """Harmonic Ritz values (zero target) from the (m+1) x m Hessenberg of a GMRES(m) cycle (Sec. 3).

    They are the eigenvalues of H_m + |h_{m+1,m}|^2 f e_m^T with
    f = H_m^{-H} e_m, the roots of the GMRES residual polynomial.
    """
    m = H.shape[1]
    Hm = H[:m, :m]
    em = np.zeros(m, dtype=np.complex128)
    em[-1] = 1.0
    f = np.linalg.solve(Hm.conj().T, em)
    A = Hm + (abs(H[m, m - 1]) ** 2) * np.outer(f, em)
    return np.linalg.eigvals(A)


def leja_order(theta):
    """Leja ordering of a set of complex points (Sec. 3, Reichel's ordering)."""
    theta = np.asarray(theta, dtype=np.complex128)
    m = theta.size
    order = []
    remaining = list(range(m))
    first = max(remaining, key=lambda i: (abs(theta[i]), -i))
    order.append(first)
    remaining.remove(first)
    while remaining:
        best, best_val = None, None
        for i in remaining:
            d = np.abs(theta[i] - theta[order])
            val = -np.inf if np.any(d == 0) else float(np.sum(np.log(d)))
            if best is None or val > best_val:
                best, best_val = i, val
        order.append(best)
        remaining.remove(best)
    return theta[order]


def gmres_poly_roots(op, b, m):
    """Leja-ordered harmonic Ritz values of one GMRES(m) cycle of ``op`` from ``b`` (Sec. 3)."""
    _, H, _ = arnoldi(op, b, m)
    return leja_order(harmonic_ritz(H))


def apply_poly(op, theta, x):
    """p(op) x = sum_k u_k (Sec. 3), u_k = (1/theta_k) prod_{j<k}(1 - op/theta_j) x.

    Recurrence: prod = x, y = 0; for k = 1..m: y += prod/theta_k and, for
    k < m, prod -= op(prod)/theta_k.  m - 1 applications of ``op``.
    """
    prod = np.array(x, dtype=np.complex128, copy=True)
    y = np.zeros_like(prod)
    m = len(theta)
    for k in range(m):
        y = y + prod / theta[k]
        if k < m - 1:
            prod = prod - op(prod) / theta[k]
    return y


def apply_pi(op, theta, x):
    """pi(op) x = prod_i (1 - op/theta_i) x, the GMRES residual polynomial (Sec. 3)."""
    v = np.array(x, dtype=np.complex128, copy=True)
    for t in theta:
        v = v - op(v) / t
    return v


def poly_scalar(theta, a):
    """p(a) for scalar (or array) a, by the same recurrence as apply_poly."""
    return apply_poly(lambda v: a * v, theta, np.ones_like(np.asarray(a, dtype=np.complex128)))


def pi_scalar(theta, a):
    a = np.asarray(a, dtype=np.complex128)
    out = np.ones_like(a)
    for t in theta:
        out = out * (1 - a / t)
    return out


def double_poly_roots(op, b, m_in, m_out):
    """Double polynomial (Sec. 5): GMRES(m_in) on M gives theta_in; GMRES(m_out) on
    phi_in(M) = M p_in(M) from the same start vector gives theta_out."""
    theta_in = gmres_poly_roots(op, b, m_in)
    phi_in = lambda v: op(apply_poly(op, theta_in, v))
    theta_out = gmres_poly_roots(phi_in, b, m_out)
    return theta_in, theta_out


def apply_double(op, theta_in, theta_out, x):
    """p_double(M) x = p_in(M) p_out(phi_in(M)) x (Sec. 5)."""
    phi_in = lambda v: op(apply_poly(op, theta_in, v))
    y = apply_poly(phi_in, theta_out, x)
    return apply_poly(op, theta_in, y)


def double_scalar(theta_in, theta_out, a):
    """p_double(a) = p_in(a) p_out(a p_in(a))."""
    a = np.asarray(a, dtype=np.complex128)
    pin = poly_scalar(theta_in, a)
    return pin * poly_scalar(theta_out, a * pin)


def gmres_solve(op, b, tol=1e-12, m=100, max_restarts=200, x0=None, deflate=None):
    """Restarted GMRES(m) in FP64 with MGS Arnoldi and a dense least-squares solve.

    ``deflate``, if given, is a function r -> correction added to x at every
    restart (an oblique eigen-projection, see deflation.deflated_guess).
    Returns (x, iterations, relative residual).  Raises if not converged.
    """
    b = np.asarray(b, dtype=np.complex128).ravel()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).ravel()
    bnorm = np.linalg.norm(b)
    its = 0
    for _ in range(max_restarts):
        r = b - np.asarray(op(x)).ravel()
        if deflate is not None:
            x = x + deflate(r)
            r = b - np.asarray(op(x)).ravel()
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol:
            return x, its, rel
        n = b.size
        V = np.zeros((n, m + 1), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        beta = np.linalg.norm(r)
        V[:, 0] = r / beta
        k_used = m
        for j in range(m):
            w = np.asarray(op(V[:, j])).ravel()
            for i in range(j + 1):
                H[i, j] = np.vdot(V[:, i], w)
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            its += 1
            e1 = np.zeros(j + 2, dtype=np.complex128)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[: j + 2, : j + 1], e1, rcond=None)
            res = np.linalg.norm(e1 - H[: j + 2, : j + 1] @ y) / bnorm
            if H[j + 1, j] == 0 or res <= tol * 0.5:
                k_used = j + 1
                break
            V[:, j + 1] = w / H[j + 1, j]
        e1 = np.zeros(k_used + 1, dtype=np.complex128)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(H[: k_used + 1, :k_used], e1, rcond=None)
        x = x + V[:, :k_used] @ y
    r = b - np.asarray(op(x)).ravel()
    rel = np.linalg.norm(r) / bnorm
    if rel <= tol:
        return x, its, rel
    raise ArithmeticError("GMRES did not converge: relative residual %.3e" % rel)
