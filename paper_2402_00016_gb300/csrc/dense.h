// Host FP64 dense complex linear algebra for the small matrices of the
// method: Arnoldi Hessenberg matrices, harmonic Ritz values (Sec. 3), Ritz
// pairs of PP-Arnoldi (Sec. 7), GMRES least squares, k x k biorthonormalisation.
#pragma once
#include <complex>
#include <vector>

namespace mmc {
using cd = std::complex<double>;

// Column-major n x n matrix helper.
struct CMat {
  int rows = 0, cols = 0;
  std::vector<cd> a;
  CMat() = default;
  CMat(int r, int c) : rows(r), cols(c), a(size_t(r) * c, cd(0, 0)) {}
  cd& operator()(int i, int j) { return a[size_t(i) + size_t(j) * rows]; }
  const cd& operator()(int i, int j) const { return a[size_t(i) + size_t(j) * rows]; }
};

// Eigenvalues w (n) and, if vr != nullptr, unit-norm right eigenvectors (columns)
// of a general complex matrix: Householder Hessenberg reduction followed by the
// single-shift complex QR algorithm (Wilkinson shifts).  Returns false if the
// QR iteration did not converge.
bool eig(const CMat& A, std::vector<cd>& w, CMat* vr);

// Solve A X = B in place (B overwritten), Gaussian elimination with partial
// pivoting.  Returns false if A is singular to working precision.
bool lu_solve(CMat A, CMat& B);

// Least squares min || rhs - H y || for an (m+1) x m upper Hessenberg H by
// Givens rotations; returns y (m) and the residual norm.
std::vector<cd> hessenberg_lstsq(const CMat& H, int m, const std::vector<cd>& rhs, double* resnorm);

// Harmonic Ritz values (zero target) of a GMRES(m) cycle from its (m+1) x m
// Hessenberg: eigenvalues of H_m + |h_{m+1,m}|^2 H_m^{-H} e_m e_m^T (Sec. 3).
bool harmonic_ritz(const CMat& H, int m, std::vector<cd>& theta);

// Leja ordering (Sec. 3): first the largest modulus; next the maximiser of the
// sum of log distances to the chosen points; ties to the lowest index.
std::vector<cd> leja_order(const std::vector<cd>& pts);

// Kept candidates of the deflation (Sec. 8 acceptance): those with res < tol_accept,
// ordered by |lambda| (stable), the first k; a real one (|Im| < real_tol) is its own
// gamma_5 partner, a complex one takes the nearest candidate to its conjugate that is
// neither itself nor already taken, within 10 max(real_tol, 1e-6 |lambda|), else it is
// dropped.  keep[i], partner[i]: candidate indices.
void deflation_pairs(const std::vector<cd>& lam, const std::vector<double>& res, double tol_accept, int k,
                     double real_tol, std::vector<int>& keep, std::vector<int>& partner);

// Drop rules on the q x q overlap S(i, j) = w_i^H z_j of the kept pairs: while S
// restricted to the selection is singular drop the last position, while a column of
// its inverse conjugate transpose has norm above max_u drop the position of the
// largest; each drop takes the position's partner mates[pos] with it.  sel: kept
// positions (increasing); Inv = (S_sel)^{-H}.  Returns false if nothing is left.
bool deflation_condition(const CMat& S, const std::vector<int>& mates, double max_u, std::vector<int>& sel,
                         CMat& Inv);

// Scalar p(a) of the Leja recurrence (Sec. 3) and pi(a) = prod (1 - a/theta).
cd poly_scalar(const std::vector<cd>& theta, cd a);
cd pi_scalar(const std::vector<cd>& theta, cd a);
}  // namespace mmc
