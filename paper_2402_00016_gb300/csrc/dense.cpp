// Host FP64 dense complex linear algebra (see dense.h).  Textbook methods:
// Householder reduction to Hessenberg form, the implicit single-shift complex
// QR algorithm with Wilkinson shifts (Golub & Van Loan, Matrix Computations,
// Sec. 7.5), back substitution for the eigenvectors of the Schur factor,
// Gaussian elimination with partial pivoting and Givens least squares.
#include "dense.h"

#include <algorithm>
#include <cmath>
#include <limits>

namespace mmc {
namespace {
const double kEps = std::numeric_limits<double>::epsilon();

// Householder reduction A -> Q^H A Q upper Hessenberg; accumulates Q.
void to_hessenberg(CMat& H, CMat& Q) {
  const int n = H.rows;
  Q = CMat(n, n);
  for (int i = 0; i < n; ++i) Q(i, i) = 1.0;
  std::vector<cd> v(n);
  for (int k = 0; k < n - 2; ++k) {
    double alpha2 = 0;
    for (int i = k + 1; i < n; ++i) alpha2 += std::norm(H(i, k));
    double xnorm = std::sqrt(alpha2);
    if (xnorm == 0) continue;
    cd x0 = H(k + 1, k);
    cd phase = std::abs(x0) > 0 ? x0 / std::abs(x0) : cd(1, 0);
    // v = x + phase*|x| e1
    for (int i = 0; i < n; ++i) v[i] = 0;
    for (int i = k + 1; i < n; ++i) v[i] = H(i, k);
    v[k + 1] += phase * xnorm;
    double vn2 = 0;
    for (int i = k + 1; i < n; ++i) vn2 += std::norm(v[i]);
    if (vn2 == 0) continue;
    // H = (I - 2 v v^H / vn2) H
    for (int j = 0; j < n; ++j) {
      cd s = 0;
      for (int i = k + 1; i < n; ++i) s += std::conj(v[i]) * H(i, j);
      s *= 2.0 / vn2;
      for (int i = k + 1; i < n; ++i) H(i, j) -= v[i] * s;
    }
    // H = H (I - 2 v v^H / vn2), Q likewise
    for (int i = 0; i < n; ++i) {
      cd s = 0, t = 0;
      for (int j = k + 1; j < n; ++j) {
        s += H(i, j) * v[j];
        t += Q(i, j) * v[j];
      }
      s *= 2.0 / vn2;
      t *= 2.0 / vn2;
      for (int j = k + 1; j < n; ++j) {
        H(i, j) -= s * std::conj(v[j]);
        Q(i, j) -= t * std::conj(v[j]);
      }
    }
    for (int i = k + 2; i < n; ++i) H(i, k) = 0;
  }
}

// Givens rotation G = [[c, s], [-conj(s), c]] with G [x; y] = [r; 0].
inline void givens(cd x, cd y, double& c, cd& s) {
  double ax = std::abs(x), ay = std::abs(y);
  if (ay == 0) {
    c = 1;
    s = 0;
    return;
  }
  if (ax == 0) {
    c = 0;
    s = std::conj(y) / ay;
    return;
  }
  double r = std::hypot(ax, ay);
  cd alpha = x / ax;
  c = ax / r;
  s = alpha * std::conj(y) / r;
}

// Schur form of an upper Hessenberg matrix in place; accumulates into Q.
bool hessenberg_qr(CMat& H, CMat& Q) {
  const int n = H.rows;
  int hi = n - 1;
  int iter = 0, total = 0;
  const int max_total = 100 * std::max(n, 10);
  while (hi > 0) {
    int l = hi;
    while (l > 0) {
      double s = std::abs(H(l - 1, l - 1)) + std::abs(H(l, l));
      if (s == 0) s = 1.0;
      if (std::abs(H(l, l - 1)) <= kEps * s) {
        H(l, l - 1) = 0;
        break;
      }
      --l;
    }
    if (l == hi) {
      --hi;
      iter = 0;
      continue;
    }
    if (++total > max_total) return false;
    ++iter;
    cd mu;
    if (iter % 11 == 10) {
      mu = H(hi, hi) + cd(0.75 * std::abs(H(hi, hi - 1)), 0.0);  // exceptional shift
    } else {
      cd a = H(hi - 1, hi - 1), b = H(hi - 1, hi), c = H(hi, hi - 1), d = H(hi, hi);
      cd half = 0.5 * (a - d);
      cd disc = std::sqrt(half * half + b * c);
      cd m1 = 0.5 * (a + d) + disc, m2 = 0.5 * (a + d) - disc;
      mu = (std::abs(m1 - d) < std::abs(m2 - d)) ? m1 : m2;
    }
    // implicit single-shift QR sweep on rows/cols l..hi
    cd x = H(l, l) - mu, y = H(l + 1, l);
    for (int k = l; k < hi; ++k) {
      if (k > l) {
        x = H(k, k - 1);
        y = H(k + 1, k - 1);
      }
      double c;
      cd s;
      givens(x, y, c, s);
      int jstart = (k > l) ? k - 1 : l;
      for (int j = jstart; j < n; ++j) {
        cd t1 = H(k, j), t2 = H(k + 1, j);
        H(k, j) = c * t1 + s * t2;
        H(k + 1, j) = -std::conj(s) * t1 + c * t2;
      }
      if (k > l) H(k + 1, k - 1) = 0;
      int iend = std::min(k + 2, hi);
      for (int i = 0; i <= iend; ++i) {
        cd t1 = H(i, k), t2 = H(i, k + 1);
        H(i, k) = c * t1 + std::conj(s) * t2;
        H(i, k + 1) = -s * t1 + c * t2;
      }
      for (int i = 0; i < n; ++i) {
        cd t1 = Q(i, k), t2 = Q(i, k + 1);
        Q(i, k) = c * t1 + std::conj(s) * t2;
        Q(i, k + 1) = -s * t1 + c * t2;
      }
    }
  }
  return true;
}
}  // namespace

bool eig(const CMat& A, std::vector<cd>& w, CMat* vr) {
  const int n = A.rows;
  w.assign(n, cd(0, 0));
  if (n == 0) return true;
  CMat T = A, Q;
  to_hessenberg(T, Q);
  if (!hessenberg_qr(T, Q)) return false;
  for (int i = 0; i < n; ++i) w[i] = T(i, i);
  if (!vr) return true;
  double tnorm = 0;
  for (auto& v : T.a) tnorm = std::max(tnorm, std::abs(v));
  const double small = std::max(tnorm, 1e-300) * kEps;
  *vr = CMat(n, n);
  std::vector<cd> v(n);
  for (int i = 0; i < n; ++i) {
    std::fill(v.begin(), v.end(), cd(0, 0));
    v[i] = 1.0;
    for (int j = i - 1; j >= 0; --j) {
      cd s = 0;
      for (int k = j + 1; k <= i; ++k) s += T(j, k) * v[k];
      cd d = T(j, j) - w[i];
      if (std::abs(d) < small) d = small;
      v[j] = -s / d;
    }
    double nrm = 0;
    std::vector<cd> x(n, cd(0, 0));
    for (int r = 0; r < n; ++r) {
      cd s = 0;
      for (int k = 0; k <= i; ++k) s += Q(r, k) * v[k];
      x[r] = s;
      nrm += std::norm(s);
    }
    nrm = std::sqrt(nrm);
    for (int r = 0; r < n; ++r) (*vr)(r, i) = x[r] / nrm;
  }
  return true;
}

bool lu_solve(CMat A, CMat& B) {
  const int n = A.rows;
  std::vector<int> piv(n);
  double amax = 0;
  for (auto& v : A.a) amax = std::max(amax, std::abs(v));
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::abs(A(k, k));
    for (int i = k + 1; i < n; ++i)
      if (std::abs(A(i, k)) > best) {
        best = std::abs(A(i, k));
        p = i;
      }
    if (best <= amax * 1e-300 || best == 0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A(k, j), A(p, j));
      for (int j = 0; j < B.cols; ++j) std::swap(B(k, j), B(p, j));
    }
    for (int i = k + 1; i < n; ++i) {
      cd f = A(i, k) / A(k, k);
      A(i, k) = f;
      for (int j = k + 1; j < n; ++j) A(i, j) -= f * A(k, j);
      for (int j = 0; j < B.cols; ++j) B(i, j) -= f * B(k, j);
    }
  }
  for (int j = 0; j < B.cols; ++j)
    for (int i = n - 1; i >= 0; --i) {
      cd s = B(i, j);
      for (int k = i + 1; k < n; ++k) s -= A(i, k) * B(k, j);
      B(i, j) = s / A(i, i);
    }
  return true;
}

std::vector<cd> hessenberg_lstsq(const CMat& H0, int m, const std::vector<cd>& rhs, double* resnorm) {
  CMat H(m + 1, m);
  for (int j = 0; j < m; ++j)
    for (int i = 0; i <= std::min(j + 1, m); ++i) H(i, j) = H0(i, j);
  std::vector<cd> g(rhs.begin(), rhs.begin() + (m + 1));
  for (int k = 0; k < m; ++k) {
    double c;
    cd s;
    givens(H(k, k), H(k + 1, k), c, s);
    for (int j = k; j < m; ++j) {
      cd t1 = H(k, j), t2 = H(k + 1, j);
      H(k, j) = c * t1 + s * t2;
      H(k + 1, j) = -std::conj(s) * t1 + c * t2;
    }
    cd t1 = g[k], t2 = g[k + 1];
    g[k] = c * t1 + s * t2;
    g[k + 1] = -std::conj(s) * t1 + c * t2;
  }
  std::vector<cd> y(m);
  for (int i = m - 1; i >= 0; --i) {
    cd s = g[i];
    for (int k = i + 1; k < m; ++k) s -= H(i, k) * y[k];
    y[i] = (H(i, i) != cd(0, 0)) ? s / H(i, i) : cd(0, 0);
  }
  if (resnorm) *resnorm = std::abs(g[m]);
  return y;
}

bool harmonic_ritz(const CMat& H, int m, std::vector<cd>& theta) {
  CMat Hm(m, m);
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m; ++i) Hm(i, j) = H(i, j);
  CMat HmH(m, m);
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m; ++i) HmH(i, j) = std::conj(Hm(j, i));
  CMat f(m, 1);
  f(m - 1, 0) = 1.0;
  if (!lu_solve(HmH, f)) return false;
  double h2 = std::norm(H(m, m - 1));
  CMat A = Hm;
  for (int i = 0; i < m; ++i) A(i, m - 1) += h2 * f(i, 0);
  return eig(A, theta, nullptr);
}

std::vector<cd> leja_order(const std::vector<cd>& pts) {
  const int m = int(pts.size());
  std::vector<cd> out;
  std::vector<int> chosen;
  std::vector<bool> used(m, false);
  if (m == 0) return out;
  int first = 0;
  for (int i = 1; i < m; ++i)
    if (std::abs(pts[i]) > std::abs(pts[first])) first = i;
  chosen.push_back(first);
  used[first] = true;
  while (int(chosen.size()) < m) {
    int best = -1;
    double bestv = 0;
    for (int i = 0; i < m; ++i) {
      if (used[i]) continue;
      double v = 0;
      bool zero = false;
      for (int j : chosen) {
        double d = std::abs(pts[i] - pts[j]);
        if (d == 0) {
          zero = true;
          break;
        }
        v += std::log(d);
      }
      if (zero) v = -std::numeric_limits<double>::infinity();
      if (best < 0 || v > bestv) {
        best = i;
        bestv = v;
      }
    }
    chosen.push_back(best);
    used[best] = true;
  }
  for (int i : chosen) out.push_back(pts[i]);
  return out;
}

cd poly_scalar(const std::vector<cd>& theta, cd a) {
  cd prod = 1.0, y = 0.0;
  const int m = int(theta.size());
  for (int k = 0; k < m; ++k) {
    y += prod / theta[k];
    if (k < m - 1) prod -= a * prod / theta[k];
  }
  return y;
}

cd pi_scalar(const std::vector<cd>& theta, cd a) {
  cd v = 1.0;
  for (auto t : theta) v -= a * v / t;
  return v;
}
}  // namespace mmc
