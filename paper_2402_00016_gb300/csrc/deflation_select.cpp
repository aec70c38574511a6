// Kept set of the deflation eigenpairs (Sec. 7, Sec. 8): the acceptance test of
// Sec. 8 on the candidate Ritz pairs, gamma_5 partners for the left vectors, and
// the drop rules on the overlap W^H Z that bound the size of the left vectors.
// Host FP64 only (see dense.h).
#include <algorithm>
#include <cmath>

#include "dense.h"

namespace mmc {

void deflation_pairs(const std::vector<cd>& lam, const std::vector<double>& res, double tol_accept, int k,
                     double real_tol, std::vector<int>& keep, std::vector<int>& partner) {
  keep.clear();
  partner.clear();
  std::vector<int> acc;
  for (int i = 0; i < int(lam.size()); ++i)
    if (std::isfinite(res[i]) && res[i] < tol_accept) acc.push_back(i);
  std::stable_sort(acc.begin(), acc.end(), [&](int a, int b) { return std::abs(lam[a]) < std::abs(lam[b]); });
  if (int(acc.size()) > k) acc.resize(std::max(k, 0));
  // a complex eigenvalue takes the nearest candidate to its conjugate that no earlier
  // one has taken, so a degenerate eigenvalue's vectors get distinct partners
  std::vector<char> taken(lam.size(), 0);
  for (size_t a = 0; a < acc.size(); ++a) {
    const cd l = lam[acc[a]];
    if (std::abs(l.imag()) < real_tol) {
      keep.push_back(acc[a]);
      partner.push_back(acc[a]);
      continue;
    }
    int best = -1;
    double bd = 1e300;
    for (size_t b = 0; b < acc.size(); ++b) {
      if (b == a || taken[acc[b]]) continue;
      const double d = std::abs(lam[acc[b]] - std::conj(l));
      if (d < bd) {
        bd = d;
        best = acc[b];
      }
    }
    if (best >= 0 && bd < 10 * std::max(real_tol, 1e-6 * std::abs(l))) {
      keep.push_back(acc[a]);
      partner.push_back(best);
      taken[best] = 1;
    }
  }
}

bool deflation_condition(const CMat& S, const std::vector<int>& mates, double max_u, std::vector<int>& sel,
                         CMat& Inv) {
  const int q0 = S.rows;
  sel.resize(q0);
  for (int i = 0; i < q0; ++i) sel[i] = i;
  while (!sel.empty()) {
    const int q = int(sel.size());
    CMat SH(q, q);
    Inv = CMat(q, q);
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) SH(i, j) = std::conj(S(sel[j], sel[i]));
    for (int i = 0; i < q; ++i) Inv(i, i) = 1.0;
    int victim;
    if (!lu_solve(SH, Inv)) {
      victim = q - 1;  // singular: the pair of largest |lambda|
    } else {
      victim = 0;
      double cmax = -1;
      for (int i = 0; i < q; ++i) {
        double c2 = 0;
        for (int j = 0; j < q; ++j) c2 += std::norm(Inv(j, i));
        if (c2 > cmax) {
          cmax = c2;
          victim = i;
        }
      }
      if (std::isfinite(cmax) && std::sqrt(cmax) <= max_u) return true;
    }
    // drop the victim together with its gamma_5 partner, so the kept eigenvalues stay
    // closed under conjugation
    const int v = sel[victim];
    const int mate = mates[v];
    std::vector<int> next;
    for (int s : sel)
      if (s != v && s != mate) next.push_back(s);
    sel.swap(next);
  }
  Inv = CMat(0, 0);
  return false;
}

}  // namespace mmc
