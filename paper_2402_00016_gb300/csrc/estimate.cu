// Multilevel estimate with adaptive noise counts (Sec. 8 stopping by standard
// error, checked after a first batch and then every few noises; Sec. 9 names the
// cost-optimal allocation of Giles as the refinement).  Host code only: every
// sample comes from mmc_trace_level, run on consecutive noise indices of each
// level, so the samples of several batches are those of one call over all of them.
#include "internal.h"

using mmc::cd;

namespace {

struct LevelRun {
  std::vector<cd> x;   // samples in noise order
  cd corr{0, 0};       // exact trace of the deflated part (the same every batch)
  int kd = 0;
  double seconds = 0;
  long long matvecs = 0;
};

double part_var(const std::vector<cd>& x, int n, bool imag) {
  if (n < 2) return 0.0;
  double m = 0;
  for (int i = 0; i < n; ++i) m += imag ? x[i].imag() : x[i].real();
  m /= n;
  double v = 0;
  for (int i = 0; i < n; ++i) {
    const double d = (imag ? x[i].imag() : x[i].real()) - m;
    v += d * d;
  }
  return v / (n - 1);
}

void fill(const LevelRun& r, mmc_level_stats* out) {
  const int n = int(r.x.size());
  cd mean(0, 0);
  for (const cd& v : r.x) mean += v;
  mean /= double(std::max(1, n));
  double vr = 0, vi = 0, cv = 0;
  for (const cd& v : r.x) {
    const cd d = v - mean;
    vr += d.real() * d.real();
    vi += d.imag() * d.imag();
    cv += std::norm(d);
  }
  const double dn = n > 1 ? double(n - 1) : 1.0;
  std::memset(out, 0, sizeof(*out));
  out->n = n;
  out->k_deflated = r.kd;
  out->mean_re = mean.real();
  out->mean_im = mean.imag();
  out->var_re = n > 1 ? vr / dn : 0.0;
  out->var_im = n > 1 ? vi / dn : 0.0;
  out->cvar = n > 1 ? cv / dn : 0.0;
  out->stderr_re = n > 0 ? std::sqrt(out->var_re / n) : 0.0;
  out->stderr_im = n > 0 ? std::sqrt(out->var_im / n) : 0.0;
  out->corr_re = r.corr.real();
  out->corr_im = r.corr.imag();
  out->value_re = mean.real() + r.corr.real();
  out->value_im = mean.imag() + r.corr.imag();
  out->seconds = r.seconds;
  out->matvecs = r.matvecs;
}

}  // namespace

extern "C" {

int mmc_estimate(mmc_ctx* ctx, int n_levels, const mmc_level_spec* levels, int theta_op, int prec, int precond,
                 double eps, int alloc, const double* cost, uint32_t first_noise, mmc_level_stats* out,
                 double* total) {
  if (!ctx) return MMC_ERR_ARG;
  if (n_levels < 1 || !levels || !out || !(eps > 0) || (alloc != MMC_ALLOC_EQUAL && alloc != MMC_ALLOC_COST))
    RET(MMC_ERR_ARG, "mmc_estimate: bad argument");
  for (int l = 0; l < n_levels; ++l) {
    const mmc_level_spec& s = levels[l];
    if (s.n_first < 2 || s.n_check < 1 || s.n_max < s.n_first)
      RET(MMC_ERR_ARG, "mmc_estimate: each level needs n_first >= 2, n_check >= 1, n_max >= n_first");
    if (cost && !(cost[l] > 0)) RET(MMC_ERR_ARG, "mmc_estimate: costs must be positive");
  }
  const bool imag = theta_op == MMC_THETA_G4;  // Tr(gamma_4 M^-1) is imaginary
  std::vector<LevelRun> run(n_levels);
  // run `add` more noises of level l (consecutive noise indices)
  auto more = [&](int l, int add) -> int {
    const mmc_level_spec& s = levels[l];
    LevelRun& r = run[l];
    mmc_level_stats st;
    std::vector<double> smp(2 * size_t(add));
    const int rc = mmc_trace_level(ctx, s.hi, s.lo, theta_op, s.deflate, add, first_noise + uint32_t(r.x.size()),
                                   s.level, prec, precond, &st, smp.data());
    if (rc != MMC_OK) return rc;
    for (int i = 0; i < add; ++i) r.x.push_back(cd(smp[2 * i], smp[2 * i + 1]));
    r.corr = cd(st.corr_re, st.corr_im);
    r.kd = st.k_deflated;
    r.seconds += st.seconds;
    r.matvecs += st.matvecs;
    return MMC_OK;
  };
  for (int l = 0; l < n_levels; ++l) TRY(more(l, levels[l].n_first));
  if (alloc == MMC_ALLOC_EQUAL) {
    // each level until its standard error is at most eps / sqrt(L)
    const double target = eps / std::sqrt(double(n_levels));
    for (int l = 0; l < n_levels; ++l) {
      const mmc_level_spec& s = levels[l];
      while (true) {
        const int n = int(run[l].x.size());
        const double se = std::sqrt(part_var(run[l].x, n, imag) / n);
        if (se <= target || n >= s.n_max) break;
        TRY(more(l, std::min(s.n_check, s.n_max - n)));
      }
    }
  } else {
    // counts N_l = eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k); C_l from `cost`, else the
    // matvecs spent per sample so far (the paper's cost unit; deterministic, unlike wall time)
    while (true) {
      std::vector<double> V(n_levels), C(n_levels);
      double s = 0;
      for (int l = 0; l < n_levels; ++l) {
        const int n = int(run[l].x.size());
        V[l] = part_var(run[l].x, n, imag);
        C[l] = cost ? cost[l] : std::max(1.0, double(run[l].matvecs) / n);
        s += std::sqrt(V[l] * C[l]);
      }
      bool grew = false;
      for (int l = 0; l < n_levels; ++l) {
        const mmc_level_spec& sp = levels[l];
        const int n = int(run[l].x.size());
        const double target = std::ceil(std::sqrt(V[l] / C[l]) * s / (eps * eps));
        const double shortfall = std::min(target, double(sp.n_max)) - n;
        if (shortfall > 0 && n < sp.n_max) {
          const long long add = (static_cast<long long>(shortfall) + sp.n_check - 1) / sp.n_check * sp.n_check;
          TRY(more(l, int(std::min<long long>(add, sp.n_max - n))));
          grew = true;
        }
      }
      if (!grew) break;
    }
  }
  double sum = 0, var = 0;
  for (int l = 0; l < n_levels; ++l) {
    fill(run[l], &out[l]);
    sum += imag ? out[l].value_im : out[l].value_re;
    var += (imag ? out[l].var_im : out[l].var_re) / out[l].n;
  }
  if (total) {
    total[0] = sum;
    total[1] = std::sqrt(var);
  }
  return MMC_OK;
}

}  // extern "C"
