// Deflation (Sec. 7, Sec. 8), refined deflated solves (Sec. 1, Sec. 8), Monte
// Carlo levels (Eq. 2, Sec. 6, Sec. 7), exact traces by unit vectors or
// probing (Sec. 6) and the probing colouring search.
#include <algorithm>
#include <array>
#include <chrono>
#include <numeric>
#include <random>

#include "internal.h"

using namespace mmc::host;
using mmc::cd;
using mmc::CMat;
using mmc::geom;

namespace {

const int kSpc = 256;  // sites per CTA of the reduction kernels

// Sum the partials [nbx][nvec][npad] on the device and copy nvec x npad values to host.
int reduce_to_host(mmc_ctx* ctx, const double2* partial, int nbx, int nvec, int npad, std::vector<cd>& out,
                   cudaStream_t s) {
  void* red;
  TRY(scratch(ctx, "red_out", size_t(nvec) * npad * sizeof(double2), &red));
  CK(mmc::launch_reduce(partial, nbx, nvec, npad, (double2*)red, 0, s));
  std::vector<double2> h(size_t(nvec) * npad);
  CK(cudaMemcpyAsync(h.data(), red, h.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
  TRY(check_step_err(ctx, s));  // synchronises
  out.resize(h.size());
  for (size_t i = 0; i < h.size(); ++i) out[i] = cd(h[i].x, h[i].y);
  return MMC_OK;
}

// Per-rhs squared norms of a field (prec 0 or 1).
int norms2(mmc_ctx* ctx, int prec, const geom& g, const void* f, std::vector<double>& out, cudaStream_t s) {
  const int nbx = (g.V + kSpc - 1) / kSpc;
  void* part;
  TRY(scratch(ctx, "n2_part", size_t(nbx) * g.npad * sizeof(double2), &part));
  CK(mmc::launch_multidot(prec, g, f, 0, 1, f, 0, kSpc, (double2*)part, s));
  std::vector<cd> v;
  TRY(reduce_to_host(ctx, (double2*)part, nbx, 1, g.npad, v, s));
  out.resize(g.npad);
  for (int r = 0; r < g.npad; ++r) out[r] = v[r].real();
  return MMC_OK;
}

int upload(mmc_ctx* ctx, const std::string& key, const std::vector<cd>& h, void** dev, cudaStream_t s) {
  std::vector<double2> t(h.size());
  for (size_t i = 0; i < h.size(); ++i) t[i] = make_double2(h[i].real(), h[i].imag());
  TRY(scratch(ctx, key, std::max<size_t>(1, t.size()) * sizeof(double2), dev));
  CK(cudaMemcpyAsync(*dev, t.data(), t.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // host staging vector goes out of scope
  return MMC_OK;
}

// r = b - M x (FP64): one step launch with a = -1, b = kappa, g = 1 (aux = b).
int residual_f64(mmc_ctx* ctx, const geom& g, const void* b, const void* x, void* r, cudaStream_t s) {
  Run run;
  run.g = g;
  run.prec = MMC_F64;
  Step st;
  st.in = x;
  st.out = r;
  st.aux = b;
  st.flags = mmc::SF_HOP | mmc::SF_WRITE | mmc::SF_AUX;
  st.coef = coef_block(g.npad);
  for (int i = 0; i < g.npad; ++i) set_coef(st.coef, g.npad, i, -1.0, ctx->kappa, 1.0, 0, 0);
  run.steps.push_back(st);
  return exec_run(ctx, run, s);
}

// ri = r32 - M e (FP32 storage): the same step launch as residual_f64 in FP32.
int residual_f32(mmc_ctx* ctx, const geom& g, const void* r32, const void* e, void* ri, cudaStream_t s) {
  Run run;
  run.g = g;
  run.prec = MMC_F32;
  Step st;
  st.in = e;
  st.out = ri;
  st.aux = r32;
  st.flags = mmc::SF_HOP | mmc::SF_WRITE | mmc::SF_AUX;
  st.coef = coef_block(g.npad);
  for (int i = 0; i < g.npad; ++i) set_coef(st.coef, g.npad, i, -1.0, ctx->kappa, 1.0, 0, 0);
  run.steps.push_back(st);
  return exec_run(ctx, run, s);
}

// ------------------------------------------------------------------ solves
// x += Z Lambda^-1 U^H r for every rhs (oblique eigen-projection of the residual).
// fp32: projections and update from the FP32 copies of U and Z (inside a solve with
// an FP32 inner stage; the next FP64 residual takes up their rounding); otherwise FP64.
// rx_prec: precision of the fields r and x (MMC_F64, or MMC_F32 inside the FP32 restarts of
// a refined solve, which always take the FP32 copies).
int deflate_residual(mmc_ctx* ctx, const geom& g, const void* r, void* x, bool fp32, cudaStream_t s,
                     int rx_prec = MMC_F64) {
  const int k = ctx->k_defl;
  if (k == 0) return MMC_OK;
  fp32 = fp32 && ctx->U32 && ctx->Z32 && size_t(k) * g.R * 8 <= 48 * 1024;
  if (rx_prec != MMC_F64 && !fp32) RET(MMC_ERR_ARG, "deflated FP32 residual needs the FP32 eigenvector copies");
  const int nbx = (g.V + kSpc - 1) / kSpc;
  void* part;
  TRY(scratch(ctx, "dr_part", size_t(nbx) * k * g.npad * sizeof(double2), &part));
  if (fp32)
    CK(mmc::launch_vec_proj32(rx_prec, g, (const float2*)ctx->U32, k, r, kSpc, (double2*)part, s));
  else
    CK(mmc::launch_vec_proj(MMC_F64, g, ctx->U, k, r, kSpc, (double2*)part, s));
  std::vector<cd> c;
  TRY(reduce_to_host(ctx, (double2*)part, nbx, k, g.npad, c, s));
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < g.npad; ++j) c[size_t(i) * g.npad + j] /= ctx->lambda[i];
  void* dc;
  TRY(upload(ctx, "dr_coef", c, &dc, s));
  if (fp32)
    CK(mmc::launch_vec_update32(rx_prec, g, (const float2*)ctx->Z32, k, (const double2*)dc, x, s));
  else
    CK(mmc::launch_vec_update(MMC_F64, g, ctx->Z, k, (const double2*)dc, x, s));
  return MMC_OK;
}

int solve_impl(mmc_ctx* ctx, const void* b, void* x, int nrhs, double tol, int precond, int prec_inner, int m,
               int max_outer, int* iters, std::vector<double>& rel, cudaStream_t s) {
  const geom g = make_geom(ctx, nrhs);
  // inner precision: F32 basis for F32/BF16 inner solves, F64 basis for the plain FP64 form
  const int ip = prec_inner == MMC_F64 ? MMC_F64 : MMC_F32;
  const size_t f64 = field_bytes(g, MMC_F64), fi = field_bytes(g, ip);
  const size_t ebytes = elem_bytes(ip);
  void *r, *Vb, *Zb = nullptr, *ei, *e64;
  TRY(scratch(ctx, "sv_r", f64, &r));
  TRY(scratch(ctx, ip == MMC_F64 ? "sv_V64" : "sv_V", fi * (m + 1), &Vb));
  if (precond != MMC_ZERO) TRY(scratch(ctx, ip == MMC_F64 ? "sv_Z64" : "sv_Z", fi * m, &Zb));
  TRY(scratch(ctx, ip == MMC_F64 ? "sv_e64i" : "sv_e32", fi, &ei));
  TRY(scratch(ctx, "sv_e64", f64, &e64));
  std::vector<double> bn2, rn2;
  TRY(norms2(ctx, MMC_F64, g, b, bn2, s));
  int inner = 0;
  rel.assign(nrhs, 0.0);
  const size_t stride = size_t(g.npad) * g.V * 12;  // elements per basis field
  // One FGMRES(m) cycle on M e = v0 (v0 in the inner precision, already in Vb[0]): the
  // correction e = sum_j y_j Z_j (Z = preconditioned basis) into ei.
  auto op = [&](const void* vj, void* w) -> int {
    const void* zj = vj;
    if (precond != MMC_ZERO) {
      const size_t j = (reinterpret_cast<const char*>(vj) - reinterpret_cast<const char*>(Vb)) / (stride * ebytes);
      void* zdst = reinterpret_cast<char*>(Zb) + j * stride * ebytes;
      Run base;
      base.g = g;
      if (is_net(ctx, precond)) {
        if (ip != MMC_F32) RET(MMC_ERR_ARG, "mmc_solve: the learned preconditioner needs an FP32 inner solve");
        TRY(net_apply(ctx, precond, vj, zdst, g.npad, s, nullptr));
      } else if (ctx->polys[precond].kind == 0 && ctx->polys[precond].op == MMC_OP_M &&
                 ctx->polys[precond].theta.size() >= 2) {
        // single polynomial: Horner nesting, no accumulator field (3 field passes per degree)
        const int hp = prec_inner == MMC_BF16 ? MMC_BF16 : ip;
        // the paired-component layout (one 16-byte access per two components of an rhs)
        // for FP32 chains of 8-rhs blocks run by the fourth kernel form
        const bool paired = ctx->horner_paired && hp == MMC_F32 && ip == MMC_F32 && g.R == 8 &&
                            ctx->var_ver[MMC_F32][rclass(g.R)] == 4;
        void *Q0, *Q1, *src = const_cast<void*>(vj), *dst = zdst;
        TRY(scratch(ctx, "sv_h0", field_bytes(g, hp), &Q0));
        TRY(scratch(ctx, "sv_h1", field_bytes(g, hp), &Q1));
        if (hp != ip) {
          void* v16;
          void* o16;
          TRY(scratch(ctx, "sv_v16", field_bytes(g, hp), &v16));
          TRY(scratch(ctx, "sv_o16", field_bytes(g, hp), &o16));
          CK(mmc::launch_convert(hp, v16, ip, vj, g, s));
          src = v16;
          dst = o16;
        } else if (paired) {
          void *vp, *op;
          TRY(scratch(ctx, "sv_vp", field_bytes(g, hp), &vp));
          TRY(scratch(ctx, "sv_op", field_bytes(g, hp), &op));
          CK(mmc::launch_pair_layout(vp, vj, g, 1, s));
          src = vp;
          dst = op;
        }
        base.prec = hp;
        build_horner(ctx, base, ctx->polys[precond].theta, src, Q0, Q1, dst, g.npad);
        if (paired)
          for (Step& st : base.steps) st.flags |= mmc::SF_PAIRED;
        TRY(exec_run(ctx, base, s));
        if (hp != ip) CK(mmc::launch_convert(ip, zdst, hp, dst, g, s));
        if (paired) CK(mmc::launch_pair_layout(zdst, dst, g, 0, s));
      } else if (prec_inner == MMC_BF16) {
        void* v16;
        TRY(scratch(ctx, "sv_v16", field_bytes(g, MMC_BF16), &v16));
        CK(mmc::launch_convert(MMC_BF16, v16, MMC_F32, vj, g, s));
        base.prec = MMC_BF16;
        TRY(apply_poly_impl(ctx, precond, v16, g.npad, MMC_BF16, ACC_Y, zdst, base, s));
      } else {
        base.prec = ip;
        TRY(apply_poly_impl(ctx, precond, vj, g.npad, ip, ACC_Y, zdst, base, s));
      }
      zj = zdst;
    }
    return apply_M_impl(ctx, zj, w, g.npad, ip, false, s);
  };
  auto cycle = [&]() -> int {
    ArnoldiOut ao;
    TRY(arnoldi_cgs2(ctx, g, ip, Vb, m, op, ao, s, ip == MMC_F32 ? ctx->solve_gs : 2));
    inner += m;
    std::vector<cd> ycoef(size_t(m) * g.npad, cd(0, 0));
    for (int rr = 0; rr < g.npad; ++rr) {
      if (ao.beta[rr] == 0) continue;
      std::vector<cd> rhs(m + 1, cd(0, 0));
      rhs[0] = ao.beta[rr];
      double res;
      std::vector<cd> y = mmc::hessenberg_lstsq(ao.H[rr], m, rhs, &res);
      for (int j = 0; j < m; ++j) ycoef[size_t(j) * g.npad + rr] = -y[j];  // basis_update subtracts
    }
    void* dy;
    TRY(upload(ctx, "sv_y", ycoef, &dy, s));
    CK(cudaMemsetAsync(ei, 0, fi, s));
    CK(mmc::launch_basis_update(ip, g, precond != MMC_ZERO ? Zb : Vb, stride, m, (const double2*)dy, ei, s));
    return MMC_OK;
  };
  std::vector<cd> one(g.npad, cd(1, 0));
  void* d1;
  TRY(upload(ctx, "sv_one", one, &d1, s));
  for (int outer = 0; outer <= max_outer; ++outer) {
    TRY(residual_f64(ctx, g, b, x, r, s));
    if (ctx->k_defl > 0) {
      TRY(deflate_residual(ctx, g, r, x, ip != MMC_F64, s));
      TRY(residual_f64(ctx, g, b, x, r, s));
    }
    TRY(norms2(ctx, MMC_F64, g, r, rn2, s));
    bool done = true;
    for (int i = 0; i < nrhs; ++i) {
      if (!std::isfinite(rn2[i])) RET(MMC_ERR_NAN, "mmc_solve: NaN in the residual");
      rel[i] = bn2[i] > 0 ? std::sqrt(rn2[i] / bn2[i]) : 0.0;
      if (rel[i] > tol) done = false;
    }
    if (done) {
      if (iters) *iters = inner;
      return MMC_OK;
    }
    if (outer == max_outer) break;
    if (ip == MMC_F64) {
      // the plain FP64 form: one FGMRES(m) cycle per FP64 residual
      CK(mmc::launch_convert(ip, Vb, MMC_F64, r, g, s));
      TRY(cycle());
      CK(mmc::launch_axpby(MMC_F64, g, (const double2*)d1, ei, (const double2*)d1, x, s));
      continue;
    }
    // Mixed precision: restarted FGMRES(m) cycles on M e = r in FP32, each later one restarted
    // from the FP32 residual r - M e (with deflation, from its deflated form), until every
    // vector's residual is solve_red of the FP64 one (or what the tolerance still needs),
    // stagnates, or solve_cycles cycles ran; then x += e and one FP64 residual.
    // FP64 M applications (the FP64 pipe is 1/62 of the FP32 one) fall from one or two per
    // cycle to one or two per refinement step.
    const double kInnerReduction = ctx->solve_red;
    const int kInnerCycles = ctx->solve_cycles;
    void *r32, *ri, *et;
    TRY(scratch(ctx, "sv_r32", fi, &r32));
    TRY(scratch(ctx, "sv_ri32", fi, &ri));
    TRY(scratch(ctx, "sv_et32", fi, &et));
    CK(mmc::launch_convert(MMC_F32, r32, MMC_F64, r, g, s));
    CK(cudaMemcpyAsync(ri, r32, fi, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(et, 0, fi, s));
    std::vector<double> tgt(nrhs), prev(rn2.begin(), rn2.begin() + nrhs), ri2;
    for (int i = 0; i < nrhs; ++i)
      tgt[i] = std::max(kInnerReduction * kInnerReduction * rn2[i], 0.25 * tol * tol * bn2[i]);
    for (int cyc = 0; cyc < kInnerCycles; ++cyc) {
      if (ctx->k_defl > 0 && cyc > 0) {  // the first cycle starts from the deflated FP64 residual
        TRY(deflate_residual(ctx, g, ri, et, true, s, MMC_F32));
        TRY(residual_f32(ctx, g, r32, et, ri, s));
      }
      CK(cudaMemcpyAsync(Vb, ri, fi, cudaMemcpyDeviceToDevice, s));
      TRY(cycle());
      CK(mmc::launch_axpby(MMC_F32, g, (const double2*)d1, ei, (const double2*)d1, et, s));
      TRY(residual_f32(ctx, g, r32, et, ri, s));
      TRY(norms2(ctx, MMC_F32, g, ri, ri2, s));
      bool ok = true, moving = false;
      for (int i = 0; i < nrhs; ++i) {
        if (!std::isfinite(ri2[i])) RET(MMC_ERR_NAN, "mmc_solve: NaN in the inner residual");
        if (ri2[i] > tgt[i]) ok = false;
        if (ri2[i] > tgt[i] && ri2[i] < 0.81 * prev[i]) moving = true;  // norm still falls by 10% a cycle
        prev[i] = ri2[i];
      }
      if (ok || !moving) break;
    }
    CK(mmc::launch_convert(MMC_F64, e64, MMC_F32, et, g, s));
    CK(mmc::launch_axpby(MMC_F64, g, (const double2*)d1, e64, (const double2*)d1, x, s));
  }
  if (iters) *iters = inner;
  RET(MMC_ERR_NOCONV, "mmc_solve: relative residual above tolerance after max_outer cycles");
}

// ------------------------------------------------------------- colouring
// Lattice colourings c(x) = sum_k ((a_k . x) mod q_k) * stride_k with q_k | gcd(L):
// same-colour displacements form a sublattice; valid when no displacement of
// periodic L1 norm 1..reach lies in it.
struct Colouring {
  int n = 0;
  std::vector<int> colour;  // per site
};

void displacements(const int* L, int reach, std::vector<std::array<int, 4>>& out) {
  out.clear();
  int lo[4], hi[4];
  for (int m = 0; m < 4; ++m) {
    hi[m] = std::min(reach, L[m] / 2);
    lo[m] = -std::min(reach, (L[m] - 1) / 2);
  }
  for (int a = lo[0]; a <= hi[0]; ++a)
    for (int b = lo[1]; b <= hi[1]; ++b)
      for (int c = lo[2]; c <= hi[2]; ++c)
        for (int d = lo[3]; d <= hi[3]; ++d) {
          int n1 = std::abs(a) + std::abs(b) + std::abs(c) + std::abs(d);
          if (n1 == 0 || n1 > reach) continue;
          out.push_back({a, b, c, d});
        }
}

Colouring find_colouring(const int* L, int V, int reach) {
  Colouring col;
  if (reach <= 0) {
    col.n = 1;
    col.colour.assign(V, 0);
    return col;
  }
  int G = L[0];
  for (int m = 1; m < 4; ++m) G = std::gcd(G, L[m]);
  std::vector<std::array<int, 4>> D;
  displacements(L, reach, D);
  // candidate moduli tuples, by number of colours
  std::vector<int> divs;
  for (int q = 2; q <= G; ++q)
    if (G % q == 0) divs.push_back(q);
  struct Cand {
    std::vector<int> q;
    long long n;
  };
  std::vector<Cand> cands;
  for (int q1 : divs) {
    cands.push_back({{q1}, q1});
    for (int q2 : divs) {
      if (q2 > q1) continue;
      cands.push_back({{q1, q2}, (long long)q1 * q2});
      for (int q3 : divs) {
        if (q3 > q2) continue;
        cands.push_back({{q1, q2, q3}, (long long)q1 * q2 * q3});
      }
    }
  }
  std::sort(cands.begin(), cands.end(), [](const Cand& a, const Cand& b) { return a.n < b.n; });
  // lower bound: the points of an L1 ball of radius reach/2 need distinct colours
  long long lower = 1;
  for (auto& d : D)
    if (std::abs(d[0]) + std::abs(d[1]) + std::abs(d[2]) + std::abs(d[3]) <= reach / 2) ++lower;
  std::mt19937 rng(12345);
  for (const Cand& c : cands) {
    if (c.n >= V || c.n < lower) continue;
    const int K = int(c.q.size());
    for (int trial = 0; trial < 4000; ++trial) {
      int a[3][4];
      for (int k = 0; k < K; ++k)
        for (int m = 0; m < 4; ++m) a[k][m] = int(rng() % c.q[k]);
      bool ok = true;
      for (auto& d : D) {
        bool sep = false;
        for (int k = 0; k < K && !sep; ++k) {
          long long v = 0;
          for (int m = 0; m < 4; ++m) v += (long long)a[k][m] * d[m];
          if (((v % c.q[k]) + c.q[k]) % c.q[k] != 0) sep = true;
        }
        if (!sep) {
          ok = false;
          break;
        }
      }
      if (!ok) continue;
      col.n = int(c.n);
      col.colour.resize(V);
      for (int s = 0; s < V; ++s) {
        int x[4] = {s % L[0], (s / L[0]) % L[1], (s / (L[0] * L[1])) % L[2], s / (L[0] * L[1] * L[2])};
        int cc = 0, stride = 1;
        for (int k = 0; k < K; ++k) {
          long long v = 0;
          for (int m = 0; m < 4; ++m) v += (long long)a[k][m] * x[m];
          cc += int(v % c.q[k]) * stride;
          stride *= c.q[k];
        }
        col.colour[s] = cc;
      }
      return col;
    }
  }
  col.n = V;  // fall back to unit vectors: every site its own colour
  col.colour.resize(V);
  std::iota(col.colour.begin(), col.colour.end(), 0);
  return col;
}

}  // namespace

extern "C" {

int mmc_deflate(mmc_ctx* ctx, int k, int poly_handle, int m_arn, double tol_accept, double* lambda_out,
                int* k_accepted) {
  TRY(check_ctx(ctx));
  if (k < 1 || m_arn < 2 || !k_accepted) RET(MMC_ERR_ARG, "mmc_deflate: bad argument");
  if (poly_handle != MMC_OP_M &&
      (!valid_poly(ctx, poly_handle) || ctx->polys[poly_handle].kind != 0 || ctx->polys[poly_handle].op != MMC_OP_M))
    RET(MMC_ERR_ARG, "mmc_deflate: poly_handle must be a single polynomial in M");
  cudaStream_t s = ctx->stream;
  const geom g = make_geom(ctx, 1);
  const size_t fb = field_bytes(g, MMC_F64);
  const size_t n = size_t(ctx->V) * 12;
  void *V;
  TRY(scratch(ctx, "df_V", fb * (m_arn + 1), &V));
  std::vector<uint2> ids(1, make_uint2(0u, 0u));
  void* dids;
  TRY(scratch(ctx, "ids", sizeof(uint2), &dids));
  CK(cudaMemcpyAsync(dids, ids.data(), sizeof(uint2), cudaMemcpyHostToDevice, s));
  CK(mmc::launch_noise(MMC_F64, g, (const uint2*)dids, MMC_TAG_ARNOLDI, ctx->seed, V, nullptr, s));
  ArnoldiOut ao;
  auto op = [&](const void* in, void* out) { return apply_op_f64(ctx, poly_handle, in, out, 1, s); };
  TRY(arnoldi_cgs2(ctx, g, MMC_F64, V, m_arn, op, ao, s));
  CMat Hm(m_arn, m_arn);
  for (int j = 0; j < m_arn; ++j)
    for (int i = 0; i < m_arn; ++i) Hm(i, j) = ao.H[0](i, j);
  std::vector<cd> mu;
  CMat G;
  if (!mmc::eig(Hm, mu, &G)) RET(MMC_ERR_NOCONV, "mmc_deflate: Ritz eigenproblem did not converge");
  // every Ritz vector z = V_m g, its Rayleigh quotient on M and residual
  void *Zc, *MZ, *Rv, *part;
  TRY(scratch(ctx, "df_Zc", fb * m_arn, &Zc));
  TRY(scratch(ctx, "df_MZ", fb, &MZ));
  TRY(scratch(ctx, "df_R", fb, &Rv));
  const int nbx = (g.V + kSpc - 1) / kSpc;
  TRY(scratch(ctx, "df_part", size_t(nbx) * std::max(m_arn, k) * sizeof(double2), &part));
  std::vector<cd> lam(m_arn);
  std::vector<double> res(m_arn);
  for (int i = 0; i < m_arn; ++i) {
    std::vector<cd> h(m_arn);
    for (int j = 0; j < m_arn; ++j) h[j] = -G(j, i);
    void* dh;
    TRY(upload(ctx, "df_h", h, &dh, s));
    char* zi = reinterpret_cast<char*>(Zc) + size_t(i) * fb;
    CK(cudaMemsetAsync(zi, 0, fb, s));
    CK(mmc::launch_basis_update(MMC_F64, g, V, n, m_arn, (const double2*)dh, zi, s));
    std::vector<double> nz;
    TRY(norms2(ctx, MMC_F64, g, zi, nz, s));
    std::vector<cd> sc(1, cd(1.0 / std::sqrt(nz[0]), 0));
    void* dsc;
    TRY(upload(ctx, "df_sc", sc, &dsc, s));
    CK(mmc::launch_axpby(MMC_F64, g, (const double2*)dsc, zi, nullptr, zi, s));
    TRY(apply_M_impl(ctx, zi, MZ, 1, MMC_F64, false, s));
    CK(mmc::launch_multidot(MMC_F64, g, zi, 0, 1, MZ, 0, kSpc, (double2*)part, s));
    std::vector<cd> l;
    TRY(reduce_to_host(ctx, (double2*)part, nbx, 1, 1, l, s));
    lam[i] = l[0];
    std::vector<cd> ca(1, -lam[i]), cb(1, cd(1, 0));
    void *dca, *dcb;
    TRY(upload(ctx, "df_ca", ca, &dca, s));
    TRY(upload(ctx, "df_cb", cb, &dcb, s));
    CK(cudaMemcpyAsync(Rv, MZ, fb, cudaMemcpyDeviceToDevice, s));
    CK(mmc::launch_axpby(MMC_F64, g, (const double2*)dca, zi, (const double2*)dcb, Rv, s));
    std::vector<double> rn;
    TRY(norms2(ctx, MMC_F64, g, Rv, rn, s));
    res[i] = std::sqrt(rn[0]);
  }
  // kept candidates and their gamma_5 partners (Sec. 8 acceptance; left vectors from
  // gamma_5-hermiticity, |Im| < 2e-4 counts as real)
  std::vector<int> keep, partner;
  mmc::deflation_pairs(lam, res, tol_accept, k, 2e-4, keep, partner);
  int kk = int(keep.size());
  if (ctx->Z) cudaFree(ctx->Z);
  if (ctx->U) cudaFree(ctx->U);
  if (ctx->Z32) cudaFree(ctx->Z32);
  if (ctx->U32) cudaFree(ctx->U32);
  ctx->Z = ctx->U = nullptr;
  ctx->Z32 = ctx->U32 = nullptr;
  for (auto& d : ctx->tc_dots) d.clear();
  for (auto& b : ctx->tcB) {
    if (b) cudaFree(b);
    b = nullptr;
  }
  ctx->k_defl = 0;
  ctx->lambda.clear();
  if (kk > 0) {
    CK(cudaMalloc(&ctx->Z, fb * kk));
    CK(cudaMalloc(&ctx->U, fb * kk));
    void* W;
    TRY(scratch(ctx, "df_W", fb * kk, &W));
    for (int i = 0; i < kk; ++i) {
      CK(cudaMemcpyAsync(reinterpret_cast<char*>(ctx->Z) + size_t(i) * fb,
                         reinterpret_cast<char*>(Zc) + size_t(keep[i]) * fb, fb, cudaMemcpyDeviceToDevice, s));
      CK(mmc::launch_gamma(MMC_F64, g, 2, reinterpret_cast<char*>(Zc) + size_t(partner[i]) * fb,
                           reinterpret_cast<char*>(W) + size_t(i) * fb, s));
    }
    // S = W^H Z (kk x kk), U = W S^{-H}
    CMat S(kk, kk);
    for (int j = 0; j < kk; ++j) {
      CK(mmc::launch_multidot(MMC_F64, g, W, n, kk, reinterpret_cast<char*>(ctx->Z) + size_t(j) * fb, 0, kSpc,
                              (double2*)part, s));
      std::vector<cd> col;
      TRY(reduce_to_host(ctx, (double2*)part, nbx, kk, 1, col, s));
      for (int i = 0; i < kk; ++i) S(i, j) = col[i];
    }
    // Variance control: with unit w_j, ||u_i|| follows the norm of column i of
    // Inv = (W^H Z)^{-H}, which grows where the kept set is nearly dependent, and the
    // deflated sample carries (eta^H Theta z_i)(u_i^H eta).  While the overlap is
    // singular the pair of largest |lambda| is dropped, while a column norm exceeds
    // the bound (100 by default) the pair with the largest one; either drop takes the
    // gamma_5 partner along.
    std::vector<int> mates(kk);
    for (int i = 0; i < kk; ++i) {
      mates[i] = i;
      for (int j = 0; j < kk; ++j)
        if (j != i && keep[j] == partner[i]) mates[i] = j;
    }
    std::vector<int> sel;
    CMat Inv;
    mmc::deflation_condition(S, mates, ctx->defl_max_u, sel, Inv);
    kk = int(sel.size());
    if (kk == 0) RET(MMC_ERR_BREAKDOWN, "mmc_deflate: W^H Z is singular");
    // compact Z and W to the selection (sel increases, so every copy moves a vector forward)
    for (int p2 = 0; p2 < kk; ++p2) {
      if (sel[p2] == p2) continue;
      CK(cudaMemcpyAsync(reinterpret_cast<char*>(ctx->Z) + size_t(p2) * fb,
                         reinterpret_cast<char*>(ctx->Z) + size_t(sel[p2]) * fb, fb, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(reinterpret_cast<char*>(W) + size_t(p2) * fb, reinterpret_cast<char*>(W) + size_t(sel[p2]) * fb,
                         fb, cudaMemcpyDeviceToDevice, s));
    }
    // Inv = S^{-H};  U_i = sum_j W_j Inv(j, i)
    for (int i = 0; i < kk; ++i) {
      std::vector<cd> h(kk);
      for (int j = 0; j < kk; ++j) h[j] = -Inv(j, i);
      void* dh;
      TRY(upload(ctx, "df_h", h, &dh, s));
      char* ui = reinterpret_cast<char*>(ctx->U) + size_t(i) * fb;
      CK(cudaMemsetAsync(ui, 0, fb, s));
      CK(mmc::launch_basis_update(MMC_F64, g, W, n, kk, (const double2*)dh, ui, s));
    }
    CK(cudaMalloc(&ctx->Z32, fb / 2 * kk));
    CK(cudaMalloc(&ctx->U32, fb / 2 * kk));
    const geom gk = {ctx->V * kk, 1, 1, 1};  // kk single vectors as one flat field
    CK(mmc::launch_convert(MMC_F32, ctx->Z32, MMC_F64, ctx->Z, gk, s));
    CK(mmc::launch_convert(MMC_F32, ctx->U32, MMC_F64, ctx->U, gk, s));
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < kk; ++i) ctx->lambda.push_back(lam[keep[sel[i]]]);
    ctx->k_defl = kk;
  }
  *k_accepted = kk;
  if (lambda_out)
    for (int i = 0; i < kk; ++i) {
      lambda_out[2 * i] = ctx->lambda[i].real();
      lambda_out[2 * i + 1] = ctx->lambda[i].imag();
    }
  return MMC_OK;
}

int mmc_set_deflation(mmc_ctx* ctx, int k, const double* lambda, const double* Z, const double* U) {
  TRY(check_ctx(ctx));
  if (k < 0 || (k > 0 && (!lambda || !Z || !U))) RET(MMC_ERR_ARG, "mmc_set_deflation: bad argument");
  cudaStream_t s = ctx->stream;
  if (ctx->Z) cudaFree(ctx->Z);
  if (ctx->U) cudaFree(ctx->U);
  if (ctx->Z32) cudaFree(ctx->Z32);
  if (ctx->U32) cudaFree(ctx->U32);
  ctx->Z = ctx->U = nullptr;
  ctx->Z32 = ctx->U32 = nullptr;
  for (auto& d : ctx->tc_dots) d.clear();
  for (auto& b : ctx->tcB) {
    if (b) cudaFree(b);
    b = nullptr;
  }
  ctx->k_defl = 0;
  ctx->lambda.clear();
  if (k == 0) return MMC_OK;
  const geom g1 = make_geom(ctx, 1);
  const size_t fb = field_bytes(g1, MMC_F64);
  const size_t n = size_t(ctx->V) * 12;
  CK(cudaMalloc(&ctx->Z, fb * k));
  CK(cudaMalloc(&ctx->U, fb * k));
  void* canon;
  TRY(scratch(ctx, "canon", fb, &canon));
  for (int i = 0; i < k; ++i) {  // canonical host order -> device single-vector layout ([site][12] either way)
    CK(cudaMemcpy(canon, Z + 2 * n * i, fb, cudaMemcpyHostToDevice));
    CK(mmc::launch_pack(MMC_F64, g1, 1, (const double2*)canon, ctx->Z + n * i, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(canon, U + 2 * n * i, fb, cudaMemcpyHostToDevice));
    CK(mmc::launch_pack(MMC_F64, g1, 1, (const double2*)canon, ctx->U + n * i, s));
    CK(cudaStreamSynchronize(s));
  }
  CK(cudaMalloc(&ctx->Z32, fb / 2 * k));
  CK(cudaMalloc(&ctx->U32, fb / 2 * k));
  const geom gk = {ctx->V * k, 1, 1, 1};
  CK(mmc::launch_convert(MMC_F32, ctx->Z32, MMC_F64, ctx->Z, gk, s));
  CK(mmc::launch_convert(MMC_F32, ctx->U32, MMC_F64, ctx->U, gk, s));
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < k; ++i) ctx->lambda.push_back(cd(lambda[2 * i], lambda[2 * i + 1]));
  ctx->k_defl = k;
  return MMC_OK;
}

int mmc_get_deflation(mmc_ctx* ctx, int* k, double* lambda, double* Z, double* U) {
  if (!ctx || !k) return MMC_ERR_ARG;
  *k = ctx->k_defl;
  if (!lambda && !Z && !U) return MMC_OK;
  CK(cudaSetDevice(ctx->device));
  const size_t n = size_t(ctx->V) * 12;
  for (int i = 0; i < ctx->k_defl; ++i) {
    if (lambda) {
      lambda[2 * i] = ctx->lambda[i].real();
      lambda[2 * i + 1] = ctx->lambda[i].imag();
    }
    if (Z) CK(cudaMemcpy(Z + 2 * n * i, ctx->Z + n * i, n * sizeof(double2), cudaMemcpyDeviceToHost));
    if (U) CK(cudaMemcpy(U + 2 * n * i, ctx->U + n * i, n * sizeof(double2), cudaMemcpyDeviceToHost));
  }
  return MMC_OK;
}

int mmc_set_tensor_projections(mmc_ctx* ctx, int enable) {
  if (!ctx) return MMC_ERR_ARG;
  ctx->use_tc = enable != 0;
  return MMC_OK;
}

int mmc_solve(mmc_ctx* ctx, const void* b, void* x, int nrhs, double rel_tol, int precond, int prec_inner,
              int m_inner, int max_outer, int* iters, double* relres_out) {
  TRY(check_ctx(ctx));
  if (!b || !x || b == x || nrhs < 1 || m_inner < 1 || max_outer < 0 || !(rel_tol > 0))
    RET(MMC_ERR_ARG, "mmc_solve: bad argument");
  if (prec_inner < MMC_F64 || prec_inner > MMC_BF16) RET(MMC_ERR_ARG, "mmc_solve: bad prec_inner");
  if (precond != MMC_ZERO && !valid_poly(ctx, precond) && !is_net(ctx, precond))
    RET(MMC_ERR_ARG, "mmc_solve: bad preconditioner handle");
  std::vector<double> rel;
  int rc = solve_impl(ctx, b, x, nrhs, rel_tol, precond, prec_inner, m_inner, max_outer, iters, rel, ctx->stream);
  if (relres_out)
    for (int i = 0; i < nrhs && i < int(rel.size()); ++i) relres_out[i] = rel[i];
  CK(cudaStreamSynchronize(ctx->stream));
  return rc;
}

namespace {

// Deflation correction and statistics of one level whose raw samples x[r] (r < n_noise)
// are formed: subtracts sum_i c_i (eta^H Theta z_i)(u_i^H eta) with c_i the level's
// scalar function at lambda_i and reports the exact correction sum_i c_i u_i^H Theta z_i
// (Sec. 7); mean, unbiased variances and standard errors (Sec. 4, Sec. 8).  g and codes
// describe the level's noise (rhs blocks of g.R, codes [rb][site][g.R]); `seconds` is
// the time already spent on the level, this call's own time is added.
int finish_level(mmc_ctx* ctx, int hi, int lo, int theta_op, int deflate, int n_noise, const geom& g,
                 const uint32_t* codes, int prec, std::vector<cd>& x, long long matvecs, double seconds,
                 mmc_level_stats* out, double* samples_out, cudaStream_t s) {
  const auto t1 = std::chrono::steady_clock::now();
  void* part;
  TRY(scratch(ctx, "lv_fpart", size_t((g.V + kSpc - 1) / kSpc) * std::max(g.npad, 1) * sizeof(double2), &part));
  cd corr(0, 0);
  int kd = 0;
  if (deflate && ctx->k_defl > 0) {
    const int k = ctx->k_defl;
    kd = k;
    const geom g1 = make_geom(ctx, 1);
    const int nb2 = (g.V + kSpc - 1) / kSpc;
    void *pa, *pb;
    TRY(scratch(ctx, "lv_pa", size_t(nb2) * k * g.npad * sizeof(double2), &pa));
    TRY(scratch(ctx, "lv_pb", size_t(nb2) * k * g.npad * sizeof(double2), &pb));
    const size_t n = size_t(ctx->V) * 12;
    std::vector<cd> A, B, D(k);
    if (prec != MMC_F64 && ctx->use_tc && k <= 128) {
      // tensor cores: one BF16 GEMM for both projections; the correction from the same BF16 copy
      const long long Kp = ((24ll * ctx->V + 63) / 64) * 64;
      if (!ctx->tcB[theta_op]) {
        CK(cudaMalloc(&ctx->tcB[theta_op], size_t(256) * Kp * 2));
        CK(mmc::launch_tc_pack_eig(ctx->V, k, Kp, theta_op, ctx->Z32, ctx->U32, ctx->tcB[theta_op], s));
      }
      const int mtiles = (2 * g.npad + 127) / 128;
      int nsplit = std::max(1, 148 / mtiles);
      nsplit = int(std::min<long long>(nsplit, Kp / 64));
      void *tpart, *tP, *terr, *tdots;
      TRY(scratch(ctx, "tc_part", size_t(nsplit) * mtiles * 128 * 256 * sizeof(float), &tpart));
      TRY(scratch(ctx, "tc_P", size_t(mtiles) * 128 * 256 * sizeof(double), &tP));
      TRY(scratch(ctx, "tc_err", sizeof(int), &terr));
      TRY(scratch(ctx, "tc_dots", size_t(k) * sizeof(double2), &tdots));
      CK(cudaMemsetAsync(terr, 0, sizeof(int), s));
      CK(mmc::launch_tc_proj(g, (const uint32_t*)codes, ctx->tcB[theta_op], Kp, nsplit, (float*)tpart, (double*)tP,
                             (int*)terr, s));
      // the exact correction's dots depend on the deflation data only: computed once per Theta
      const bool new_dots = ctx->tc_dots[theta_op].size() != size_t(k);
      if (new_dots) CK(mmc::launch_tc_pair_dots(Kp, k, ctx->tcB[theta_op], (double2*)tdots, s));
      std::vector<double> P(size_t(mtiles) * 128 * 256);
      std::vector<double2> dd(k);
      int herr = 0;
      CK(cudaMemcpyAsync(P.data(), tP, P.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      if (new_dots) CK(cudaMemcpyAsync(dd.data(), tdots, dd.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(&herr, terr, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (herr == 2) {
        // a bulk copy may still have been in flight when its CTA exited
        ctx->failed = true;
        RET(MMC_ERR_TIMEOUT, "mmc_trace_level: tensor-core projection gave up with copies in flight; "
                             "the context is retired (destroy it)");
      }
      if (herr) RET(MMC_ERR_TIMEOUT, "mmc_trace_level: tensor-core projection wait timed out");
      A.assign(size_t(k) * g.npad, cd(0, 0));
      B.assign(size_t(k) * g.npad, cd(0, 0));
      for (int i = 0; i < k; ++i)
        for (int r = 0; r < g.npad; ++r) {
          const double* row0 = &P[size_t(2 * r) * 256];
          const double* row1 = &P[size_t(2 * r + 1) * 256];
          A[size_t(i) * g.npad + r] = cd(row0[i], -row1[i]);
          B[size_t(i) * g.npad + r] = cd(row0[128 + i], row1[128 + i]);
        }
      if (new_dots) {
        ctx->tc_dots[theta_op].resize(k);
        for (int i = 0; i < k; ++i) ctx->tc_dots[theta_op][i] = cd(dd[i].x, dd[i].y);
      }
      D = ctx->tc_dots[theta_op];
    } else {
      const int dp = prec == MMC_F64 ? MMC_F64 : MMC_F32;  // eigenvector copy matching the level's precision
      const void* Zd = dp == MMC_F64 ? (const void*)ctx->Z : (const void*)ctx->Z32;
      const void* Ud = dp == MMC_F64 ? (const void*)ctx->U : (const void*)ctx->U32;
      CK(mmc::launch_defl_proj(dp, g, (const uint32_t*)codes, theta_op, Zd, Ud, k, kSpc, (double2*)pa, (double2*)pb,
                               s));
      TRY(reduce_to_host(ctx, (double2*)pa, nb2, k, g.npad, A, s));
      TRY(reduce_to_host(ctx, (double2*)pb, nb2, k, g.npad, B, s));
      for (int i = 0; i < k; ++i) {
        const void* ui =
            dp == MMC_F64 ? (const void*)(ctx->U + size_t(i) * n) : (const void*)(ctx->U32 + size_t(i) * n);
        const void* zi =
            dp == MMC_F64 ? (const void*)(ctx->Z + size_t(i) * n) : (const void*)(ctx->Z32 + size_t(i) * n);
        CK(mmc::launch_multidot(dp, g1, ui, 0, 1, zi, theta_op, kSpc, (double2*)part, s));
        std::vector<cd> d;
        TRY(reduce_to_host(ctx, (double2*)part, nb2, 1, 1, d, s));
        D[i] = d[0];
      }
    }
    for (int i = 0; i < k; ++i) {
      // c_i: the level's scalar function at lambda_i (1/lambda_i for M^-1)
      const cd fhi = hi == MMC_INV ? 1.0 / ctx->lambda[i] : poly_value(ctx, hi, ctx->lambda[i]);
      cd c = fhi - (lo == MMC_ZERO ? cd(0, 0) : poly_value(ctx, lo, ctx->lambda[i]));
      for (int r = 0; r < n_noise; ++r) x[r] -= c * A[size_t(i) * g.npad + r] * B[size_t(i) * g.npad + r];
      corr += c * D[i];
    }
  }
  // statistics (Sec. 4, Sec. 8 readings: unbiased variance of each part, stderr = s / sqrt(N))
  cd mean(0, 0);
  for (int r = 0; r < n_noise; ++r) mean += x[r];
  mean /= double(n_noise);
  double vr = 0, vi = 0, cv = 0;
  for (int r = 0; r < n_noise; ++r) {
    cd d = x[r] - mean;
    vr += d.real() * d.real();
    vi += d.imag() * d.imag();
    cv += std::norm(d);
  }
  const double dn = n_noise > 1 ? double(n_noise - 1) : 1.0;
  std::memset(out, 0, sizeof(*out));
  out->n = n_noise;
  out->k_deflated = kd;
  out->mean_re = mean.real();
  out->mean_im = mean.imag();
  out->var_re = n_noise > 1 ? vr / dn : 0.0;
  out->var_im = n_noise > 1 ? vi / dn : 0.0;
  out->cvar = n_noise > 1 ? cv / dn : 0.0;
  out->stderr_re = std::sqrt(out->var_re / n_noise);
  out->stderr_im = std::sqrt(out->var_im / n_noise);
  out->corr_re = corr.real();
  out->corr_im = corr.imag();
  out->value_re = mean.real() + corr.real();
  out->value_im = mean.imag() + corr.imag();
  out->matvecs = matvecs;
  out->seconds = seconds + std::chrono::duration<double>(std::chrono::steady_clock::now() - t1).count();
  if (samples_out)
    for (int r = 0; r < n_noise; ++r) {
      samples_out[2 * r] = x[r].real();
      samples_out[2 * r + 1] = x[r].imag();
    }
  for (int r = 0; r < n_noise; ++r)
    if (!std::isfinite(x[r].real()) || !std::isfinite(x[r].imag())) RET(MMC_ERR_NAN, "mmc_trace_level: NaN sample");
  return MMC_OK;
}

}  // namespace

int mmc_trace_level(mmc_ctx* ctx, int hi, int lo, int theta_op, int deflate, int n_noise, uint32_t first,
                    uint32_t level, int prec, int precond, mmc_level_stats* out, double* samples_out) {
  TRY(check_ctx(ctx));
  if (!out || n_noise < 1 || prec < 0 || prec > 2 || theta_op < 0 || theta_op > 2)
    RET(MMC_ERR_ARG, "mmc_trace_level: bad argument");
  if (!(hi == MMC_INV || valid_poly(ctx, hi) || is_net(ctx, hi)) ||
      !(lo == MMC_ZERO || valid_poly(ctx, lo) || is_net(ctx, lo)))
    RET(MMC_ERR_ARG, "mmc_trace_level: bad level operands");
  if (deflate && (is_net(ctx, hi) || is_net(ctx, lo)))
    RET(MMC_ERR_ARG, "mmc_trace_level: deflation needs polynomial operands (c_i = p_hi(lambda_i) - p_lo(lambda_i))");
  if (deflate && hi == MMC_INV && ctx->k_defl > 0)
    for (const cd& l : ctx->lambda)
      if (l == cd(0, 0)) RET(MMC_ERR_ARG, "mmc_trace_level: a deflated eigenvalue is zero (c_i = 1/lambda_i - ...)");
  const auto t0 = std::chrono::steady_clock::now();
  const long long mv0 = ctx->matvecs;
  cudaStream_t s = ctx->stream;
  const geom g = make_geom(ctx, n_noise);
  const int nbx = nbx_step(ctx);
  void *codes, *X, *part, *dids;
  TRY(scratch(ctx, "lv_codes", size_t(g.npad) * g.V * sizeof(uint32_t), &codes));
  TRY(scratch(ctx, "lv_X", field_bytes(g, prec), &X));
  TRY(scratch(ctx, "lv_part", size_t(std::max(nbx, (g.V + kSpc - 1) / kSpc)) * g.npad * sizeof(double2), &part));
  std::vector<uint2> ids(g.npad);
  for (int r = 0; r < g.npad; ++r) ids[r] = r < n_noise ? make_uint2(level, first + r) : make_uint2(0xffffffffu, 0);
  TRY(scratch(ctx, "lv_ids", ids.size() * sizeof(uint2), &dids));
  CK(cudaMemcpyAsync(dids, ids.data(), ids.size() * sizeof(uint2), cudaMemcpyHostToDevice, s));
  CK(mmc::launch_noise(prec, g, (const uint2*)dids, MMC_TAG_NOISE, ctx->seed, X, (uint32_t*)codes, s));
  std::vector<cd> x(g.npad, cd(0, 0));
  auto poly_bilinear = [&](int h, double sign) -> int {
    if (is_net(ctx, h)) {
      // learned operand: y = N eta in FP32, then eta^H Theta y
      void *x32, *y32;
      TRY(scratch(ctx, "lv_x32", field_bytes(g, MMC_F32), &x32));
      TRY(scratch(ctx, "lv_y32", field_bytes(g, MMC_F32), &y32));
      CK(mmc::launch_noise(MMC_F32, g, (const uint2*)dids, MMC_TAG_NOISE, ctx->seed, x32, nullptr, s));
      TRY(net_apply(ctx, h, x32, y32, g.npad, s, nullptr));
      const int nb2 = (g.V + kSpc - 1) / kSpc;
      CK(cudaMemsetAsync(part, 0, size_t(nb2) * g.npad * sizeof(double2), s));
      CK(mmc::launch_bilinear_codes(MMC_F32, g, (const uint32_t*)codes, theta_op, y32, kSpc, (double2*)part, s));
      std::vector<cd> v;
      TRY(reduce_to_host(ctx, (double2*)part, nb2, 1, g.npad, v, s));
      for (int r = 0; r < g.npad; ++r) x[r] += sign * v[r];
      return MMC_OK;
    }
    CK(cudaMemsetAsync(part, 0, size_t(nbx) * g.npad * sizeof(double2), s));
    Run base;
    base.g = g;
    base.prec = prec;
    base.codes = (const uint32_t*)codes;
    base.theta = theta_op;
    base.partial = (double2*)part;
    base.nbx = nbx;
    TRY(apply_poly_impl(ctx, h, X, n_noise, prec, ACC_BIL, nullptr, base, s));
    std::vector<cd> v;
    TRY(reduce_to_host(ctx, (double2*)part, nbx, 1, g.npad, v, s));
    for (int r = 0; r < g.npad; ++r) x[r] += sign * v[r];
    return MMC_OK;
  };
  if (hi == MMC_INV) {
    void *b64, *x64;
    TRY(scratch(ctx, "lv_b64", field_bytes(g, MMC_F64), &b64));
    TRY(scratch(ctx, "lv_x64", field_bytes(g, MMC_F64), &x64));
    CK(mmc::launch_noise(MMC_F64, g, (const uint2*)dids, MMC_TAG_NOISE, ctx->seed, b64, nullptr, s));
    // With a subtracted operand the solve starts at x0 = y = A_lo eta, whose residual
    // eta - M A_lo eta (pi_lo(M) eta for a polynomial, Sec. 3) is already small, and the
    // sample is eta^H Theta (x - y) with x - y formed in FP64: the difference M^-1 - A_lo
    // is never taken between two large bilinears.
    void* y64 = nullptr;
    if (lo != MMC_ZERO) {
      const size_t f64 = field_bytes(g, MMC_F64);
      TRY(scratch(ctx, "lv_y64", f64, &y64));
      if (is_net(ctx, lo)) {
        void *x32, *y32;
        TRY(scratch(ctx, "lv_x32", field_bytes(g, MMC_F32), &x32));
        TRY(scratch(ctx, "lv_y32", field_bytes(g, MMC_F32), &y32));
        CK(mmc::launch_noise(MMC_F32, g, (const uint2*)dids, MMC_TAG_NOISE, ctx->seed, x32, nullptr, s));
        TRY(net_apply(ctx, lo, x32, y32, g.npad, s, nullptr));
        CK(mmc::launch_convert(MMC_F64, y64, MMC_F32, y32, g, s));
      } else if (prec == MMC_F64) {
        Run base;
        base.g = g;
        base.prec = prec;
        TRY(apply_poly_impl(ctx, lo, X, n_noise, prec, ACC_Y, y64, base, s));
      } else {
        void* y32;
        TRY(scratch(ctx, "lv_y32", field_bytes(g, MMC_F32), &y32));
        Run base;
        base.g = g;
        base.prec = prec;
        TRY(apply_poly_impl(ctx, lo, X, n_noise, prec, ACC_Y, y32, base, s));
        CK(mmc::launch_convert(MMC_F64, y64, MMC_F32, y32, g, s));
      }
      CK(cudaMemcpyAsync(x64, y64, f64, cudaMemcpyDeviceToDevice, s));
    } else {
      CK(cudaMemsetAsync(x64, 0, field_bytes(g, MMC_F64), s));
    }
    std::vector<double> rel;
    int its = 0;
    // the plain FP64 form (prec = MMC_F64) solves in FP64 throughout; otherwise FP32 inner
    TRY(solve_impl(ctx, b64, x64, n_noise, 1e-10, precond, prec == MMC_F64 ? MMC_F64 : ctx->solve_inner, ctx->solve_m,
                   ctx->solve_max_outer, &its, rel, s));
    if (y64) {  // y <- x - y
      std::vector<cd> one(g.npad, cd(1, 0)), minus(g.npad, cd(-1, 0));
      void *d1, *dm;
      TRY(upload(ctx, "lv_one", one, &d1, s));
      TRY(upload(ctx, "lv_minus", minus, &dm, s));
      CK(mmc::launch_axpby(MMC_F64, g, (const double2*)d1, x64, (const double2*)dm, y64, s));
    }
    const int nb2 = (g.V + kSpc - 1) / kSpc;
    CK(cudaMemsetAsync(part, 0, size_t(nb2) * g.npad * sizeof(double2), s));
    CK(mmc::launch_bilinear_codes(MMC_F64, g, (const uint32_t*)codes, theta_op, y64 ? y64 : x64, kSpc,
                                  (double2*)part, s));
    std::vector<cd> v;
    TRY(reduce_to_host(ctx, (double2*)part, nb2, 1, g.npad, v, s));
    for (int r = 0; r < g.npad; ++r) x[r] += v[r];
  } else {
    TRY(poly_bilinear(hi, 1.0));
  }
  if (lo != MMC_ZERO && hi != MMC_INV) TRY(poly_bilinear(lo, -1.0));
  return finish_level(ctx, hi, lo, theta_op, deflate, n_noise, g, (const uint32_t*)codes, prec, x,
                      ctx->matvecs - mv0,
                      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(), out,
                      samples_out, s);
}

// Several polynomial levels in one batch.  Every level's hi and lo operand gets its own
// slot of rhs blocks (its noise repeated), and all single polynomials in M (Leja
// products, Sec. 3) run as one step chain: one launch per degree over the slots of
// every chain still running (per-block chain lengths), so the uneven noise counts
// and degrees of the levels share launches.  Double polynomials (Sec. 5) and
// degree-0 operands run on their own slots afterwards.  Samples, deflation and
// statistics are those of mmc_trace_level on the same noises.
int mmc_trace_levels(mmc_ctx* ctx, int n_levels, const int* hi, const int* lo, const int* n_noise,
                     const uint32_t* first, const uint32_t* level, int theta_op, int deflate, int prec,
                     mmc_level_stats* out, double* const* samples_out) {
  TRY(check_ctx(ctx));
  if (n_levels < 1 || !hi || !lo || !n_noise || !first || !level || !out || prec < 0 || prec > 2 || theta_op < 0 ||
      theta_op > 2)
    RET(MMC_ERR_ARG, "mmc_trace_levels: bad argument");
  for (int l = 0; l < n_levels; ++l) {
    if (n_noise[l] < 1) RET(MMC_ERR_ARG, "mmc_trace_levels: a level has no noise");
    if (!valid_poly(ctx, hi[l]) || !(lo[l] == MMC_ZERO || valid_poly(ctx, lo[l])))
      RET(MMC_ERR_ARG, "mmc_trace_levels: level operands must be polynomial handles (lo may be MMC_ZERO); "
                       "solve and network levels run through mmc_trace_level");
    for (int h : {hi[l], lo[l]})
      if (h != MMC_ZERO && ctx->polys[h].kind == 0 && ctx->polys[h].op != MMC_OP_M)
        RET(MMC_ERR_ARG, "mmc_trace_levels: polynomial in phi_h is not applicable alone");
  }
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = ctx->stream;
  struct Chain {
    int l, h;
    double sign;
    bool merged;
    int r0, slot;  // first rhs and padded rhs count of the chain's slot
  };
  std::vector<Chain> ch;
  long long nsum = 0;
  for (int pass = 0; pass < 2; ++pass)  // the merged chains first: their slots form a prefix
    for (int l = 0; l < n_levels; ++l)
      for (int side = 0; side < 2; ++side) {
        const int h = side == 0 ? hi[l] : lo[l];
        if (h == MMC_ZERO) continue;
        const Poly& P = ctx->polys[h];
        const bool merged = P.kind == 0 && P.theta.size() >= 2;
        if (merged != (pass == 0)) continue;
        ch.push_back({l, h, side == 0 ? 1.0 : -1.0, merged, 0, 0});
        nsum += n_noise[l];
      }
  // the longest merged chains first: the blocks still running at any step are a prefix,
  // so every launch's grid covers exactly them
  std::stable_sort(ch.begin(), ch.end(), [&](const Chain& a, const Chain& b) {
    if (a.merged != b.merged) return a.merged;
    if (!a.merged) return false;
    return ctx->polys[a.h].theta.size() > ctx->polys[b.h].theta.size();
  });
  if (nsum > (1ll << 24)) RET(MMC_ERR_ARG, "mmc_trace_levels: too many noise vectors in one batch");
  const int R = rhs_block(int(nsum), ctx->rhs_max);
  int npad_m = 0, npad_a = 0;
  for (Chain& c : ch) {
    c.slot = (n_noise[c.l] + R - 1) / R * R;
    c.r0 = npad_a;
    npad_a += c.slot;
    if (c.merged) npad_m = npad_a;
  }
  auto geom_of = [&](int npad) {
    geom g;
    g.V = ctx->V;
    g.R = R;
    g.nrb = npad / R;
    g.npad = npad;
    return g;
  };
  const geom ga = geom_of(npad_a);
  const int nbx = nbx_step(ctx);
  void *codes, *X, *part, *dids;
  TRY(scratch(ctx, "lv_codes", size_t(npad_a) * ga.V * sizeof(uint32_t), &codes));
  TRY(scratch(ctx, "lv_X", field_bytes(ga, prec), &X));
  TRY(scratch(ctx, "lv_part", size_t(std::max(nbx, (ga.V + kSpc - 1) / kSpc)) * npad_a * sizeof(double2), &part));
  std::vector<uint2> ids(npad_a);
  for (const Chain& c : ch)
    for (int j = 0; j < c.slot; ++j)
      ids[c.r0 + j] = j < n_noise[c.l] ? make_uint2(level[c.l], first[c.l] + j) : make_uint2(0xffffffffu, 0);
  TRY(scratch(ctx, "lv_ids", ids.size() * sizeof(uint2), &dids));
  CK(cudaMemcpyAsync(dids, ids.data(), ids.size() * sizeof(uint2), cudaMemcpyHostToDevice, s));
  CK(mmc::launch_noise(prec, ga, (const uint2*)dids, MMC_TAG_NOISE, ctx->seed, X, (uint32_t*)codes, s));

  std::vector<std::vector<cd>> x(n_levels);
  std::vector<double> secs(n_levels, 0.0);
  std::vector<long long> mvs(n_levels, 0);
  for (int l = 0; l < n_levels; ++l) x[l].assign(size_t(n_noise[l]), cd(0, 0));
  const size_t elem = elem_bytes(prec);
  if (npad_m > 0) {
    const geom gm = geom_of(npad_m);
    void *P0, *P1, *dlen;
    TRY(scratch(ctx, "P0", field_bytes(gm, prec), &P0));
    TRY(scratch(ctx, "P1", field_bytes(gm, prec), &P1));
    Run run;
    run.g = gm;
    run.prec = prec;
    run.codes = (const uint32_t*)codes;
    run.theta = theta_op;
    run.partial = (double2*)part;
    run.nbx = nbx;
    run.rb_len_host.assign(gm.nrb, 0);
    int steps = 0;
    for (const Chain& c : ch)
      if (c.merged) {
        const int len = int(ctx->polys[c.h].theta.size()) - 1;
        for (int b = c.r0 / R; b < (c.r0 + c.slot) / R; ++b) run.rb_len_host[b] = len;
        steps = std::max(steps, len);
      }
    TRY(scratch(ctx, "lv_rblen", size_t(gm.nrb) * sizeof(int), &dlen));
    CK(cudaMemcpyAsync(dlen, run.rb_len_host.data(), size_t(gm.nrb) * sizeof(int), cudaMemcpyHostToDevice, s));
    run.rb_len = (const int*)dlen;
    const double kap = ctx->kappa;
    void* P[2] = {P0, P1};
    for (int k = 0; k < steps; ++k) {
      // step k of every chain still running: prod_{k+1} = (1 - M/theta_k) prod_k, the
      // bilinear taking (1/theta_k) eta^H Theta prod_k and, on a chain's last step, its
      // last term (1/theta_m) eta^H Theta prod_m from the output (build_single's program)
      Step st;
      st.in = (k == 0) ? X : P[(k - 1) & 1];
      st.out = P[k & 1];
      st.flags = mmc::SF_HOP | mmc::SF_WRITE | mmc::SF_BIL_CODES;
      st.coef = coef_block(npad_m);
      for (const Chain& c : ch) {
        if (!c.merged) continue;
        const std::vector<cd>& th = ctx->polys[c.h].theta;
        const int m = int(th.size());
        if (k >= m - 1) continue;
        const cd it = 1.0 / th[k];
        const cd wo = (k == m - 2) ? 1.0 / th[m - 1] : cd(0, 0);
        if (k == m - 2) st.flags |= mmc::SF_BIL_OUT;
        for (int j = 0; j < n_noise[c.l]; ++j) set_coef(st.coef, npad_m, c.r0 + j, 1.0 - it, kap * it, 0, it, wo);
      }
      run.steps.push_back(st);
    }
    CK(cudaMemsetAsync(part, 0, size_t(nbx) * npad_m * sizeof(double2), s));
    const auto tm = std::chrono::steady_clock::now();
    TRY(exec_run(ctx, run, s));
    std::vector<cd> v;
    TRY(reduce_to_host(ctx, (double2*)part, nbx, 1, npad_m, v, s));
    // chain time shared by the levels in proportion to their rhs steps; the noise to all
    // levels in proportion to their slots
    const double t_chain = std::chrono::duration<double>(std::chrono::steady_clock::now() - tm).count();
    const double t_noise = std::chrono::duration<double>(tm - t0).count();
    double work = 0;
    for (const Chain& c : ch)
      if (c.merged) work += double(c.slot) * (ctx->polys[c.h].theta.size() - 1);
    for (const Chain& c : ch) {
      secs[c.l] += t_noise * double(c.slot) / npad_a;
      if (!c.merged) continue;
      const double w = double(c.slot) * (ctx->polys[c.h].theta.size() - 1);
      secs[c.l] += work > 0 ? t_chain * w / work : 0.0;
      mvs[c.l] += (long long)c.slot * (long long)(ctx->polys[c.h].theta.size() - 1);
      for (int j = 0; j < n_noise[c.l]; ++j) x[c.l][j] += c.sign * v[c.r0 + j];
    }
  } else {
    const double t_noise = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (const Chain& c : ch) secs[c.l] += t_noise * double(c.slot) / npad_a;
  }
  for (const Chain& c : ch) {
    if (c.merged) continue;
    const auto tc = std::chrono::steady_clock::now();
    const long long mv0 = ctx->matvecs;
    Run base;
    base.g = geom_of(c.slot);
    base.prec = prec;
    base.codes = (const uint32_t*)codes + size_t(c.r0) * ga.V;
    base.theta = theta_op;
    base.partial = (double2*)part;
    base.nbx = nbx;
    CK(cudaMemsetAsync(part, 0, size_t(nbx) * c.slot * sizeof(double2), s));
    const char* xc = (const char*)X + size_t(c.r0) * ga.V * 12 * elem;
    TRY(apply_poly_impl(ctx, c.h, xc, n_noise[c.l], prec, ACC_BIL, nullptr, base, s));
    std::vector<cd> v;
    TRY(reduce_to_host(ctx, (double2*)part, nbx, 1, c.slot, v, s));
    for (int j = 0; j < n_noise[c.l]; ++j) x[c.l][j] += c.sign * v[j];
    secs[c.l] += std::chrono::duration<double>(std::chrono::steady_clock::now() - tc).count();
    mvs[c.l] += ctx->matvecs - mv0;
  }
  for (int l = 0; l < n_levels; ++l) {
    // the level's noise: the slot of its first chain
    int r0 = -1;
    for (const Chain& c : ch)
      if (c.l == l && r0 < 0) r0 = c.r0;
    const geom gl = geom_of((n_noise[l] + R - 1) / R * R);
    TRY(finish_level(ctx, hi[l], lo[l], theta_op, deflate, n_noise[l], gl, (const uint32_t*)codes + size_t(r0) * ga.V,
                     prec, x[l], mvs[l], secs[l], &out[l], samples_out ? samples_out[l] : nullptr, s));
  }
  return MMC_OK;
}

int mmc_gmres_poly_deflated(mmc_ctx* ctx, int m, int op_handle, double* theta_out, int* handle) {
  TRY(check_ctx(ctx));
  if (m < 1 || !handle) RET(MMC_ERR_ARG, "mmc_gmres_poly_deflated: bad argument");
  if (ctx->k_defl < 1) RET(MMC_ERR_STATE, "mmc_gmres_poly_deflated: no deflation eigenpairs (mmc_deflate first)");
  if (op_handle != MMC_OP_M &&
      (!valid_poly(ctx, op_handle) || ctx->polys[op_handle].kind != 0 || ctx->polys[op_handle].op != MMC_OP_M))
    RET(MMC_ERR_ARG, "mmc_gmres_poly_deflated: op_handle must be a single polynomial in M");
  cudaStream_t s = ctx->stream;
  const geom g = make_geom(ctx, 1);
  void* V;
  TRY(scratch(ctx, "gmres_V", field_bytes(g, MMC_F64) * (m + 1), &V));
  std::vector<uint2> ids(g.npad, make_uint2(0u, 0u));
  void* dids;
  TRY(scratch(ctx, "ids", ids.size() * sizeof(uint2), &dids));
  CK(cudaMemcpyAsync(dids, ids.data(), ids.size() * sizeof(uint2), cudaMemcpyHostToDevice, s));
  CK(mmc::launch_noise(MMC_F64, g, (const uint2*)dids, MMC_TAG_GMRES, ctx->seed, V, nullptr, s));
  // b <- b - Z (U^H b): the start vector without its components along the deflated eigenvectors
  const int k = ctx->k_defl;
  const int nbx = (g.V + kSpc - 1) / kSpc;
  void* part;
  TRY(scratch(ctx, "gd_part", size_t(nbx) * k * g.npad * sizeof(double2), &part));
  CK(mmc::launch_vec_proj(MMC_F64, g, ctx->U, k, V, kSpc, (double2*)part, s));
  std::vector<cd> c;
  TRY(reduce_to_host(ctx, (double2*)part, nbx, k, g.npad, c, s));
  for (auto& v : c) v = -v;
  void* dc;
  TRY(upload(ctx, "gd_coef", c, &dc, s));
  CK(mmc::launch_vec_update(MMC_F64, g, ctx->Z, k, (const double2*)dc, V, s));
  ArnoldiOut ao;
  auto op = [&](const void* in, void* out) { return apply_op_f64(ctx, op_handle, in, out, 1, s); };
  TRY(arnoldi_cgs2(ctx, g, MMC_F64, V, m, op, ao, s));
  for (int j = 0; j < m; ++j)
    if (ao.H[0](j + 1, j) == cd(0, 0) && j < m - 1) RET(MMC_ERR_BREAKDOWN, "Arnoldi breakdown");
  std::vector<cd> th;
  if (!mmc::harmonic_ritz(ao.H[0], m, th)) RET(MMC_ERR_NOCONV, "harmonic Ritz eigenvalues did not converge");
  th = mmc::leja_order(th);
  for (auto& t : th)
    if (!std::isfinite(t.real()) || !std::isfinite(t.imag()) || t == cd(0, 0)) RET(MMC_ERR_NAN, "bad Ritz value");
  Poly P;
  P.kind = 0;
  P.theta = th;
  P.op = op_handle;
  ctx->polys.push_back(P);
  *handle = int(ctx->polys.size()) - 1;
  if (theta_out)
    for (int i = 0; i < m; ++i) {
      theta_out[2 * i] = th[i].real();
      theta_out[2 * i + 1] = th[i].imag();
    }
  return MMC_OK;
}

int mmc_probe_colours(mmc_ctx* ctx, int reach, int* n_colours) {
  if (!ctx || reach < 0 || !n_colours) return MMC_ERR_ARG;
  Colouring c = find_colouring(ctx->dims, ctx->V, reach);
  *n_colours = c.n;
  return MMC_OK;
}

int mmc_probe_colouring(const int dims[4], int reach, int* colour, int* n_colours) {
  if (!dims || reach < 0 || !n_colours) return MMC_ERR_ARG;
  long long V = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 2) return MMC_ERR_ARG;
    V *= dims[m];
  }
  if (V > (1ll << 30)) return MMC_ERR_ARG;
  Colouring c = find_colouring(dims, int(V), reach);
  *n_colours = c.n;
  if (colour) std::copy(c.colour.begin(), c.colour.end(), colour);
  return MMC_OK;
}

int mmc_set_deflation_bound(mmc_ctx* ctx, double max_u) {
  if (!ctx || !(max_u > 0)) return MMC_ERR_ARG;
  ctx->defl_max_u = max_u;
  return MMC_OK;
}

int mmc_trace_exact(mmc_ctx* ctx, int handle, int theta_op, int method, int prec, double* out) {
  TRY(check_ctx(ctx));
  const bool net = is_net(ctx, handle);
  if (!(valid_poly(ctx, handle) || net) || !out || prec < 0 || prec > 2 || theta_op < 0 || theta_op > 2)
    RET(MMC_ERR_ARG, "mmc_trace_exact: bad argument");
  if (net) prec = MMC_F32;  // the network runs in FP32
  cudaStream_t s = ctx->stream;
  Colouring col;
  if (method == MMC_EXACT_PROBE) {
    col = find_colouring(ctx->dims, ctx->V, net ? 3 : poly_degree(ctx, handle));
  } else {
    col.n = ctx->V;
    col.colour.resize(ctx->V);
    std::iota(col.colour.begin(), col.colour.end(), 0);
  }
  const long long nprobe = (long long)col.n * 12;
  const int batch = int(std::min<long long>(nprobe, 256));
  const geom g = make_geom(ctx, batch);
  const int nbx = nbx_step(ctx);
  void *dcol, *dpr, *X, *part;
  TRY(scratch(ctx, "ex_col", size_t(ctx->V) * sizeof(int), &dcol));
  CK(cudaMemcpyAsync(dcol, col.colour.data(), size_t(ctx->V) * sizeof(int), cudaMemcpyHostToDevice, s));
  TRY(scratch(ctx, "ex_pr", size_t(g.npad) * sizeof(int2), &dpr));
  TRY(scratch(ctx, "ex_X", field_bytes(g, prec), &X));
  TRY(scratch(ctx, "ex_part", size_t(nbx) * g.npad * sizeof(double2), &part));
  CK(cudaMemsetAsync(part, 0, size_t(nbx) * g.npad * sizeof(double2), s));
  std::vector<int2> pr(g.npad);
  cd net_total(0, 0);
  for (long long p0 = 0; p0 < nprobe; p0 += batch) {
    int nb = int(std::min<long long>(batch, nprobe - p0));
    for (int r = 0; r < g.npad; ++r) {
      long long pidx = p0 + r;
      pr[r] = (r < nb) ? make_int2(int(pidx / 12), int(pidx % 12)) : make_int2(-1, 0);
    }
    CK(cudaMemcpyAsync(dpr, pr.data(), pr.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    CK(mmc::launch_probe(prec, g, (const int*)dcol, (const int2*)dpr, X, s));
    if (net) {
      void* Y;
      TRY(scratch(ctx, "ex_Y", field_bytes(g, MMC_F32), &Y));
      TRY(net_apply(ctx, handle, X, Y, g.npad, s, nullptr));
      const int nb2 = (g.V + kSpc - 1) / kSpc;
      void* p2;
      TRY(scratch(ctx, "ex_part2", size_t(nb2) * g.npad * sizeof(double2), &p2));
      CK(mmc::launch_multidot(MMC_F32, g, X, 0, 1, Y, theta_op, kSpc, (double2*)p2, s));
      std::vector<cd> v;
      TRY(reduce_to_host(ctx, (double2*)p2, nb2, 1, g.npad, v, s));
      for (auto& z : v) net_total += z;
      continue;
    }
    Run base;
    base.g = g;
    base.prec = prec;
    base.left = X;
    base.theta = theta_op;
    base.partial = (double2*)part;
    base.nbx = nbx;
    TRY(apply_poly_impl(ctx, handle, X, g.npad, prec, ACC_BIL, nullptr, base, s));
    CK(cudaStreamSynchronize(s));  // probe table is rewritten by the next batch
  }
  cd tot = net_total;
  if (!net) {
    std::vector<cd> v;
    TRY(reduce_to_host(ctx, (double2*)part, nbx, 1, g.npad, v, s));
    for (auto& z : v) tot += z;
  }
  out[0] = tot.real();
  out[1] = tot.imag();
  return MMC_OK;
}

}  // extern "C"
