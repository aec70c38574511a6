// Host side of the C ABI declared in include/mmc.h: the context, the
// polynomial programs (Sec. 3, Sec. 5) turned into sequences of fused step
// launches, the CGS2 Arnoldi process (Sec. 3, Sec. 7), deflation (Sec. 7,
// Sec. 8), the refined deflated solves (Sec. 1, Sec. 8) and the Monte Carlo
// levels (Eq. 2, Sec. 6, Sec. 7).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "internal.h"

using namespace mmc::host;
using mmc::cd;
using mmc::CMat;
using mmc::geom;

// =====================================================================  C ABI
extern "C" {

int mmc_rhs_block(int nrhs) { return nrhs < 1 ? 1 : rhs_block(nrhs); }

size_t mmc_field_bytes(const mmc_ctx* ctx, int nrhs, int prec) {
  if (!ctx || nrhs < 1 || prec < 0 || prec > 2) return 0;
  return field_bytes(make_geom(ctx, nrhs), prec);
}

int mmc_create(mmc_ctx** out, const int dims[4], uint64_t seed, int device) {
  if (!out || !dims) return MMC_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 2) return MMC_ERR_ARG;
  mmc_ctx* ctx = new (std::nothrow) mmc_ctx();
  if (!ctx) return MMC_ERR_NOMEM;
  for (int i = 0; i < 4; ++i) ctx->dims[i] = dims[i];
  ctx->V = dims[0] * dims[1] * dims[2] * dims[3];
  ctx->seed = seed;
  ctx->device = device;
  cudaError_t e = cudaSetDevice(device);
  // a blocking stream: ordered with work on the legacy default stream (where torch allocates by default)
  if (e == cudaSuccess) e = cudaStreamCreate(&ctx->stream);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->step_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->step_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    if (ctx->step_err) cudaFree(ctx->step_err);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return MMC_ERR_CUDA;
  }
  *out = ctx;
  return MMC_OK;
}

int mmc_destroy(mmc_ctx* ctx) {
  if (!ctx) return MMC_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->scratch)
    if (kv.second.p) cudaFree(kv.second.p);
  if (ctx->links64) cudaFree(ctx->links64);
  if (ctx->links32) cudaFree(ctx->links32);
  if (ctx->nbr) cudaFree(ctx->nbr);
  if (ctx->order) cudaFree(ctx->order);
  if (ctx->order_zh) cudaFree(ctx->order_zh);
  if (ctx->salt) cudaFree(ctx->salt);
  for (auto& n : ctx->nets) {
    if (n.dw) cudaFree(n.dw);
    if (n.dwb) cudaFree(n.dwb);
  }
  if (ctx->step_err) cudaFree(ctx->step_err);
  if (ctx->Z) cudaFree(ctx->Z);
  if (ctx->U) cudaFree(ctx->U);
  if (ctx->Z32) cudaFree(ctx->Z32);
  if (ctx->U32) cudaFree(ctx->U32);
  for (auto b : ctx->tcB)
    if (b) cudaFree(b);
  prof_collect(ctx);
  clear_graphs(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (auto& kv : ctx->coef_cache) cudaFree(kv.second.p);
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return MMC_OK;
}

const char* mmc_last_error(const mmc_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

int mmc_set_seed(mmc_ctx* ctx, uint64_t seed) {
  if (!ctx) return MMC_ERR_ARG;
  ctx->seed = seed;
  return MMC_OK;
}

int mmc_load_gauge(mmc_ctx* ctx, const double* U, double kappa, int t_antiperiodic) {
  if (!ctx || !U) return MMC_ERR_ARG;
  CK(cudaSetDevice(ctx->device));
  const int V = ctx->V;
  // canonical [mu][site][3][3] -> device [site][mu][9] (FP64) and [site][mu][10] (FP32, padded)
  std::vector<double2> h64(size_t(V) * 4 * 9);
  std::vector<float2> h32(size_t(V) * 4 * 10, make_float2(0.f, 0.f));
  // the antiperiodic time phase is folded into U_t at t = Lt-1: both hops across the
  // boundary (forward from t = Lt-1, backward from t = 0) use that link
  const int slice = ctx->dims[0] * ctx->dims[1] * ctx->dims[2];
  for (int mu = 0; mu < 4; ++mu)
    for (int s = 0; s < V; ++s)
      for (int k = 0; k < 9; ++k) {
        size_t src = ((size_t(mu) * V + s) * 9 + k) * 2;
        const double ph = (t_antiperiodic && mu == 3 && s / slice == ctx->dims[3] - 1) ? -1.0 : 1.0;
        double re = ph * U[src], im = ph * U[src + 1];
        h64[(size_t(s) * 4 + mu) * 9 + k] = make_double2(re, im);
        h32[(size_t(s) * 4 + mu) * 10 + k] = make_float2(float(re), float(im));
      }
  {
    // neighbour table [site][8]: x + mu for mu = 0..3, then x - mu (periodic)
    std::vector<int> nb(size_t(V) * 8);
    const int* L = ctx->dims;
    for (int s = 0; s < V; ++s) {
      int c[4] = {s % L[0], (s / L[0]) % L[1], (s / (L[0] * L[1])) % L[2], s / (L[0] * L[1] * L[2])};
      int stride = 1;
      for (int mu = 0; mu < 4; ++mu) {
        nb[size_t(s) * 8 + mu] = (c[mu] == L[mu] - 1) ? s - (L[mu] - 1) * stride : s + stride;
        nb[size_t(s) * 8 + 4 + mu] = (c[mu] == 0) ? s + (L[mu] - 1) * stride : s - stride;
        stride *= L[mu];
      }
    }
    if (!ctx->nbr) CK(cudaMalloc(&ctx->nbr, nb.size() * sizeof(int)));
    CK(cudaMemcpy(ctx->nbr, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice));
    // traversal order in 4 x 4 x 2 x 2 blocks (64 sites, one CTA chunk): neighbours mostly in-block
    const int bl[4] = {4, 4, 2, 2};
    bool ok = true;
    for (int m = 0; m < 4; ++m) ok = ok && (L[m] % bl[m] == 0);
    if (ok) {
      std::vector<int> ord;
      ord.reserve(V);
      for (int bt = 0; bt < L[3] / bl[3]; ++bt)
        for (int bz = 0; bz < L[2] / bl[2]; ++bz)
          for (int by = 0; by < L[1] / bl[1]; ++by)
            for (int bx = 0; bx < L[0] / bl[0]; ++bx)
              for (int t = 0; t < bl[3]; ++t)
                for (int z = 0; z < bl[2]; ++z)
                  for (int y = 0; y < bl[1]; ++y)
                    for (int x = 0; x < bl[0]; ++x) {
                      const int X = bx * bl[0] + x, Y = by * bl[1] + y, Zc = bz * bl[2] + z, T = bt * bl[3] + t;
                      ord.push_back(X + L[0] * (Y + L[1] * (Zc + L[2] * T)));
                    }
      if (!ctx->order) CK(cudaMalloc(&ctx->order, ord.size() * sizeof(int)));
      CK(cudaMemcpy(ctx->order, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice));
    } else if (ctx->order) {
      cudaFree(ctx->order);
      ctx->order = nullptr;
    }
    // traversal z-half by z-half, each half t-major (t, z, y, x): the sites between a
    // spinor's reads as a t+1 neighbour and as a t-1 neighbour are two t-slices of a
    // half lattice, half of the lexicographic order's window
    if (L[2] % 2 == 0 && L[2] >= 4) {
      std::vector<int> ord;
      ord.reserve(V);
      const int hz = L[2] / 2;
      for (int zh = 0; zh < 2; ++zh)
        for (int t = 0; t < L[3]; ++t)
          for (int z = zh * hz; z < (zh + 1) * hz; ++z)
            for (int y = 0; y < L[1]; ++y)
              for (int x = 0; x < L[0]; ++x) ord.push_back(x + L[0] * (y + L[1] * (z + L[2] * t)));
      if (!ctx->order_zh) CK(cudaMalloc(&ctx->order_zh, ord.size() * sizeof(int)));
      CK(cudaMemcpy(ctx->order_zh, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice));
    } else if (ctx->order_zh) {
      cudaFree(ctx->order_zh);
      ctx->order_zh = nullptr;
    }
  }
  if (!ctx->links64) CK(cudaMalloc(&ctx->links64, h64.size() * sizeof(double2)));
  if (!ctx->links32) CK(cudaMalloc(&ctx->links32, h32.size() * sizeof(float2)));
  CK(cudaMemcpy(ctx->links64, h64.data(), h64.size() * sizeof(double2), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->links32, h32.data(), h32.size() * sizeof(float2), cudaMemcpyHostToDevice));
  {
    // special unitary links (third row = conjugate cross product of the first two, to
    // 1e-10): the step-kernel form that rebuilds third rows may then run
    void* flag;
    TRY(scratch(ctx, "su3_flag", sizeof(int), &flag));
    CK(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
    CK(mmc::launch_su3_rows_check((const double2*)ctx->links64, V, slice, ctx->dims[3], t_antiperiodic ? 1 : 0,
                                  (int*)flag, ctx->stream));
    int bad = 1;
    CK(cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->links_su3 = bad == 0;
  }
  ctx->kappa = kappa;
  ctx->tap = t_antiperiodic ? 1 : 0;
  ctx->gauge = true;
  ctx->polys.clear();
  ctx->k_defl = 0;
  ctx->lambda.clear();
  return MMC_OK;
}

int mmc_update_gauge(mmc_ctx* ctx, const double* U) {
  if (!ctx || !U) return MMC_ERR_ARG;
  if (!ctx->gauge) RET(MMC_ERR_STATE, "mmc_update_gauge: no gauge field loaded");
  auto polys = ctx->polys;
  const int kd = ctx->k_defl;
  auto lam = ctx->lambda;
  TRY(mmc_load_gauge(ctx, U, ctx->kappa, ctx->tap));
  ctx->polys = polys;
  ctx->k_defl = kd;
  ctx->lambda = lam;
  return MMC_OK;
}

int mmc_profile(mmc_ctx* ctx, int enable) {
  if (!ctx) return MMC_ERR_ARG;
  CK(cudaSetDevice(ctx->device));
  TRY(prof_collect(ctx));
  if (enable) {
    ctx->prof_launches = 0;
    ctx->prof_ms = ctx->prof_bytes = ctx->prof_flops = 0;
    ctx->prof_classes.clear();
    ctx->launches0 = mmc::launch_count();
    ctx->graph_launches0 = ctx->graph_launches;
    ctx->graph_captures0 = ctx->graph_captures;
  }
  ctx->prof = enable != 0;
  return MMC_OK;
}

int mmc_profile_read(mmc_ctx* ctx, mmc_profile_stats* out) {
  if (!ctx || !out) return MMC_ERR_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  TRY(prof_collect(ctx));
  out->step_launches = ctx->prof_launches;
  out->step_ms = ctx->prof_ms;
  out->step_bytes = ctx->prof_bytes;
  out->step_flops = ctx->prof_flops;
  out->all_launches = mmc::launch_count() - ctx->launches0;
  out->graph_launches = ctx->graph_launches - ctx->graph_launches0;
  out->graph_captures = ctx->graph_captures - ctx->graph_captures0;
  return MMC_OK;
}

int mmc_set_rounding(mmc_ctx* ctx, int mode, uint64_t seed) {
  if (!ctx || mode < 0 || mode > 1) return MMC_ERR_ARG;
  CK(cudaSetDevice(ctx->device));
  if (mode == 1) {
    if (!ctx->salt) CK(cudaMalloc(&ctx->salt, sizeof(uint32_t)));
    const uint32_t v = uint32_t(seed ^ (seed >> 32)) ^ 0x2545F491u;
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(ctx->salt, &v, sizeof(v), cudaMemcpyHostToDevice));
  }
  ctx->rounding = mode;
  return MMC_OK;
}

int mmc_profile_classes(mmc_ctx* ctx, int max_classes, mmc_profile_class* out, int* n_classes) {
  if (!ctx || !n_classes || max_classes < 0 || (max_classes > 0 && !out)) return MMC_ERR_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  TRY(prof_collect(ctx));
  *n_classes = int(ctx->prof_classes.size());
  for (int i = 0; i < std::min(max_classes, *n_classes); ++i) out[i] = ctx->prof_classes[i];
  return MMC_OK;
}

int mmc_set_solve_params(mmc_ctx* ctx, int m_inner, int max_outer) {
  if (!ctx) return MMC_ERR_ARG;
  if (m_inner > 0) ctx->solve_m = m_inner;
  if (max_outer > 0) ctx->solve_max_outer = max_outer;
  return MMC_OK;
}

int mmc_set_solve_refinement(mmc_ctx* ctx, double inner_reduction, int inner_cycles) {
  if (!ctx) return MMC_ERR_ARG;
  if (!(inner_reduction > 0.0 && inner_reduction <= 1.0) || inner_cycles < 1 || inner_cycles > 64)
    RET(MMC_ERR_ARG, "mmc_set_solve_refinement: reduction in (0, 1], cycles 1..64");
  ctx->solve_red = inner_reduction;
  ctx->solve_cycles = inner_cycles;
  return MMC_OK;
}

int mmc_set_gram_schmidt(mmc_ctx* ctx, int passes) {
  if (!ctx) return MMC_ERR_ARG;
  if (passes != 1 && passes != 2) RET(MMC_ERR_ARG, "mmc_set_gram_schmidt: 1 or 2 passes");
  ctx->solve_gs = passes;
  return MMC_OK;
}

int mmc_set_horner_layout(mmc_ctx* ctx, int paired) {
  if (!ctx) return MMC_ERR_ARG;
  if (paired != 0 && paired != 1) RET(MMC_ERR_ARG, "mmc_set_horner_layout: 0 or 1");
  ctx->horner_paired = paired;
  return MMC_OK;
}

int mmc_test_stall_staged(mmc_ctx* ctx, int enable, long long wait_iters) {
  if (!ctx || wait_iters < 0) return MMC_ERR_ARG;
  ctx->stall_test = enable != 0;
  ctx->wait_iters = wait_iters;
  return MMC_OK;
}

int mmc_set_rhs_block_max(mmc_ctx* ctx, int rmax) {
  if (!ctx) return MMC_ERR_ARG;
  if (rmax != 8 && rmax != 16) RET(MMC_ERR_ARG, "mmc_set_rhs_block_max: 8 or 16");
  ctx->rhs_max = rmax;
  return MMC_OK;
}

int mmc_set_solve_storage(mmc_ctx* ctx, int prec_inner) {
  if (!ctx) return MMC_ERR_ARG;
  if (prec_inner != MMC_F32 && prec_inner != MMC_BF16) RET(MMC_ERR_ARG, "mmc_set_solve_storage: MMC_F32 or MMC_BF16");
  ctx->solve_inner = prec_inner;
  return MMC_OK;
}

int mmc_set_step_variant(mmc_ctx* ctx, int prec, int rpt, int minb, int spc) {
  if (!ctx || prec < 0 || prec > 2) return MMC_ERR_ARG;
  if (minb >= 400) {  // minb = 400 + h: store hint of the fourth form (1: L2 evict-first)
    const int h = minb - 400;
    if (h < 0 || h > 1) RET(MMC_ERR_ARG, "store hint must be 0 or 1");
    ctx->var_hint[prec][0] = ctx->var_hint[prec][1] = h;
    minb = 0;
  } else if (minb >= 300) {  // minb = 300 + n: ring slots of the staged kernel (0: as many as fit)
    const int n = minb - 300;
    if (n != 0 && (n < 2 || n > 6)) RET(MMC_ERR_ARG, "ring slots must be 2..6 (or 0)");
    ctx->var_ns[prec][0] = ctx->var_ns[prec][1] = n;
    minb = 0;
  } else if (minb >= 200) {  // minb = 200 + b: traversal (0 lexicographic, 1 4D blocks, 2 z-halves)
    const int b = minb - 200;
    if (b < 0 || b > 2) RET(MMC_ERR_ARG, "traversal must be 0, 1 or 2");
    ctx->order_v[prec][0] = ctx->order_v[prec][1] = b;
    minb = 0;
  } else if (minb >= 100) {  // minb = 100 + v selects kernel version v (1: generic, 2: compile-time rhs block)
    ctx->var_ver[prec][0] = ctx->var_ver[prec][1] = minb - 100;
    minb = 0;
  }
  if (rpt > 0) {
    if (rpt != 1 && rpt != 2) RET(MMC_ERR_ARG, "rpt must be 1 or 2");
    ctx->var_rpt[prec][0] = ctx->var_rpt[prec][1] = prec == MMC_F64 ? 1 : rpt;
  }
  if (minb > 0) ctx->var_minb[prec][0] = ctx->var_minb[prec][1] = minb;
  if (spc > 0) {
    if (spc < 16 || spc > 1024 || (spc & (spc - 1))) RET(MMC_ERR_ARG, "spc must be a power of two in 16..1024");
    ctx->spc_v[prec][0] = ctx->spc_v[prec][1] = spc;
  }
  return MMC_OK;
}

int mmc_set_graphs(mmc_ctx* ctx, int enable) {
  if (!ctx) return MMC_ERR_ARG;
  if (!enable && ctx->use_graphs) {
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    clear_graphs(ctx);
  }
  ctx->use_graphs = enable != 0;
  if (enable) ctx->graph_note.clear();
  return MMC_OK;
}

const char* mmc_graph_note(const mmc_ctx* ctx) { return ctx ? ctx->graph_note.c_str() : ""; }

int mmc_set_step_variant_class(mmc_ctx* ctx, int prec, int rhs_class, int version, int rpt, int minb, int spc,
                               int blocked, int ns) {
  if (!ctx || prec < 0 || prec > 2 || rhs_class < 0 || rhs_class > 1) return MMC_ERR_ARG;
  if (version < 1 || version > 5 || (prec == MMC_F64 && version != 1)) RET(MMC_ERR_ARG, "bad kernel version");
  if (blocked < 0 || blocked > 2) RET(MMC_ERR_ARG, "traversal must be 0, 1 or 2");
  if (rpt != 1 && rpt != 2) RET(MMC_ERR_ARG, "rpt must be 1 or 2");
  if (minb < 1 || minb > 8) RET(MMC_ERR_ARG, "minb must be 1..8");
  if (spc < 16 || spc > 1024 || (spc & (spc - 1))) RET(MMC_ERR_ARG, "spc must be a power of two in 16..1024");
  if (ns != 0 && (ns < 2 || ns > 6)) RET(MMC_ERR_ARG, "ring slots must be 2..6 (or 0)");
  if (version == 5 && ns != 0 && ns != (prec == MMC_F32 ? 3 : 6) && ns != 4)
    RET(MMC_ERR_ARG, "pipeline depth of version 5: 3 or 4 (FP32), 4 or 6 (BF16), 0 for 4");
  ctx->var_ver[prec][rhs_class] = version;
  ctx->var_rpt[prec][rhs_class] = prec == MMC_F64 ? 1 : rpt;
  ctx->var_minb[prec][rhs_class] = minb;
  ctx->spc_v[prec][rhs_class] = spc;
  ctx->order_v[prec][rhs_class] = blocked;
  ctx->var_ns[prec][rhs_class] = ns;
  return MMC_OK;
}

int mmc_autotune(mmc_ctx* ctx, int nrhs, int prec, int* best, double* ms_out) {
  TRY(check_ctx(ctx));
  if (nrhs < 1 || prec < 0 || prec > 2) RET(MMC_ERR_ARG, "mmc_autotune: bad argument");
  cudaStream_t s = ctx->stream;
  geom g = make_geom(ctx, nrhs);
  void *x, *y, *codes, *part;
  TRY(scratch(ctx, "tune_x", field_bytes(g, prec), &x));
  TRY(scratch(ctx, "tune_y", field_bytes(g, prec), &y));
  TRY(scratch(ctx, "tune_codes", size_t(g.npad) * g.V * sizeof(uint32_t), &codes));
  // one row of bilinear partials per CTA of every variant tried, down to 16 sites per CTA
  const int nbx = std::max(nbx_step(ctx), nbx_for(ctx, 16));
  TRY(scratch(ctx, "tune_part", size_t(nbx) * g.npad * sizeof(double2), &part));
  std::vector<uint2> ids(g.npad);
  for (int r = 0; r < g.npad; ++r) ids[r] = make_uint2(7u, uint32_t(r));
  void* dids;
  TRY(scratch(ctx, "ids", ids.size() * sizeof(uint2), &dids));
  CK(cudaMemcpyAsync(dids, ids.data(), ids.size() * sizeof(uint2), cudaMemcpyHostToDevice, s));
  CK(mmc::launch_noise(prec, g, (const uint2*)dids, MMC_TAG_NOISE, ctx->seed, x, (uint32_t*)codes, s));
  CK(cudaMemsetAsync(part, 0, size_t(nbx) * g.npad * sizeof(double2), s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // The timed launch is one degree of a polynomial level chain, the form the levels
  // spend their time in: y = (1 - 1/t) x + (kappa/t) D x with the Z(4)-code bilinear
  // of x accumulated (the step kernel's epilogue decides its cost as much as the hop).
  Run run;
  run.g = g;
  run.prec = prec;
  run.codes = (const uint32_t*)codes;
  run.partial = (double2*)part;
  run.nbx = nbx;
  {
    Step st;
    st.in = x;
    st.out = y;
    st.flags = mmc::SF_HOP | mmc::SF_WRITE | mmc::SF_BIL_CODES;
    st.coef = coef_block(g.npad);
    const cd it(0.8, 0.3);
    for (int r = 0; r < g.npad; ++r) set_coef(st.coef, g.npad, r, 1.0 - it, ctx->kappa * it, 0, it, 0);
    run.steps.push_back(st);
  }
  float med = 0;
  auto time_variant = [&]() -> int {
    TRY(exec_run(ctx, run, s));
    std::vector<float> t;
    for (int rep = 0; rep < 3; ++rep) {
      CK(cudaEventRecord(e0, s));
      TRY(exec_run(ctx, run, s));
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      t.push_back(ms);
    }
    TRY(check_step_err(ctx, s));
    std::sort(t.begin(), t.end());
    med = t[1];
    return MMC_OK;
  };
  const int rpts[2] = {1, 2};
  const int minbs[3] = {1, 3, 4};
  const int minbs2[2] = {4, 6};  // v2, one rhs per lane: 128 or 80 registers
  const int spcs[4] = {32, 64, 128, 256};
  double best_ms = 1e300;
  const int rc = rclass(g.R);  // the variant is kept for this rhs-block class only
  int br = ctx->var_rpt[prec][rc], bm = ctx->var_minb[prec][rc], bs = ctx->spc_v[prec][rc], bv = ctx->var_ver[prec][rc];
  const bool v2ok = prec != MMC_F64 && (g.R == 8 || g.R == 16);
  int bo = ctx->order_v[prec][rc];
  for (int ordr = 0; ordr <= (v2ok ? 2 : 0); ++ordr)
  for (int ver = 1; ver <= (v2ok ? 2 : 1); ++ver)
  for (int ri = 0; ri < 2; ++ri) {
    if (ordr > 0 && ver == 1) continue;  // the traversal orders exist in the v2 and v4 kernels only
    if ((ordr == 1 && !ctx->order) || (ordr == 2 && !ctx->order_zh)) continue;
    if (prec == MMC_F64 && rpts[ri] != 1) continue;
    if (rpts[ri] > g.R) continue;
    const int nmb = ver == 1 ? 3 : (rpts[ri] == 1 ? 2 : 1);  // v2 with two rhs per lane has one cap
    for (int mi = 0; mi < nmb; ++mi) {
      const int mbv = ver == 1 ? minbs[mi] : (rpts[ri] == 1 ? minbs2[mi] : 3);
      for (int si = 0; si < 4; ++si) {
        ctx->var_ver[prec][rc] = ver;
        ctx->var_rpt[prec][rc] = rpts[ri];
        ctx->var_minb[prec][rc] = mbv;
        ctx->order_v[prec][rc] = ordr;
        ctx->spc_v[prec][rc] = spcs[si];
        TRY(time_variant());
        if (med < best_ms) {
          best_ms = med;
          br = rpts[ri];
          bm = mbv;
          bs = spcs[si];
          bv = ver;
          bo = ordr;
        }
      }
    }
  }
  int bn = ctx->var_ns[prec][rc];
  if (v2ok) {
    // the staged form (version 3) with its ring depths; rpt, caps and traversal do not apply
    const int nss[3] = {0, 2, 4};
    for (int ri = 0; ri < 2; ++ri)
    for (int ni = 0; ni < 3; ++ni) {
      if (rpts[ri] > g.R) continue;
      ctx->var_ver[prec][rc] = 3;
      ctx->var_ns[prec][rc] = nss[ni];
      ctx->var_rpt[prec][rc] = rpts[ri];
      ctx->order_v[prec][rc] = 0;
      TRY(time_variant());
      if (med < best_ms) {
        best_ms = med;
        bv = 3;
        bn = nss[ni];
        br = rpts[ri];
        bo = 0;
      }
    }
    // the persistent form with operands staged by asynchronous copies (version 5): depths, traversals
    for (int ordr = 0; ordr <= 2; ++ordr)
    for (int dp = 0; dp < 2; ++dp) {
      if ((ordr == 1 && !ctx->order) || (ordr == 2 && !ctx->order_zh)) continue;
      const int depth = prec == MMC_F32 ? (dp ? 4 : 3) : (dp ? 6 : 4);
      ctx->var_ver[prec][rc] = 5;
      ctx->var_rpt[prec][rc] = 1;
      ctx->var_ns[prec][rc] = depth;
      ctx->order_v[prec][rc] = ordr;
      TRY(time_variant());
      if (med < best_ms) {
        best_ms = med;
        bv = 5;
        br = 1;
        bn = depth;
        bo = ordr;
      }
    }
    // the persistent, pipelined form (version 4, one rhs per lane): register caps (3: 168
    // registers; 4: 128; 5: 128 with the links staged in shared memory; 6, special unitary
    // links: 168 with each link's third row rebuilt) and traversals
    for (int ordr = 0; ordr <= 2; ++ordr)
    for (int mb = 3; mb <= 6; ++mb) {
      if (mb == 6 && !ctx->links_su3) continue;
      if ((ordr == 1 && !ctx->order) || (ordr == 2 && !ctx->order_zh)) continue;
      ctx->var_ver[prec][rc] = 4;
      ctx->var_rpt[prec][rc] = 1;
      ctx->var_minb[prec][rc] = mb;
      ctx->var_ns[prec][rc] = 0;
      ctx->order_v[prec][rc] = ordr;
      TRY(time_variant());
      if (med < best_ms) {
        best_ms = med;
        bv = 4;
        br = 1;
        bm = mb;
        bn = 0;
        bo = ordr;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->var_rpt[prec][rc] = br;
  ctx->var_minb[prec][rc] = bm;
  ctx->spc_v[prec][rc] = bs;
  ctx->var_ver[prec][rc] = bv;
  ctx->var_ns[prec][rc] = bn;
  ctx->order_v[prec][rc] = bo;
  if (best) {
    best[0] = br;
    best[1] = bm;
    best[2] = bs;
    best[3] = bv;
    best[4] = bo;
    best[5] = bn;
  }
  if (ms_out) *ms_out = best_ms;
  return MMC_OK;
}

int mmc_pack(mmc_ctx* ctx, const double* host, int nrhs, int prec, void* field) {
  if (!ctx || !host || !field || nrhs < 1 || prec < 0 || prec > 2) return MMC_ERR_ARG;
  CK(cudaSetDevice(ctx->device));
  geom g = make_geom(ctx, nrhs);
  void* canon;
  const size_t bytes = size_t(nrhs) * ctx->V * 12 * sizeof(double2);
  TRY(scratch(ctx, "canon", bytes, &canon));
  CK(cudaMemcpyAsync(canon, host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  CK(mmc::launch_pack(prec, g, nrhs, (const double2*)canon, field, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MMC_OK;
}

int mmc_unpack(mmc_ctx* ctx, const void* field, int nrhs, int prec, double* host) {
  if (!ctx || !host || !field || nrhs < 1 || prec < 0 || prec > 2) return MMC_ERR_ARG;
  CK(cudaSetDevice(ctx->device));
  geom g = make_geom(ctx, nrhs);
  void* canon;
  const size_t bytes = size_t(nrhs) * ctx->V * 12 * sizeof(double2);
  TRY(scratch(ctx, "canon", bytes, &canon));
  CK(mmc::launch_unpack(prec, g, nrhs, field, (double2*)canon, ctx->stream));
  CK(cudaMemcpyAsync(host, canon, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MMC_OK;
}

int mmc_convert(mmc_ctx* ctx, const void* src, int src_prec, void* dst, int dst_prec, int nrhs, void* stream) {
  if (!ctx || !src || !dst || nrhs < 1 || src_prec < 0 || src_prec > 2 || dst_prec < 0 || dst_prec > 2)
    return MMC_ERR_ARG;
  if (src == dst) RET(MMC_ERR_ARG, "mmc_convert: src and dst must differ");
  CK(cudaSetDevice(ctx->device));
  CK(mmc::launch_convert(dst_prec, dst, src_prec, src, make_geom(ctx, nrhs), static_cast<cudaStream_t>(stream)));
  return MMC_OK;
}

int mmc_apply_M(mmc_ctx* ctx, const void* x, void* y, int nrhs, int prec, int dagger, void* stream) {
  TRY(check_ctx(ctx));
  if (!x || !y || x == y || nrhs < 1 || prec < 0 || prec > 2) RET(MMC_ERR_ARG, "mmc_apply_M: bad argument");
  return apply_M_impl(ctx, x, y, nrhs, prec, dagger != 0, (cudaStream_t)stream);
}

int mmc_noise(mmc_ctx* ctx, uint32_t level, uint32_t first, uint32_t tag, int nrhs, int prec, void* field,
              void* stream) {
  if (!ctx || !field || nrhs < 1 || prec < 0 || prec > 2) return MMC_ERR_ARG;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  geom g = make_geom(ctx, nrhs);
  std::vector<uint2> ids(g.npad);
  for (int r = 0; r < g.npad; ++r) ids[r] = r < nrhs ? make_uint2(level, first + r) : make_uint2(0xffffffffu, 0);
  void* dids;
  TRY(scratch(ctx, "ids", ids.size() * sizeof(uint2), &dids));
  CK(cudaMemcpyAsync(dids, ids.data(), ids.size() * sizeof(uint2), cudaMemcpyHostToDevice, s));
  CK(mmc::launch_noise(prec, g, (const uint2*)dids, tag, ctx->seed, field, nullptr, s));
  CK(cudaStreamSynchronize(s));  // ids buffer is reused by the next call
  return MMC_OK;
}

int mmc_poly_from_roots(mmc_ctx* ctx, int m, const double* theta, int* handle) {
  if (!ctx || m < 1 || !theta || !handle) return MMC_ERR_ARG;
  Poly P;
  P.kind = 0;
  for (int i = 0; i < m; ++i) {
    P.theta.push_back(cd(theta[2 * i], theta[2 * i + 1]));
    if (P.theta.back() == cd(0, 0)) RET(MMC_ERR_ARG, "zero root");
  }
  ctx->polys.push_back(P);
  *handle = int(ctx->polys.size()) - 1;
  return MMC_OK;
}

int mmc_poly_double(mmc_ctx* ctx, int h_in, int h_out, int* handle) {
  if (!ctx || !handle || !valid_poly(ctx, h_in) || !valid_poly(ctx, h_out)) return MMC_ERR_ARG;
  const Poly &Pi = ctx->polys[h_in], &Po = ctx->polys[h_out];
  if (Pi.kind != 0 || Pi.op != MMC_OP_M || Po.kind != 0) RET(MMC_ERR_ARG, "mmc_poly_double: needs single polynomials");
  Poly P;
  P.kind = 1;
  P.h_in = h_in;
  P.h_out = h_out;
  ctx->polys.push_back(P);
  *handle = int(ctx->polys.size()) - 1;
  return MMC_OK;
}

int mmc_poly_degree(const mmc_ctx* ctx, int handle) {
  if (!ctx || !valid_poly(ctx, handle)) return MMC_ERR_ARG;
  return poly_degree(ctx, handle);
}

int mmc_poly_eval(const mmc_ctx* ctx, int handle, int n, const double* alpha, double* out) {
  if (!ctx || !valid_poly(ctx, handle) || n < 0 || (n && (!alpha || !out))) return MMC_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    cd v = poly_value(ctx, handle, cd(alpha[2 * i], alpha[2 * i + 1]));
    out[2 * i] = v.real();
    out[2 * i + 1] = v.imag();
  }
  return MMC_OK;
}

int mmc_apply_poly(mmc_ctx* ctx, int handle, const void* x, void* y, int nrhs, int prec, void* stream) {
  TRY(check_ctx(ctx));
  if (!valid_poly(ctx, handle) || !x || !y || x == y || nrhs < 1 || prec < 0 || prec > 2)
    RET(MMC_ERR_ARG, "mmc_apply_poly: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  Run base;
  base.g = make_geom(ctx, nrhs);
  base.prec = prec;
  if (prec == MMC_BF16) {
    void* Y;
    TRY(scratch(ctx, "yacc", size_t(base.g.npad) * ctx->V * 12 * 8, &Y));
    TRY(apply_poly_impl(ctx, handle, x, nrhs, prec, ACC_Y, Y, base, s));
    CK(mmc::launch_convert(MMC_BF16, y, MMC_F32, Y, base.g, s));
    return MMC_OK;
  }
  return apply_poly_impl(ctx, handle, x, nrhs, prec, ACC_Y, y, base, s);
}

int mmc_gmres_poly(mmc_ctx* ctx, int m, int op_handle, double* theta_out, int* handle) {
  TRY(check_ctx(ctx));
  if (m < 1 || !handle) RET(MMC_ERR_ARG, "mmc_gmres_poly: bad argument");
  if (op_handle != MMC_OP_M) {
    if (!valid_poly(ctx, op_handle) || ctx->polys[op_handle].kind != 0 || ctx->polys[op_handle].op != MMC_OP_M)
      RET(MMC_ERR_ARG, "mmc_gmres_poly: op_handle must be a single polynomial in M");
  }
  cudaStream_t s = ctx->stream;
  geom g = make_geom(ctx, 1);
  void* V;
  TRY(scratch(ctx, "gmres_V", field_bytes(g, MMC_F64) * (m + 1), &V));
  std::vector<uint2> ids(g.npad, make_uint2(0u, 0u));
  void* dids;
  TRY(scratch(ctx, "ids", ids.size() * sizeof(uint2), &dids));
  CK(cudaMemcpyAsync(dids, ids.data(), ids.size() * sizeof(uint2), cudaMemcpyHostToDevice, s));
  CK(mmc::launch_noise(MMC_F64, g, (const uint2*)dids, MMC_TAG_GMRES, ctx->seed, V, nullptr, s));
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

int mmc_harmonic_ritz(int m, const double* H, int ldh, double* theta_out) {
  if (m < 1 || !H || !theta_out || ldh < m + 1) return MMC_ERR_ARG;
  CMat Hm(m + 1, m);
  for (int j = 0; j < m; ++j)
    for (int i = 0; i <= m; ++i) Hm(i, j) = cd(H[2 * (i + size_t(j) * ldh)], H[2 * (i + size_t(j) * ldh) + 1]);
  std::vector<cd> th;
  if (!mmc::harmonic_ritz(Hm, m, th)) return MMC_ERR_NOCONV;
  th = mmc::leja_order(th);
  for (int i = 0; i < m; ++i) {
    theta_out[2 * i] = th[i].real();
    theta_out[2 * i + 1] = th[i].imag();
  }
  return MMC_OK;
}

int mmc_leja_order(int m, const double* in, double* out) {
  if (m < 0 || (m && (!in || !out))) return MMC_ERR_ARG;
  std::vector<cd> p(m);
  for (int i = 0; i < m; ++i) p[i] = cd(in[2 * i], in[2 * i + 1]);
  p = mmc::leja_order(p);
  for (int i = 0; i < m; ++i) {
    out[2 * i] = p[i].real();
    out[2 * i + 1] = p[i].imag();
  }
  return MMC_OK;
}

int mmc_deflation_pairs(int m, const double* lambda, const double* res, double tol_accept, int k, int* keep,
                        int* partner, int* n_keep) {
  if (m < 0 || k < 0 || !n_keep || (m > 0 && (!lambda || !res || !keep || !partner))) return MMC_ERR_ARG;
  std::vector<cd> l(m);
  std::vector<double> r(res, res + m);
  for (int i = 0; i < m; ++i) l[i] = cd(lambda[2 * i], lambda[2 * i + 1]);
  std::vector<int> kp, pt;
  mmc::deflation_pairs(l, r, tol_accept, k, 2e-4, kp, pt);
  *n_keep = int(kp.size());
  for (size_t i = 0; i < kp.size(); ++i) {
    keep[i] = kp[i];
    partner[i] = pt[i];
  }
  return MMC_OK;
}

int mmc_deflation_condition(int q, const double* S, int lds, const int* mates, double max_u, int* sel,
                            int* n_sel) {
  if (q < 0 || !n_sel || (q > 0 && (!S || !mates || !sel || lds < q))) return MMC_ERR_ARG;
  CMat M(q, q);
  std::vector<int> mt(mates, mates + q);
  for (int i = 0; i < q; ++i)
    if (mt[i] < 0 || mt[i] >= q) return MMC_ERR_ARG;
  for (int j = 0; j < q; ++j)
    for (int i = 0; i < q; ++i) M(i, j) = cd(S[2 * (i + size_t(j) * lds)], S[2 * (i + size_t(j) * lds) + 1]);
  std::vector<int> sl;
  CMat Inv;
  mmc::deflation_condition(M, mt, max_u, sl, Inv);
  *n_sel = int(sl.size());
  for (size_t i = 0; i < sl.size(); ++i) sel[i] = sl[i];
  return MMC_OK;
}

int mmc_eig(int n, const double* A, int lda, double* w, double* vr) {
  if (n < 1 || !A || !w || lda < n) return MMC_ERR_ARG;
  CMat M(n, n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) M(i, j) = cd(A[2 * (i + size_t(j) * lda)], A[2 * (i + size_t(j) * lda) + 1]);
  std::vector<cd> ev;
  CMat Vr;
  if (!mmc::eig(M, ev, vr ? &Vr : nullptr)) return MMC_ERR_NOCONV;
  for (int i = 0; i < n; ++i) {
    w[2 * i] = ev[i].real();
    w[2 * i + 1] = ev[i].imag();
  }
  if (vr)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        vr[2 * (i + size_t(j) * n)] = Vr(i, j).real();
        vr[2 * (i + size_t(j) * n) + 1] = Vr(i, j).imag();
      }
  return MMC_OK;
}

}  // extern "C"
