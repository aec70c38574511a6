// Internals shared by the host translation units: the context, scratch
// buffers, the step-program runner, polynomial programs and the Arnoldi
// process.  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/mmc.h"
#include "dense.h"
#include "kernels.h"

namespace mmc {
namespace host {

struct Poly {
  int kind = 0;                 // 0: single in `base`, 1: double
  std::vector<cd> theta;        // single: Leja-ordered roots
  int op = MMC_OP_M;            // single: MMC_OP_M, or handle h (a polynomial in phi_h)
  int h_in = -1, h_out = -1;    // double: p_in in M, p_out in phi_in
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Learned gauge-covariant stencil network: channels 4 -> 8 -> 8 -> 4, three layers,
// weights per layer [9][C_out][C_in] complex (host FP64 copy, device FP32 copy).
struct Net {
  std::vector<std::complex<double>> w;  // 1152 complex
  float2* dw = nullptr;                 // device copy, same order
  __nv_bfloat162* dwb = nullptr;        // BF16 device copy (BF16 network)
  bool bf16 = false;                    // BF16 weights and hidden activations, FP32 accumulation
};
constexpr int kNetCh[4] = {4, 8, 8, 4};
constexpr int kNetWeights = 9 * (8 * 4 + 8 * 8 + 4 * 8);
constexpr int kNetBase = 0x100000;

}  // namespace host
}  // namespace mmc

struct mmc_ctx {
  int dims[4] = {0, 0, 0, 0};
  int V = 0;
  uint64_t seed = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  double kappa = 0;
  int tap = 1;
  bool gauge = false;
  void* links64 = nullptr;
  void* links32 = nullptr;
  bool links_su3 = false;  // every link special unitary (to 1e-10): a link's third row follows from two
  std::vector<mmc::host::Poly> polys;
  std::vector<mmc::host::Net> nets;
  // deflation data (FP64 single-vector fields [site][12])
  int k_defl = 0;
  std::vector<mmc::cd> lambda;
  double2* Z = nullptr;
  double2* U = nullptr;
  float2* Z32 = nullptr;  // FP32 copies used by the FP32 / BF16 levels (projections and correction alike)
  float2* U32 = nullptr;
  // BF16 copies [Theta z; u] for the tensor-core projections of BF16 levels, per Theta
  void* tcB[3] = {nullptr, nullptr, nullptr};
  std::vector<mmc::cd> tc_dots[3];  // u_i^H Theta z_i from the BF16 copies (per Theta; kept with tcB)
  bool use_tc = true;
  std::map<std::string, mmc::host::DevBuf> scratch;
  // device copies of step coefficient tables, keyed by a hash of their contents:
  // a polynomial applied again (preconditioner, chains of later steps) reuses its
  // table without a host-to-device copy or a stream synchronisation
  std::map<uint64_t, mmc::host::DevBuf> coef_cache;
  size_t coef_cache_bytes = 0;
  // CUDA graphs of step chains, keyed by a hash of everything that decides their
  // launches (coefficient table, operand pointers, flags, kernel variant): a chain
  // run again with the same buffers replays its graph (one launch for all degrees)
  struct ChainGraph {
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;  // kernel launches captured (for the launch counter)
  };
  std::map<uint64_t, ChainGraph> graph_cache;
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;  // private non-blocking stream the graphs are captured on
  long long graph_launches = 0;       // chains run as graph replays
  long long graph_launches0 = 0;      // value at the last mmc_profile(ctx, 1)
  long long graph_captures = 0, graph_captures0 = 0;
  std::string graph_note;             // why graphs were switched off, if they were
  bool failed = false;         // set when a kernel may have left work in flight: every later call refuses
  int rounding = 0;            // BF16 chain storage: 0 round to nearest, 1 stochastic (mmc_set_rounding)
  uint32_t* salt = nullptr;    // device word: stochastic-rounding salt, advanced once per BF16 chain
  double defl_max_u = 100.0;  // mmc_deflate: bound on the norm of a left vector u_i (a column of (W^H Z)^{-H})
  int solve_m = 48;        // inner FGMRES length of the M^-1 level solves
  int solve_max_outer = 400;
  int solve_gs = 1;          // Gram-Schmidt passes of the FP32 stage's Arnoldi (1 or 2)
  int horner_paired = 1;     // FP32 8-rhs Horner chains of the solves in the paired-component layout
  double solve_red = 3e-2;   // FP32 stage of the refined solves: gain per FP64 residual
  int solve_cycles = 8;      // and its most FGMRES cycles
  long long wait_iters = 0;   // bound of the staged kernel's mbarrier waits (0: its default)
  int stall_test = 0;         // fault injection for tests: the staged kernel's producer copies nothing
  int rhs_max = 16;           // largest rhs block R of the blocked field layout (8 or 16)
  int solve_inner = MMC_F32;  // inner FGMRES storage of the reduced-precision levels' solves (F32 or BF16)
  std::string err;
  long long matvecs = 0;
  int spc_v[3][2] = {{64, 64}, {64, 64}, {64, 64}};  // sites per CTA of the step kernel (per variant class)
  // step-kernel variant per precision and rhs-block class (R < 16, R = 16)
  int var_rpt[3][2] = {{1, 1}, {2, 2}, {2, 2}};
  int var_minb[3][2] = {{1, 1}, {1, 1}, {1, 1}};
  int var_ver[3][2] = {{1, 1}, {2, 2}, {2, 2}};  // 1: step_kernel, 2: step2_kernel, 3: step3_kernel (F32, BF16)
  int var_ns[3][2] = {{0, 0}, {0, 0}, {0, 0}};   // ring slots of step3_kernel (0: as many as fit)
  int* step_err = nullptr;     // device flag of the staged step kernel's bounded waits
  int* nbr = nullptr;          // device neighbour table [site][8]
  int* order = nullptr;        // device traversal order in 4D blocks (null if the extents do not allow it)
  int* order_zh = nullptr;     // device traversal order z-half by z-half, t-major within a half (null if Lz is odd)
  // traversal of the step kernel (versions 2, 4): 0 lexicographic, 1 4D blocks, 2 z-halves
  int order_v[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  int var_hint[3][2] = {{0, 0}, {0, 0}, {0, 0}};  // store hint of the fourth form (bit 0: L2 evict-first)
  // profiling (mmc_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  struct PendingEv {
    cudaEvent_t e0, e1;
    int cls;  // index into prof_classes
  };
  std::vector<PendingEv> ev_pending;
  std::vector<mmc_profile_class> prof_classes;  // per launch class (chain kind, precision, padded rhs)
  long long prof_launches = 0;
  double prof_ms = 0, prof_bytes = 0, prof_flops = 0;
  long long launches0 = 0;
};

namespace mmc {
namespace host {
using mmc::cd;
using mmc::CMat;
using mmc::geom;

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                    \
      return MMC_ERR_CUDA;                                                              \
    }                                                                                   \
  } while (0)

#define RET(code, msg)    \
  do {                    \
    ctx->err = (msg);     \
    return (code);        \
  } while (0)

#define TRY(expr)          \
  do {                     \
    int rc_ = (expr);      \
    if (rc_ != MMC_OK) return rc_; \
  } while (0)

inline size_t elem_bytes(int prec) { return prec == MMC_F64 ? 16 : (prec == MMC_F32 ? 8 : 4); }

inline int rhs_block(int nrhs, int rmax = 16) {
  int R = 1;
  while (R < nrhs && R < rmax) R <<= 1;
  return R;
}

inline geom make_geom(const mmc_ctx* ctx, int nrhs) {
  geom g;
  g.V = ctx->V;
  g.R = rhs_block(nrhs, ctx->rhs_max);
  g.nrb = (nrhs + g.R - 1) / g.R;
  g.npad = g.nrb * g.R;
  return g;
}

inline size_t field_bytes(const geom& g, int prec) { return size_t(g.npad) * g.V * 12 * elem_bytes(prec); }

// Get (and grow) a named scratch buffer owned by the context.
inline int scratch(mmc_ctx* ctx, const std::string& key, size_t bytes, void** out) {
  DevBuf& b = ctx->scratch[key];
  if (b.bytes < bytes) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
      b.p = nullptr;
      ctx->err = "cudaMalloc(" + key + ", " + std::to_string(bytes) + "): " + cudaGetErrorString(e);
      return MMC_ERR_NOMEM;
    }
    b.bytes = bytes;
  }
  *out = b.p;
  return MMC_OK;
}

inline int rclass(int R) { return R >= 16 ? 1 : 0; }

inline int rpt_for(const mmc_ctx* ctx, int prec, int R) {
  if (prec == MMC_F64) return 1;
  return std::min(ctx->var_rpt[prec][rclass(R)], R);
}

inline int log2i(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// ------------------------------------------------------------- step runner
struct Step {
  const void* in = nullptr;
  void* out = nullptr;
  const void* aux = nullptr;
  int flags = 0;
  std::vector<cd> coef;  // [5][npad]
};

struct Run {
  geom g;
  int prec = MMC_F64;
  void* y = nullptr;              // accumulator field (double2 for F64, float2 otherwise)
  const uint32_t* codes = nullptr;
  const void* left = nullptr;
  int theta = 0;
  double2* partial = nullptr;     // [nbx][npad]
  int nbx = 0;
  const int* rb_len = nullptr;     // device: steps per rhs block (blocks with step >= len skip)
  std::vector<int> rb_len_host;   // the same on the host (launch accounting)
  bool dagger = false;
  std::vector<Step> steps;
};

inline int nbx_for(const mmc_ctx* ctx, int spc) { return (ctx->V + spc - 1) / spc; }
// Rows of the bilinear partial buffers of a step chain: one per CTA of the site-chunked
// forms (the smallest sites-per-CTA of any variant), one per compute warp of the staged
// form (up to 16 warps on each of 152 SMs).
inline int nbx_step(const mmc_ctx* ctx) {
  int spc = 1 << 30;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 2; ++b) spc = std::min(spc, ctx->spc_v[a][b]);
  return std::max(nbx_for(ctx, spc), 152 * 16);
}

inline int prof_event(mmc_ctx* ctx, cudaEvent_t* e) {
  if (ctx->ev_pool.empty()) {
    cudaEvent_t ev;
    CK(cudaEventCreate(&ev));
    ctx->ev_pool.push_back(ev);
  }
  *e = ctx->ev_pool.back();
  ctx->ev_pool.pop_back();
  return MMC_OK;
}

// Collect the elapsed times of finished event pairs (synchronises on each pair).
inline int prof_collect(mmc_ctx* ctx) {
  for (auto& pr : ctx->ev_pending) {
    CK(cudaEventSynchronize(pr.e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, pr.e0, pr.e1));
    ctx->prof_ms += ms;
    if (pr.cls >= 0 && pr.cls < int(ctx->prof_classes.size())) ctx->prof_classes[pr.cls].ms += ms;
    ctx->ev_pool.push_back(pr.e0);
    ctx->ev_pool.push_back(pr.e1);
  }
  ctx->ev_pending.clear();
  return MMC_OK;
}

inline void clear_graphs(mmc_ctx* ctx) {
  for (auto& kv : ctx->graph_cache)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  ctx->graph_cache.clear();
}

inline int exec_run(mmc_ctx* ctx, Run& run, cudaStream_t s) {
  if (run.steps.empty()) return MMC_OK;
  const geom& g = run.g;
  const size_t per = size_t(5) * g.npad;
  std::vector<double2> host(per * run.steps.size());
  for (size_t k = 0; k < run.steps.size(); ++k)
    for (size_t i = 0; i < per; ++i)
      host[k * per + i] = make_double2(run.steps[k].coef[i].real(), run.steps[k].coef[i].imag());
  // hash of the table (and its size) as the cache key: FNV-1a over 64-bit words, with
  // the high half folded in after each multiply
  uint64_t key = 1469598103934665603ull ^ host.size();
  {
    const uint64_t* w = reinterpret_cast<const uint64_t*>(host.data());
    const size_t nw = host.size() * sizeof(double2) / sizeof(uint64_t);
    for (size_t i = 0; i < nw; ++i) {
      key = (key ^ w[i]) * 1099511628211ull;
      key ^= key >> 29;
    }
  }
  void* dcoef = nullptr;
  auto hit = ctx->coef_cache.find(key);
  if (hit != ctx->coef_cache.end() && hit->second.bytes == host.size() * sizeof(double2)) {
    dcoef = hit->second.p;
  } else {
    const size_t nb = host.size() * sizeof(double2);
    if (ctx->coef_cache_bytes + nb > (size_t(256) << 20)) {  // bounded: drop the whole cache
      CK(cudaStreamSynchronize(s));
      for (auto& kv : ctx->coef_cache) cudaFree(kv.second.p);
      ctx->coef_cache.clear();
      ctx->coef_cache_bytes = 0;
      clear_graphs(ctx);
    }
    DevBuf b;
    CK(cudaMalloc(&b.p, nb));
    b.bytes = nb;
    CK(cudaMemcpyAsync(b.p, host.data(), nb, cudaMemcpyHostToDevice, s));
    ctx->coef_cache[key] = b;
    ctx->coef_cache_bytes += nb;
    dcoef = b.p;
  }
  const int rpt = rpt_for(ctx, run.prec, g.R);
  const int rc = rclass(g.R);
  const bool prof = ctx->prof;
  {
    // The site-chunked forms write one row of bilinear partials per CTA: refuse a launch
    // whose grid would need more rows than the run's partial buffer holds.
    int any = 0;
    for (const Step& st : run.steps) any |= st.flags;
    if ((any & (mmc::SF_BIL_CODES | mmc::SF_BIL_LEFT)) &&
        (!run.partial || nbx_for(ctx, ctx->spc_v[run.prec][rc]) > run.nbx))
      RET(MMC_ERR_ARG, "step chain: bilinear partial buffer has fewer rows than the launch has CTAs");
  }
  int cls = -1;  // profiling class of this run: chain kind, precision, padded rhs count
  if (prof) {
    int any = 0;
    for (const Step& st : run.steps) any |= st.flags;
    const int kind = (any & (mmc::SF_BIL_CODES | mmc::SF_BIL_LEFT)) ? MMC_PROF_BILINEAR
                     : (any & mmc::SF_YACC)                          ? MMC_PROF_ACCUMULATE
                     : (any & mmc::SF_AUX)                           ? MMC_PROF_AUX
                                                                     : MMC_PROF_PLAIN;
    for (size_t c = 0; c < ctx->prof_classes.size(); ++c) {
      const mmc_profile_class& pc = ctx->prof_classes[c];
      if (pc.kind == kind && pc.prec == run.prec && pc.nrhs_padded == g.npad) cls = int(c);
    }
    if (cls < 0) {
      mmc_profile_class pc;
      std::memset(&pc, 0, sizeof(pc));
      pc.kind = kind;
      pc.prec = run.prec;
      pc.nrhs_padded = g.npad;
      ctx->prof_classes.push_back(pc);
      cls = int(ctx->prof_classes.size()) - 1;
    }
  }
  // stochastic rounding of BF16 chains: a fresh salt per chain application, advanced on
  // the device by the chain's first launch (so a replayed graph advances it too)
  const bool sr = ctx->rounding == 1 && run.prec == MMC_BF16 && ctx->salt;
  // the staged form (3) rounds to nearest only: stochastic rounding runs the second form
  const int ver_run = (sr && ctx->var_ver[run.prec][rc] == 3) ? 2 : ctx->var_ver[run.prec][rc];
  // one launch per step; with per-launch profiling events unless the chain is captured
  auto launch_steps = [&](bool events, cudaStream_t s) -> int {
    if (sr) CK(mmc::launch_salt_advance(ctx->salt, s));
    for (size_t k = 0; k < run.steps.size(); ++k) {
      const Step& st = run.steps[k];
      // with per-block chain lengths the grid covers the blocks up to the last one still
      // running (all of them when the longest chains come first); the others skip
      int nrb_k = g.nrb;
      if (!run.rb_len_host.empty()) {
        nrb_k = 0;
        for (int b = 0; b < int(run.rb_len_host.size()); ++b)
          if (int(k) < run.rb_len_host[b]) nrb_k = b + 1;
        if (nrb_k == 0) continue;
      }
      mmc::step_params p;
      std::memset(&p, 0, sizeof(p));
      p.in = st.in;
      p.out = st.out;
      p.aux = st.aux;
      p.y = run.y;
      p.codes = run.codes;
      p.left = run.left;
      p.coef = reinterpret_cast<const double2*>(dcoef) + k * per;
      p.partial = run.partial;
      p.links = run.prec == MMC_F64 ? ctx->links64 : ctx->links32;
      p.rb_len = run.rb_len;
      p.nbr = ctx->nbr;
      p.order = ctx->order_v[run.prec][rc] == 1 ? ctx->order : ctx->order_v[run.prec][rc] == 2 ? ctx->order_zh : nullptr;
      p.hint = ctx->var_hint[run.prec][rc];
      p.salt = sr ? ctx->salt : nullptr;
      p.step = int(k);
      p.V = ctx->V;
      p.R = g.R;
      p.logL = log2i(g.R / rpt);
      p.npad = g.npad;
      p.spc = ctx->spc_v[run.prec][rc];
      p.Lx = ctx->dims[0];
      p.Ly = ctx->dims[1];
      p.Lz = ctx->dims[2];
      p.Lt = ctx->dims[3];
      p.tap = ctx->tap;
      p.theta = run.theta;
      p.flags = st.flags | (run.dagger ? mmc::SF_DAGGER : 0);
      p.err = ctx->step_err;
      p.wait_iters = ctx->wait_iters;
      p.stall_test = ctx->stall_test;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (events) {
        TRY(prof_event(ctx, &e0));
        TRY(prof_event(ctx, &e1));
        CK(cudaEventRecord(e0, s));
      }
      bool done = false;
      if (p.flags & mmc::SF_PAIRED) {
        // the paired-component layout exists in the fourth form only (FP32, 8-rhs blocks, 168
        // registers); no other kernel reads it, so there is no fallback
        cudaError_t e4 = cudaSuccess;
        const int mb = (ctx->var_minb[run.prec][rc] == 6 && ctx->links_su3) ? 6 : 3;
        if (run.prec != MMC_F32 || g.R != 8 || !mmc::launch_step4_f32(g.R, mb, p, nrb_k, 1 << 30, s, &e4))
          RET(MMC_ERR_ARG, "exec_run: the paired-component layout needs FP32 8-rhs Horner steps");
        CK(e4);
        done = true;
      }
      if (!done && ver_run == 5 && run.prec != MMC_F64 && (g.R == 8 || g.R == 16)) {
        cudaError_t e5 = cudaSuccess;
        const int ns = ctx->var_ns[run.prec][rc];
        const int nbx = run.nbx > 0 ? run.nbx : (1 << 30);
        done = run.prec == MMC_F32 ? mmc::launch_step5_f32(g.R, ns == 3 ? 3 : 4, p, nrb_k, nbx, s, &e5)
                                   : mmc::launch_step5_bf16(g.R, ns == 6 ? 6 : 4, p, nrb_k, nbx, s, &e5);
        CK(e5);
      }
      if (!done && ver_run == 4 && run.prec != MMC_F64 && (g.R == 8 || g.R == 16)) {
        cudaError_t e4 = cudaSuccess;
        const int mbr = ctx->var_minb[run.prec][rc];
        // 6 (rebuilt third link rows) needs special unitary links, else the 168-register form
        const int mb = mbr == 3 ? 3 : mbr == 5 ? 5 : mbr == 6 ? (ctx->links_su3 ? 6 : 3) : 4;
        const int nbx = run.nbx > 0 ? run.nbx : (1 << 30);
        done = run.prec == MMC_F32 ? mmc::launch_step4_f32(g.R, mb, p, nrb_k, nbx, s, &e4)
                                   : mmc::launch_step4_bf16(g.R, mb, p, nrb_k, nbx, s, &e4);
        CK(e4);
      }
      if (!done && ver_run == 3 && run.prec != MMC_F64 && (g.R == 8 || g.R == 16)) {
        cudaError_t e3 = cudaSuccess;
        done = mmc::launch_step3(run.prec, g.R, rpt, run.nbx, ctx->var_ns[run.prec][rc], p, nrb_k, s, &e3);
        CK(e3);
      }
      if (!done && ver_run >= 2 && run.prec != MMC_F64 && (g.R == 8 || g.R == 16)) {
        cudaError_t e2 = cudaSuccess;
        const int mb = ctx->var_minb[run.prec][rc];
        done = run.prec == MMC_F32 ? mmc::launch_step2_f32(g.R, rpt, mb, p, nrb_k, s, &e2)
                                   : mmc::launch_step2_bf16(g.R, rpt, mb, p, nrb_k, s, &e2);
        CK(e2);
      }
      if (!done) CK(mmc::launch_step(run.prec, rpt, ctx->var_minb[run.prec][rc], p, nrb_k, s));
      if (events) {
        CK(cudaEventRecord(e1, s));
        ctx->ev_pending.push_back({e0, e1, cls});
        if (ctx->ev_pending.size() > 65536) TRY(prof_collect(ctx));
      }
    }
    return MMC_OK;
  };

  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(s, &cap));
  mmc_ctx::ChainGraph* cgp = nullptr;  // the graph to replay, if any
  if (ctx->use_graphs && run.steps.size() >= 2 && cap == cudaStreamCaptureStatusNone) {
    // key: everything the launches depend on
    uint64_t gk = 1469598103934665603ull;
    auto mix = [&gk](uint64_t v) {
      for (int b = 0; b < 8; ++b) gk = (gk ^ ((v >> (8 * b)) & 0xff)) * 1099511628211ull;
    };
    mix(key);
    mix(reinterpret_cast<uintptr_t>(dcoef));
    mix(reinterpret_cast<uintptr_t>(run.y));
    mix(reinterpret_cast<uintptr_t>(run.codes));
    mix(reinterpret_cast<uintptr_t>(run.left));
    mix(reinterpret_cast<uintptr_t>(run.partial));
    mix(reinterpret_cast<uintptr_t>(run.rb_len));
    for (int len : run.rb_len_host) mix(uint64_t(uint32_t(len)));
    mix(reinterpret_cast<uintptr_t>(run.prec == MMC_F64 ? ctx->links64 : ctx->links32));
    mix(uint64_t(run.theta) | (uint64_t(run.nbx) << 8) | (uint64_t(run.dagger) << 40) | (uint64_t(run.prec) << 48));
    mix(uint64_t(g.npad) | (uint64_t(g.R) << 32) | (uint64_t(ctx->stall_test) << 63));
    mix(uint64_t(ctx->wait_iters) ^ (uint64_t(sr) << 62));
    mix(uint64_t(ctx->var_ver[run.prec][rc]) | (uint64_t(rpt) << 8) | (uint64_t(ctx->var_minb[run.prec][rc]) << 16) |
        (uint64_t(ctx->spc_v[run.prec][rc]) << 24) | (uint64_t(ctx->order_v[run.prec][rc]) << 40) |
        (uint64_t(ctx->var_ns[run.prec][rc]) << 48) | (uint64_t(ctx->var_hint[run.prec][rc]) << 56));
    for (const Step& st : run.steps) {
      mix(reinterpret_cast<uintptr_t>(st.in));
      mix(reinterpret_cast<uintptr_t>(st.out));
      mix(reinterpret_cast<uintptr_t>(st.aux));
      mix(uint64_t(st.flags));
    }
    auto it = ctx->graph_cache.find(gk);
    if (it == ctx->graph_cache.end()) {
      if (ctx->graph_cache.size() >= 512) {  // bounded
        CK(cudaStreamSynchronize(s));
        clear_graphs(ctx);
      }
      // captured on the context's private non-blocking stream (a blocking stream is
      // tied to the legacy default stream), replayed on s
      if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
      mmc_ctx::ChainGraph cg;
      bool built = false;
      const long long n0 = mmc::launch_count();
      cudaError_t be = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (be == cudaSuccess) {
        const int rc_launch = launch_steps(false, ctx->cap_stream);
        cudaGraph_t graph = nullptr;
        be = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (rc_launch == MMC_OK && be == cudaSuccess && graph) be = cudaGraphInstantiate(&cg.exec, graph, 0);
        built = rc_launch == MMC_OK && be == cudaSuccess && cg.exec;
        if (graph) cudaGraphDestroy(graph);
      }
      mmc::count_launch(-int(mmc::launch_count() - n0));  // counted when the graph (or the fallback) runs
      if (built) {
        cg.kernels = int(run.steps.size());
        cgp = &ctx->graph_cache.emplace(gk, cg).first->second;
        ctx->graph_captures += 1;
      } else {
        // capture refused: launch directly from now on and keep the reason
        cudaGetLastError();
        if (cg.exec) cudaGraphExecDestroy(cg.exec);
        ctx->use_graphs = false;
        ctx->graph_note = std::string("graph capture failed, direct launches: ") + cudaGetErrorString(be);
      }
    } else {
      cgp = &it->second;
    }
  }
  if (cgp) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (prof) {
      TRY(prof_event(ctx, &e0));
      TRY(prof_event(ctx, &e1));
      CK(cudaEventRecord(e0, s));
    }
    CK(cudaGraphLaunch(cgp->exec, s));
    mmc::count_launch(cgp->kernels);
    ctx->graph_launches += 1;
    if (prof) {
      CK(cudaEventRecord(e1, s));
      ctx->ev_pending.push_back({e0, e1, cls});
      if (ctx->ev_pending.size() > 65536) TRY(prof_collect(ctx));
    }
  }
  if (!cgp) TRY(launch_steps(prof, s));
  for (size_t k = 0; k < run.steps.size(); ++k) {
    const Step& st = run.steps[k];
    // rhs of the launch's active blocks (all of them without per-block chain lengths)
    int active = g.npad;
    if (!run.rb_len_host.empty()) {
      active = 0;
      for (int len : run.rb_len_host) active += (int(k) < len) ? g.R : 0;
    }
    if (prof) {
      ctx->prof_launches += 1;
      // algorithmic bytes and flops of this launch (all rhs blocks active), the bytes
      // at ideal reuse: every input, output, aux, accumulator and left-field element
      // once, the 4 links of a site (9 complex each, no padding) once for the whole
      // batch, and nothing for the Z(4) noise of the code bilinear (it could be
      // regenerated from the counter-based generator instead of read)
      const double sb = double(elem_bytes(run.prec)) * 12;  // one spinor, one rhs
      const double per_rhs = sb * ((st.flags & mmc::SF_HOP) ? 2 : 1) * ((st.flags & mmc::SF_WRITE) ? 1 : 0) +
                             (((st.flags & mmc::SF_WRITE) == 0) ? sb : 0.0) +
                             ((st.flags & mmc::SF_AUX) ? sb : 0.0) +
                             ((st.flags & mmc::SF_YACC) ? 2.0 * 12 * (run.prec == MMC_F64 ? 16 : 8) : 0.0) +
                             ((st.flags & mmc::SF_BIL_LEFT) ? sb : 0.0);
      const double links = (st.flags & mmc::SF_HOP) ? 4.0 * 9 * (run.prec == MMC_F64 ? 16 : 8) : 0.0;
      const double bytes = active ? double(ctx->V) * (double(active) * per_rhs + links) : 0.0;
      const double flops = double(ctx->V) * active * (((st.flags & mmc::SF_HOP) ? 1368.0 : 0.0) + 48.0);
      ctx->prof_bytes += bytes;
      ctx->prof_flops += flops;
      mmc_profile_class& pc = ctx->prof_classes[cls];
      pc.launches += 1;
      pc.bytes += bytes;
      pc.flops += flops;
    }
    if (st.flags & mmc::SF_HOP) ctx->matvecs += active;
  }
  return MMC_OK;
}

// The staged step kernel records a bounded wait that gave up in ctx->step_err; read
// (and clear) it once the work is done.
inline int check_step_err(mmc_ctx* ctx, cudaStream_t s) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->step_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h == 2) {
    // a staged copy may have been in flight when its CTA exited: nothing launched on this
    // context can be trusted any more
    ctx->failed = true;
    RET(MMC_ERR_TIMEOUT, "step kernel: a bounded wait for staged copies gave up with copies in flight; "
                         "the context is retired (destroy it)");
  }
  if (h) {
    CK(cudaMemsetAsync(ctx->step_err, 0, sizeof(int), s));
    RET(MMC_ERR_TIMEOUT, "step kernel: a bounded wait for staged rows gave up");
  }
  return MMC_OK;
}

inline std::vector<cd> coef_block(int npad) { return std::vector<cd>(size_t(5) * npad, cd(0, 0)); }

// coefficient setter for rhs r: out = a in + b D in + g aux; accumulations w_in, w_out
inline void set_coef(std::vector<cd>& c, int npad, int r, cd a, cd b, cd gg, cd wi, cd wo) {
  c[0 * size_t(npad) + r] = a;
  c[1 * size_t(npad) + r] = b;
  c[2 * size_t(npad) + r] = gg;
  c[3 * size_t(npad) + r] = wi;
  c[4 * size_t(npad) + r] = wo;
}

// Accumulation mode of a polynomial program.
enum AccMode { ACC_Y = 0, ACC_BIL = 1 };

inline int acc_flags(AccMode m, const Run& run) {
  if (m == ACC_Y) return mmc::SF_YACC;
  return run.codes ? mmc::SF_BIL_CODES : mmc::SF_BIL_LEFT;
}

// Append the steps of a single polynomial p (roots th, in M) applied to the field `x`:
// accumulates sum_k u_k (Sec. 3) into y (ACC_Y) or into the bilinear (ACC_BIL).
// Ping-pong buffers P0, P1.  `scale` multiplies every accumulated term.
inline void build_single(const mmc_ctx* ctx, Run& run, const std::vector<cd>& th, const void* x, void* P0, void* P1,
                  AccMode mode, cd scale, int nrhs) {
  const int m = int(th.size());
  const int npad = run.g.npad;
  const double kap = ctx->kappa;
  const int accf = acc_flags(mode, run);
  if (m == 1) {
    Step st;
    st.in = x;
    st.flags = accf;
    st.coef = coef_block(npad);
    for (int r = 0; r < nrhs; ++r) set_coef(st.coef, npad, r, 0, 0, 0, scale / th[0], 0);
    run.steps.push_back(st);
    return;
  }
  void* P[2] = {P0, P1};
  for (int k = 0; k < m - 1; ++k) {
    Step st;
    st.in = (k == 0) ? x : P[(k - 1) & 1];
    st.out = P[k & 1];
    st.flags = mmc::SF_HOP | mmc::SF_WRITE | accf;
    if (k == m - 2) st.flags |= mmc::SF_BIL_OUT;  // the last prod's term rides on this step
    st.coef = coef_block(npad);
    cd it = 1.0 / th[k];
    cd wo = (k == m - 2) ? scale / th[m - 1] : cd(0, 0);
    for (int r = 0; r < nrhs; ++r) set_coef(st.coef, npad, r, 1.0 - it, kap * it, 0, scale * it, wo);
    run.steps.push_back(st);
  }
}

// Steps of p(M) x in Horner nesting, p(M) x = c_1 x + (1 - M/t_1)(c_2 x + (1 - M/t_2)(... c_m x)),
// c_k = 1/t_k: the same polynomial as the sum of u_k (Sec. 3) with no accumulator field;
// each step reads the iterate (neighbours) and x (site-local) and writes the next iterate.
// Used where any fixed evaluation of p will do (the FGMRES preconditioner).  m >= 2.
inline void build_horner(const mmc_ctx* ctx, Run& run, const std::vector<cd>& th, const void* x, void* P0, void* P1,
                         void* out, int nrhs) {
  const int m = int(th.size());
  const int npad = run.g.npad;
  const double kap = ctx->kappa;
  void* P[2] = {P0, P1};
  int n = 0;
  for (int k = m - 2; k >= 0; --k, ++n) {
    Step st;
    st.coef = coef_block(npad);
    const cd ck = 1.0 / th[k], it = 1.0 / th[k];
    st.out = (k == 0) ? out : P[n & 1];
    st.flags = mmc::SF_HOP | mmc::SF_WRITE;
    if (k == m - 2) {
      // w = c_{m-1} x folded in: out = [c_{m-1}(1 - 1/t_k) + c_k] x + c_{m-1} (kappa/t_k) D x
      const cd cm = 1.0 / th[m - 1];
      st.in = x;
      for (int r = 0; r < nrhs; ++r) set_coef(st.coef, npad, r, cm * (1.0 - it) + ck, cm * kap * it, 0, 0, 0);
    } else {
      st.in = P[(n - 1) & 1];
      st.aux = x;
      st.flags |= mmc::SF_AUX;
      for (int r = 0; r < nrhs; ++r) set_coef(st.coef, npad, r, 1.0 - it, kap * it, ck, 0, 0);
    }
    run.steps.push_back(st);
  }
}

// Steps of the double polynomial p_in(M) p_out(phi_in(M)) (Sec. 5) applied to the
// field `w` that already holds p_in(M) x in storage precision (A[0]).  Buffers:
// P0, P1 (inner ping-pong), A0, A1 (outer iterate).  Accumulates sum_k over
// p_out's terms into y or the bilinear.
inline void build_double_outer(const mmc_ctx* ctx, Run& run, const std::vector<cd>& tin, const std::vector<cd>& tout,
                        void* P0, void* P1, void* A0, void* A1, AccMode mode, int nrhs) {
  const int mi = int(tin.size()), mo = int(tout.size());
  const int npad = run.g.npad;
  const double kap = ctx->kappa;
  const int accf = acc_flags(mode, run);
  void* P[2] = {P0, P1};
  void* A[2] = {A0, A1};
  if (mo == 1) {
    Step st;
    st.in = A[0];
    st.flags = accf;
    st.coef = coef_block(npad);
    for (int r = 0; r < nrhs; ++r) set_coef(st.coef, npad, r, 0, 0, 0, 1.0 / tout[0], 0);
    run.steps.push_back(st);
    return;
  }
  for (int k = 0; k < mo - 1; ++k) {
    const cd io = 1.0 / tout[k];
    for (int j = 0; j < mi; ++j) {
      Step st;
      st.coef = coef_block(npad);
      const cd ii = 1.0 / tin[j];
      const bool first = (j == 0), last = (j == mi - 1);
      st.in = first ? A[k & 1] : P[(j - 1) & 1];
      st.out = last ? A[(k + 1) & 1] : P[j & 1];
      st.flags = mmc::SF_HOP | mmc::SF_WRITE;
      cd a = 1.0 - ii, b = kap * ii, gg = 0, wi = 0, wo = 0;
      if (first) {
        st.flags |= accf;
        wi = io;
      }
      if (last) {
        // prod_{k+1} = (1/theta_out) (pi_in step of q) + (1 - 1/theta_out) prod_k
        a *= io;
        b *= io;
        gg = 1.0 - io;
        st.aux = A[k & 1];
        st.flags |= mmc::SF_AUX;
        if (k == mo - 2) {
          st.flags |= accf | mmc::SF_BIL_OUT;
          wo = 1.0 / tout[mo - 1];
        }
      }
      for (int r = 0; r < nrhs; ++r) set_coef(st.coef, npad, r, a, b, gg, wi, wo);
      run.steps.push_back(st);
    }
  }
}

inline bool valid_poly(const mmc_ctx* ctx, int h) { return h >= 0 && h < int(ctx->polys.size()); }

inline int poly_degree(const mmc_ctx* ctx, int h) {
  const Poly& P = ctx->polys[h];
  if (P.kind == 1) {
    int mi = int(ctx->polys[P.h_in].theta.size()), mo = int(ctx->polys[P.h_out].theta.size());
    return mi * mo - 1;
  }
  int m = int(P.theta.size());
  if (P.op == MMC_OP_M) return m - 1;
  int mb = int(ctx->polys[P.op].theta.size());
  return (m - 1) * mb;  // degree in M of p_out(phi_h), phi_h of degree mb
}

inline cd poly_value(const mmc_ctx* ctx, int h, cd a) {
  const Poly& P = ctx->polys[h];
  if (P.kind == 1) {
    cd pin = mmc::poly_scalar(ctx->polys[P.h_in].theta, a);
    return pin * mmc::poly_scalar(ctx->polys[P.h_out].theta, a * pin);
  }
  if (P.op == MMC_OP_M) return mmc::poly_scalar(P.theta, a);
  cd phi = a * mmc::poly_scalar(ctx->polys[P.op].theta, a);
  return mmc::poly_scalar(P.theta, phi);
}

// Apply polynomial h to the field x (nrhs vectors, precision prec) with accumulation
// into y (ACC_Y; y zeroed here, type double2 for F64 / float2 otherwise) or into
// run.partial (ACC_BIL; with run.codes / run.left set by the caller).
inline int apply_poly_impl(mmc_ctx* ctx, int h, const void* x, int nrhs, int prec, AccMode mode, void* y,
                    Run& base, cudaStream_t s) {
  const Poly& P = ctx->polys[h];
  geom g = base.g;
  const size_t fb = field_bytes(g, prec);
  void *P0, *P1;
  TRY(scratch(ctx, "P0", fb, &P0));
  TRY(scratch(ctx, "P1", fb, &P1));
  const size_t yb = size_t(g.npad) * g.V * 12 * (prec == MMC_F64 ? 16 : 8);
  if (mode == ACC_Y) CK(cudaMemsetAsync(y, 0, yb, s));
  if (P.kind == 0 && P.op == MMC_OP_M) {
    Run run = base;
    run.y = y;
    build_single(ctx, run, P.theta, x, P0, P1, mode, 1.0, nrhs);
    return exec_run(ctx, run, s);
  }
  if (P.kind == 0) RET(MMC_ERR_ARG, "polynomial in phi_h is not applicable alone; compose it with mmc_poly_double");
  const std::vector<cd>& tin = ctx->polys[P.h_in].theta;
  const std::vector<cd>& tout = ctx->polys[P.h_out].theta;
  // stage A: w = p_in(M) x as a vector (accumulator), then to storage precision in A0
  void *A0, *A1, *W;
  TRY(scratch(ctx, "A0", fb, &A0));
  TRY(scratch(ctx, "A1", fb, &A1));
  TRY(scratch(ctx, "W", yb, &W));
  CK(cudaMemsetAsync(W, 0, yb, s));
  {
    Run run = base;
    run.y = W;
    run.codes = nullptr;
    run.left = nullptr;
    build_single(ctx, run, tin, x, P0, P1, ACC_Y, 1.0, nrhs);
    TRY(exec_run(ctx, run, s));
  }
  if (prec == MMC_BF16 && ctx->rounding == 1 && ctx->salt)
    CK(mmc::launch_convert_sr(A0, W, g, ctx->salt, s));
  else
    CK(mmc::launch_convert(prec, A0, prec == MMC_F64 ? MMC_F64 : MMC_F32, W, g, s));
  Run run = base;
  run.y = y;
  build_double_outer(ctx, run, tin, tout, P0, P1, A0, A1, mode, nrhs);
  return exec_run(ctx, run, s);
}

// y = M x (or M^+ x) on a field: a = 1, b = -kappa.
inline int apply_M_impl(mmc_ctx* ctx, const void* x, void* y, int nrhs, int prec, bool dagger, cudaStream_t s) {
  Run run;
  run.g = make_geom(ctx, nrhs);
  run.prec = prec;
  run.dagger = dagger;
  Step st;
  st.in = x;
  st.out = y;
  st.flags = mmc::SF_HOP | mmc::SF_WRITE;
  st.coef = coef_block(run.g.npad);
  for (int r = 0; r < run.g.npad; ++r) set_coef(st.coef, run.g.npad, r, 1.0, -ctx->kappa, 0, 0, 0);
  run.steps.push_back(st);
  return exec_run(ctx, run, s);
}

// ----------------------------------------------------------- Arnoldi (CGS2)
// op(in, out): out = operator applied to in (single-vector or batched FP64 fields)
// Basis V: (m+1) FP64 fields of geometry g (contiguous), start vector in V[0]
// (unnormalised on entry).  Fills Hcol (host, per rhs (m+1) x m column-major).
struct ArnoldiOut {
  std::vector<CMat> H;  // per rhs
  std::vector<double> beta;
};

// passes: 2 (classical Gram-Schmidt twice, the default) or 1 (once; FP32 bases only).
template <class Op>
inline int arnoldi_cgs2(mmc_ctx* ctx, const geom& g, int prec, void* V, int m, Op op, ArnoldiOut& out, cudaStream_t s,
                        int passes = 2) {
  const size_t stride = size_t(g.npad) * g.V * 12;  // elements per basis field
  const size_t eb = elem_bytes(prec);
  const int spc = 256;
  const int nbx = (g.V + spc - 1) / spc;
  void *part, *h1, *h2, *hcols, *nrm, *W;
  TRY(scratch(ctx, "arn_part", size_t(nbx) * (m + 1) * g.npad * sizeof(double2), &part));
  TRY(scratch(ctx, "arn_h1", size_t(m + 1) * g.npad * sizeof(double2), &h1));
  TRY(scratch(ctx, "arn_h2", size_t(m + 1) * g.npad * sizeof(double2), &h2));
  TRY(scratch(ctx, "arn_hcols", size_t(m) * (m + 1) * g.npad * sizeof(double2), &hcols));
  TRY(scratch(ctx, "arn_nrm", size_t(m + 1) * g.npad * sizeof(double2), &nrm));
  TRY(scratch(ctx, "arn_w", stride * eb, &W));
  CK(cudaMemsetAsync(hcols, 0, size_t(m) * (m + 1) * g.npad * sizeof(double2), s));
  char* Vb = reinterpret_cast<char*>(V);
  double2* nrm2 = reinterpret_cast<double2*>(nrm);
  // normalise the start vector: nrm[0] = ||v0||^2
  CK(mmc::launch_multidot(prec, g, V, stride, 1, V, 0, spc, (double2*)part, s));
  CK(mmc::launch_reduce((double2*)part, nbx, 1, g.npad, nrm2, 0, s));
  CK(mmc::launch_normalise(prec, g, V, nrm2, V, s));
  for (int j = 0; j < m; ++j) {
    void* vj = Vb + size_t(j) * stride * eb;
    TRY(op(vj, W));
    double2* hc = reinterpret_cast<double2*>(hcols) + size_t(j) * (m + 1) * g.npad;
    CK(mmc::launch_multidot(prec, g, V, stride, j + 1, W, 0, spc, (double2*)part, s));
    CK(mmc::launch_reduce((double2*)part, nbx, j + 1, g.npad, (double2*)h1, 0, s));
    if (prec == MMC_F32 && j + 1 <= 8 && passes == 1) {
      // one pass: the update fused with the norm; the Hessenberg column is h1
      CK(mmc::launch_update_dot(g, (const float2*)V, stride, j + 1, (double2*)h1, (float2*)W, true, spc,
                                (double2*)part, s));
      CK(cudaMemcpyAsync(hc, h1, size_t(j + 1) * g.npad * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    } else if (prec == MMC_F32 && j + 1 <= 8) {
      // FP32 basis: each update fused with the dot products that follow it (the second
      // pass's projections, then the norm), one read of the basis and of w each
      CK(mmc::launch_update_dot(g, (const float2*)V, stride, j + 1, (double2*)h1, (float2*)W, false, spc,
                                (double2*)part, s));
      CK(mmc::launch_reduce((double2*)part, nbx, j + 1, g.npad, (double2*)h2, 0, s));
      CK(mmc::launch_update_dot(g, (const float2*)V, stride, j + 1, (double2*)h2, (float2*)W, true, spc,
                                (double2*)part, s));
      CK(mmc::launch_add2((double2*)h1, (double2*)h2, hc, (j + 1) * g.npad, s));
    } else {
      CK(mmc::launch_basis_update(prec, g, V, stride, j + 1, (double2*)h1, W, s));
      CK(mmc::launch_multidot(prec, g, V, stride, j + 1, W, 0, spc, (double2*)part, s));
      CK(mmc::launch_reduce((double2*)part, nbx, j + 1, g.npad, (double2*)h2, 0, s));
      CK(mmc::launch_basis_update(prec, g, V, stride, j + 1, (double2*)h2, W, s));
      CK(mmc::launch_add2((double2*)h1, (double2*)h2, hc, (j + 1) * g.npad, s));
      CK(mmc::launch_multidot(prec, g, W, stride, 1, W, 0, spc, (double2*)part, s));
    }
    CK(mmc::launch_reduce((double2*)part, nbx, 1, g.npad, nrm2 + size_t(j + 1) * g.npad, 0, s));
    CK(mmc::launch_normalise(prec, g, W, nrm2 + size_t(j + 1) * g.npad, Vb + size_t(j + 1) * stride * eb, s));
  }
  std::vector<double2> hh(size_t(m) * (m + 1) * g.npad), nn(size_t(m + 1) * g.npad);
  CK(cudaMemcpyAsync(hh.data(), hcols, hh.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(nn.data(), nrm, nn.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  out.H.assign(g.npad, CMat(m + 1, m));
  out.beta.assign(g.npad, 0.0);
  for (int r = 0; r < g.npad; ++r) {
    out.beta[r] = std::sqrt(nn[r].x);
    for (int j = 0; j < m; ++j) {
      for (int i = 0; i <= j; ++i) {
        double2 v = hh[(size_t(j) * (m + 1) + i) * g.npad + r];
        out.H[r](i, j) = cd(v.x, v.y);
      }
      out.H[r](j + 1, j) = std::sqrt(nn[size_t(j + 1) * g.npad + r].x);
    }
  }
  return MMC_OK;
}

// Operator for a single-vector FP64 Arnoldi: M, or phi_h(M) = M p_h(M).
inline int apply_op_f64(mmc_ctx* ctx, int op_handle, const void* in, void* out, int nrhs, cudaStream_t s) {
  if (op_handle == MMC_OP_M) return apply_M_impl(ctx, in, out, nrhs, MMC_F64, false, s);
  void* T;
  geom g = make_geom(ctx, nrhs);
  TRY(scratch(ctx, "phi_tmp", field_bytes(g, MMC_F64), &T));
  Run base;
  base.g = g;
  base.prec = MMC_F64;
  TRY(apply_poly_impl(ctx, op_handle, in, nrhs, MMC_F64, ACC_Y, T, base, s));
  return apply_M_impl(ctx, T, out, nrhs, MMC_F64, false, s);
}

// learned network (learned.cu)
bool is_net(const mmc_ctx* ctx, int h);
int net_apply(mmc_ctx* ctx, int h, const void* x, void* y, int nrhs, cudaStream_t s, void** acts);

inline int check_ctx(mmc_ctx* ctx) {
  if (!ctx) return MMC_ERR_ARG;
  if (ctx->failed) RET(MMC_ERR_STATE, "context retired after a failed kernel (destroy it)");
  if (!ctx->gauge) RET(MMC_ERR_STATE, "no gauge field loaded");
  CK(cudaSetDevice(ctx->device));
  return MMC_OK;
}

}  // namespace host
}  // namespace mmc
