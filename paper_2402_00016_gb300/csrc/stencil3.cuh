// Fused Wilson step kernel, third form: lattice rows staged in shared memory by
// bulk asynchronous copies.  Same arithmetic and operand conventions as
// step_kernel (stencil.cu) and step2_kernel (stencil2.cuh).
//
// Work item = one x-row (Lx sites) of one right-hand-side block: in the blocked
// layout [rb][site][c][R] that row is one contiguous run of Lx*12*R words, and so
// are its FP32 links [site][mu][10].  A persistent CTA walks items blockIdx.x,
// blockIdx.x + gridDim.x, ...  Its warps are specialised: the compute warps (thread =
// one site of the row and RPT consecutive rhs) do the hops and the epilogue; lane 0
// of the last warp streams rows with cp.async.bulk, each copy completing on an
// mbarrier:
//   - item j's own row and links into own slot j & 1 (they serve the +-x hops, the
//     forward links of every direction and the epilogue; the slot is held until the
//     item ends),
//   - its six neighbour rows y+1, y-1, z+1, z-1, t+1, t-1 (the backward ones with
//     their links) through a ring of ns slots, ring entry e in slot e % ns.
// full barriers complete when a copy lands, empty barriers when every compute warp
// has arrived after its use, so the producer runs up to ns rows (plus the next own
// row) ahead and no CTA-wide barrier exists.  No global loads remain in the hops.
// Every wait is bounded and also gives up when another warp raises the CTA's abort
// flag; the kernel then records the failure in *p.err, the producer waits (bounded)
// for the copies it has in flight, and the CTA leaves, so the host reads an error
// instead of a hang.  Bilinear partials take one row per compute warp
// (blockIdx.x * warps + warp): no cross-warp barrier can leave a warp blocked.
#pragma once
#include "kernels.h"
#include "stencil_ops.cuh"

namespace mmc {
namespace sten3 {
using namespace sten;

enum Acc { ACC_NONE = 0, ACC_CODES = 1, ACC_Y = 2, ACC_LEFT = 3 };

constexpr long long kWait = 1ll << 22;  // bounded try_wait loop (well over a second)

// CTA size bound: 384 compute threads (24 sites x 16 rhs, one rhs each) + the producer
// warp; with two rhs per thread 192 + 32, which leaves the compiler 255 registers.
template <int RPT>
constexpr int max_threads() { return RPT == 2 ? 224 : 416; }

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ bool bar_wait(uint32_t addr, uint32_t parity, long long lim) {
  for (long long i = 0; i < lim; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// bounded wait that also gives up when another warp has raised the CTA's abort flag
__device__ __forceinline__ bool bar_wait_ab(uint32_t addr, uint32_t parity, volatile int* abort_flag,
                                            long long lim) {
  for (long long i = 0; i < lim; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
    if (*abort_flag) return false;
  }
  return false;
}

__device__ __forceinline__ void bar_arrive(uint32_t addr) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

// one bulk copy global -> shared completing `bytes` on the mbarrier (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void bar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void link_sm(const unsigned char* lk, int sx, int mu, Link<float>& L) {
  const float4* q = reinterpret_cast<const float4*>(lk) + (sx * 4 + mu) * 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 v = q[k];
    L.u[2 * k] = cmake(v.x, v.y);
    L.u[2 * k + 1] = cmake(v.z, v.w);
  }
  const float4 v = q[4];
  L.u[8] = cmake(v.x, v.y);
}

// shared-memory loads of RPT consecutive rhs (one 8/16-byte access for FP32, 4/8 for BF16)
template <typename S, int RPT>
__device__ __forceinline__ void lds_rpt(const S* q, cx<float> (&v)[RPT]) {
  if constexpr (sizeof(S) * RPT == 16) {
    const uint4 raw = *reinterpret_cast<const uint4*>(q);
    const S* t = reinterpret_cast<const S*>(&raw);
#pragma unroll
    for (int j = 0; j < RPT; ++j) v[j] = to_cx(t[j]);
  } else if constexpr (sizeof(S) * RPT == 8) {
    const uint2 raw = *reinterpret_cast<const uint2*>(q);
    const S* t = reinterpret_cast<const S*>(&raw);
#pragma unroll
    for (int j = 0; j < RPT; ++j) v[j] = to_cx(t[j]);
  } else {
#pragma unroll
    for (int j = 0; j < RPT; ++j) v[j] = to_cx(q[j]);
  }
}

// sgn-weighted hop of direction MU for RPT rhs from a neighbour spinor in shared
// memory (component c at nb[c * R]); the projector algebra of sten::hop_dir.
template <typename S, int R, int RPT, int MU, bool DAGU, int SG>
__device__ __forceinline__ void hop_smr(const S* nb, const Link<float>& L, cx<float> (&acc)[12][RPT]) {
  const float sg = SG;
  cx<float> h0[3][RPT], h1[3][RPT];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    cx<float> s0[RPT], s1[RPT], s2[RPT], s3[RPT];
    lds_rpt<S, RPT>(nb + (0 * 3 + b) * R, s0);
    lds_rpt<S, RPT>(nb + (1 * 3 + b) * R, s1);
    lds_rpt<S, RPT>(nb + (2 * 3 + b) * R, s2);
    lds_rpt<S, RPT>(nb + (3 * 3 + b) * R, s3);
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      if (MU == 0) {
        h0[b][j] = cadd(s0[j], cscale(ctimes_i(s3[j]), sg));
        h1[b][j] = cadd(s1[j], cscale(ctimes_i(s2[j]), sg));
      } else if (MU == 1) {
        h0[b][j] = cadd(s0[j], cscale(s3[j], sg));
        h1[b][j] = csub(s1[j], cscale(s2[j], sg));
      } else if (MU == 2) {
        h0[b][j] = cadd(s0[j], cscale(ctimes_i(s2[j]), sg));
        h1[b][j] = csub(s1[j], cscale(ctimes_i(s3[j]), sg));
      } else {
        h0[b][j] = csub(s0[j], cscale(s2[j], sg));
        h1[b][j] = csub(s1[j], cscale(s3[j], sg));
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      cx<float> v0 = cmake(0.f, 0.f), v1 = cmake(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (DAGU) {
          v0 = cfmac(L.u[b * 3 + a], h0[b][j], v0);
          v1 = cfmac(L.u[b * 3 + a], h1[b][j], v1);
        } else {
          v0 = cfma(L.u[a * 3 + b], h0[b][j], v0);
          v1 = cfma(L.u[a * 3 + b], h1[b][j], v1);
        }
      }
      cx<float> r2, r3;
      if (MU == 0) {
        r2 = cscale(ctimes_i(v1), -sg);
        r3 = cscale(ctimes_i(v0), -sg);
      } else if (MU == 1) {
        r2 = cscale(v1, -sg);
        r3 = cscale(v0, sg);
      } else if (MU == 2) {
        r2 = cscale(ctimes_i(v0), -sg);
        r3 = cscale(ctimes_i(v1), sg);
      } else {
        r2 = cscale(v0, -sg);
        r3 = cscale(v1, -sg);
      }
      acc[0 * 3 + a][j] = cadd(acc[0 * 3 + a][j], v0);
      acc[1 * 3 + a][j] = cadd(acc[1 * 3 + a][j], v1);
      acc[2 * 3 + a][j] = cadd(acc[2 * 3 + a][j], r2);
      acc[3 * 3 + a][j] = cadd(acc[3 * 3 + a][j], r3);
    }
  }
}

// Per-CTA sequence of items (active rhs blocks only).
struct Walk {
  int n_rows, n_items;
  __device__ __forceinline__ bool active(const step_params& p, int item) const {
    return !(p.rb_len && p.step >= p.rb_len[item / n_rows]);
  }
  __device__ __forceinline__ int next(const step_params& p, int item) const {  // first active item >= item
    while (item < n_items && !active(p, item)) item += gridDim.x;
    return item;
  }
};

// global row index of role k (0..5: y+, y-, z+, z-, t+, t-) of row `row`
__device__ __forceinline__ int nbr_row(const step_params& p, int row, int k) {
  const int y = row % p.Ly, z = (row / p.Ly) % p.Lz, t = row / (p.Ly * p.Lz);
  int yy = y, zz = z, tt = t;
  if (k == 0) yy = (y + 1 == p.Ly) ? 0 : y + 1;
  if (k == 1) yy = (y == 0) ? p.Ly - 1 : y - 1;
  if (k == 2) zz = (z + 1 == p.Lz) ? 0 : z + 1;
  if (k == 3) zz = (z == 0) ? p.Lz - 1 : z - 1;
  if (k == 4) tt = (t + 1 == p.Lt) ? 0 : t + 1;
  if (k == 5) tt = (t == 0) ? p.Lt - 1 : t - 1;
  return yy + p.Ly * (zz + p.Lz * tt);
}

template <typename S, int R, int RPT, int KD, bool AUX, int ACC>
__global__ void __launch_bounds__(max_threads<RPT>(), 1) step3_kernel(step_params p, int ns, int nc) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr bool BIL = (ACC == ACC_CODES || ACC == ACC_LEFT);
  constexpr int LPS = R / RPT;  // lanes per site
  const int Lx = p.Lx;
  const uint32_t rowE = uint32_t(Lx) * 12 * R;
  const uint32_t rowB = rowE * sizeof(S);
  const uint32_t linkB = uint32_t(Lx) * 4 * 10 * sizeof(float2);
  const uint32_t slotB = rowB + linkB;
  unsigned char* ownb = smem;               // own rows (and links): 2 slots
  unsigned char* ringb = smem + 2 * slotB;  // neighbour rows: ns slots
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + size_t(2 + ns) * slotB);
  // own_full[2], own_empty[2], full[ns], empty[ns]
  const uint32_t ofull0 = su32(bars), oempty0 = ofull0 + 16, full0 = ofull0 + 32, empty0 = full0 + 8 * ns;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 4 + 2 * ns);
  const int tid = threadIdx.x;
  const int nwc = nc / 32;
  Walk w;
  w.n_rows = p.V / Lx;
  w.n_items = w.n_rows * (p.npad / R);
  const size_t rb_elems = size_t(p.V) * 12 * R;
  const long long lim = p.wait_iters > 0 ? p.wait_iters : kWait;

  if (tid == 0) {
    for (int b = 0; b < ns; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * b));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(empty0 + 8 * b), "r"(nwc));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ofull0 + 8 * b));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(oempty0 + 8 * b), "r"(nwc));
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (tid >= nc) {  // ------------------------------------------------ producer warp
    if (tid != nc) return;
    const S* in = reinterpret_cast<const S*>(p.in);
    const float2* links = reinterpret_cast<const float2*>(p.links);
    long long e = 0;
    int j = 0;
    bool ok = true;
    // fault injection (tests only): no copy is issued, so the compute warps' waits run out
    const bool copies = p.stall_test == 0;
    for (int item = w.next(p, blockIdx.x); ok && item < w.n_items; item = w.next(p, item + gridDim.x), ++j) {
      const int rb = item / w.n_rows, row = item % w.n_rows;
      const S* rbase = in + size_t(rb) * rb_elems;
      {  // own row and links into own slot j & 1, released by item j - 2
        const int b = j & 1;
        if (j >= 2 && !bar_wait_ab(oempty0 + 8 * b, uint32_t(((j >> 1) - 1) & 1), abort_flag, lim)) {
          ok = false;
          break;
        }
        unsigned char* dst = ownb + size_t(b) * slotB;
        if (*abort_flag) {  // a compute warp gave up: issue no further copy
          ok = false;
          break;
        }
        if (copies) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          bar_expect(ofull0 + 8 * b, slotB);
          bulk_load(su32(dst), rbase + size_t(row) * rowE, rowB, ofull0 + 8 * b);
          bulk_load(su32(dst + rowB), links + size_t(row) * Lx * 40, linkB, ofull0 + 8 * b);
        }
      }
      for (int k = 0; k < 6; ++k) {  // y+1, y-1, z+1, z-1, t+1, t-1 (backward ones with links)
        const int slot = int(e % ns);
        if (e >= ns && !bar_wait_ab(empty0 + 8 * slot, uint32_t(((e / ns) - 1) & 1), abort_flag, lim)) {
          ok = false;
          break;
        }
        const int nr = nbr_row(p, row, k);
        const bool with_links = (k & 1) != 0;
        unsigned char* dst = ringb + size_t(slot) * slotB;
        if (*abort_flag) {
          ok = false;
          break;
        }
        if (copies) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          bar_expect(full0 + 8 * slot, rowB + (with_links ? linkB : 0u));
          bulk_load(su32(dst), rbase + size_t(nr) * rowE, rowB, full0 + 8 * slot);
          if (with_links) bulk_load(su32(dst + rowB), links + size_t(nr) * Lx * 40, linkB, full0 + 8 * slot);
        }
        ++e;
      }
    }
    if (!ok) {
      *abort_flag = 1;
      atomicExch(p.err, 1);
    }
    // the last copies issued into each slot land before this thread (and so the CTA) leaves;
    // if one of these bounded waits gives up, a copy may still be writing into this CTA's
    // shared memory after it exits: the flag value 2 tells the host to retire the context
    if (copies) {
      bool drained = true;
      for (long long d = (e > ns ? e - ns : 0); d < e; ++d)
        drained = bar_wait(full0 + 8 * int(d % ns), uint32_t((d / ns) & 1), lim) && drained;
      for (int d = (j > 2 ? j - 2 : 0); d < j; ++d)
        drained = bar_wait(ofull0 + 8 * (d & 1), uint32_t((d >> 1) & 1), lim) && drained;
      if (!drained) atomicExch(p.err, 2);
    }
    return;
  }

  // ---------------------------------------------------------------- compute warps
  const int sx = tid / LPS, r0 = (tid % LPS) * RPT;
  const bool lane_ok = sx < Lx;
  const int xs = lane_ok ? sx : 0;
  const int warp = tid >> 5, lane = tid & 31;
  const bool bil_out = (p.flags & SF_BIL_OUT) != 0;
  cx<float> ca[RPT], cb[RPT], cg[RPT], cwi[RPT], cwo[RPT];
  int cur_rb = -1;
  double bre[RPT], bim[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) bre[q] = bim[q] = 0.0;
  long long e = 0;
  int jo = 0;  // items done by this CTA (own slot jo & 1)
  bool ok = true;

  auto flush_bil = [&](int rb) {  // this warp's sums per rhs into its own partial row
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      double sr = bre[q], si = bim[q];
#pragma unroll
      for (int off = LPS; off < 32; off <<= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, off);
        si += __shfl_xor_sync(0xffffffffu, si, off);
      }
      if (lane < LPS) {
        double2* dst = p.partial + (size_t(blockIdx.x) * nwc + warp) * p.npad + rb * R + lane * RPT + q;
        double2 c = *dst;
        c.x += sr;
        c.y += si;
        *dst = c;
      }
      bre[q] = bim[q] = 0.0;
    }
  };

  for (int item = w.next(p, blockIdx.x); item < w.n_items; item = w.next(p, item + gridDim.x)) {
    const int rb = item / w.n_rows, row = item % w.n_rows;
    if (BIL && cur_rb >= 0 && rb != cur_rb) flush_bil(cur_rb);
    if (rb != cur_rb) {
      cur_rb = rb;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int rg = rb * R + r0 + q;
        double2 v = p.coef[0 * p.npad + rg];
        ca[q] = cmake(float(v.x), float(v.y));
        v = p.coef[1 * p.npad + rg];
        cb[q] = cmake(float(v.x), float(v.y));
        cg[q] = cwi[q] = cwo[q] = cmake(0.f, 0.f);
        if (AUX) {
          v = p.coef[2 * p.npad + rg];
          cg[q] = cmake(float(v.x), float(v.y));
        }
        if (ACC != ACC_NONE) {
          v = p.coef[3 * p.npad + rg];
          cwi[q] = cmake(float(v.x), float(v.y));
          v = p.coef[4 * p.npad + rg];
          cwo[q] = cmake(float(v.x), float(v.y));
        }
      }
    }
    const int site = row * Lx + xs;
    const int xm = (xs == 0) ? Lx - 1 : xs - 1, xp = (xs + 1 == Lx) ? 0 : xs + 1;
    const size_t fofs = size_t(rb) * rb_elems + size_t(site) * 12 * R + r0;
    // epilogue operands from global memory, requested before the waits
    uint32_t code[RPT];
    if (ACC == ACC_CODES) {
#pragma unroll
      for (int q = 0; q < RPT; ++q) code[q] = lane_ok ? __ldg(p.codes + (size_t(rb) * p.V + site) * R + r0 + q) : 0u;
    }
    cx<float> ax[12][RPT];
    if (AUX) {
#pragma unroll
      for (int c = 0; c < 12; ++c) load_rpt<S, RPT>(reinterpret_cast<const S*>(p.aux) + fofs + c * R, ax[c]);
    }
    cx<float> acc[12][RPT];
#pragma unroll
    for (int c = 0; c < 12; ++c)
#pragma unroll
      for (int q = 0; q < RPT; ++q) acc[c][q] = cmake(0.f, 0.f);

    // own row: +-x hops
    {
      const bool got = bar_wait_ab(ofull0 + 8 * (jo & 1), uint32_t((jo >> 1) & 1), abort_flag, lim);
      if (!(ok = __all_sync(0xffffffffu, got))) break;
    }
    const unsigned char* own = ownb + size_t(jo & 1) * slotB;
    const S* orow = reinterpret_cast<const S*>(own) + r0;
    const unsigned char* olk = own + rowB;
    {
      Link<float> L;
      link_sm(olk, xs, 0, L);
      hop_smr<S, R, RPT, 0, false, KD>(orow + size_t(xp) * 12 * R, L, acc);
      link_sm(olk, xm, 0, L);
      hop_smr<S, R, RPT, 0, true, -KD>(orow + size_t(xm) * 12 * R, L, acc);
    }
#pragma unroll
    for (int k = 1; k < 7; ++k) {
      {
        const bool got = bar_wait_ab(full0 + 8 * int(e % ns), uint32_t((e / ns) & 1), abort_flag, lim);
        if (!(ok = __all_sync(0xffffffffu, got))) break;
      }
      const unsigned char* sb = ringb + size_t(e % ns) * slotB;
      const S* nrow = reinterpret_cast<const S*>(sb) + size_t(xs) * 12 * R + r0;
      Link<float> L;
      const int mu = (k + 1) / 2;
      if (k % 2 == 1) link_sm(olk, xs, mu, L);  // forward: U_mu(x) from the own row
      else link_sm(sb + rowB, xs, mu, L);       // backward: U_mu(x - mu) from that row
      if (k == 1) hop_smr<S, R, RPT, 1, false, KD>(nrow, L, acc);
      if (k == 2) hop_smr<S, R, RPT, 1, true, -KD>(nrow, L, acc);
      if (k == 3) hop_smr<S, R, RPT, 2, false, KD>(nrow, L, acc);
      if (k == 4) hop_smr<S, R, RPT, 2, true, -KD>(nrow, L, acc);
      if (k == 5) hop_smr<S, R, RPT, 3, false, KD>(nrow, L, acc);
      if (k == 6) hop_smr<S, R, RPT, 3, true, -KD>(nrow, L, acc);
      __syncwarp();
      if (lane == 0) bar_arrive(empty0 + 8 * int(e % ns));
      ++e;
    }
    if (!ok) break;

    if (lane_ok) {
      cx<float> si[RPT], so[RPT];
#pragma unroll
      for (int q = 0; q < RPT; ++q) si[q] = so[q] = cmake(0.f, 0.f);
      const S* vin_p = orow + size_t(xs) * 12 * R;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        cx<float> vin[RPT], vout[RPT];
        lds_rpt<S, RPT>(vin_p + c * R, vin);
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          vout[q] = cfma(cb[q], acc[c][q], cmul(ca[q], vin[q]));
          if (AUX) vout[q] = cfma(cg[q], ax[c][q], vout[q]);
        }
        store_rpt<S, RPT>(reinterpret_cast<S*>(p.out) + fofs + c * R, vout);
        if (ACC == ACC_Y) {
          float2* yp = reinterpret_cast<float2*>(p.y) + fofs + c * R;
#pragma unroll
          for (int q = 0; q < RPT; ++q) {
            const float2 yv = yp[q];
            cx<float> a = cmake(yv.x, yv.y);
            a = cfma(cwi[q], vin[q], a);
            if (bil_out) a = cfma(cwo[q], vout[q], a);
            yp[q] = make_float2(a.re, a.im);
          }
        }
        if (BIL) {
          const int cp = (p.theta == 1) ? (c + 6) % 12 : c;
          const float sg = (p.theta == 2 && c >= 6) ? -1.f : 1.f;
          if (ACC == ACC_CODES) {
            // conj(i^k) v: k odd swaps (re, im) -> (im, -re), k >= 2 negates (gamma_5 sign folded in)
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
              const uint32_t kq = (code[q] >> (2 * cp)) & 3u;
              const float f = (kq & 2u) ? -sg : sg;
              const bool odd = (kq & 1u) != 0;
              si[q].re = fmaf(f, odd ? vin[q].im : vin[q].re, si[q].re);
              si[q].im = fmaf(f, odd ? -vin[q].re : vin[q].im, si[q].im);
              if (bil_out) {
                so[q].re = fmaf(f, odd ? vout[q].im : vout[q].re, so[q].re);
                so[q].im = fmaf(f, odd ? -vout[q].re : vout[q].im, so[q].im);
              }
            }
          } else {
            cx<float> eta[RPT];
            load_rpt<S, RPT>(reinterpret_cast<const S*>(p.left) + fofs + size_t(cp) * R, eta);
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
              si[q] = cfmac(eta[q], cscale(vin[q], sg), si[q]);
              if (bil_out) so[q] = cfmac(eta[q], cscale(vout[q], sg), so[q]);
            }
          }
        }
      }
      if (BIL) {
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          cx<float> contrib = cmul(cwi[q], si[q]);
          if (bil_out) contrib = cfma(cwo[q], so[q], contrib);
          bre[q] += double(contrib.re);
          bim[q] += double(contrib.im);
        }
      }
    }
    __syncwarp();
    if (lane == 0) bar_arrive(oempty0 + 8 * (jo & 1));
    ++jo;
  }
  if (!ok) {
    *abort_flag = 1;
    atomicExch(p.err, 1);
    return;
  }
  if (BIL && cur_rb >= 0) flush_bil(cur_rb);
}

// Shared memory of one CTA: two own slots and ns ring slots (row and links each),
// 4 + 2 ns mbarriers and a flag.
inline size_t smem_bytes(int Lx, int R, int elem, int ns) {
  return size_t(2 + ns) * (size_t(Lx) * 12 * R * elem + size_t(Lx) * 4 * 10 * 8) + 8 * size_t(4 + 2 * ns) + 16;
}

// Launch for one (S, R, RPT) family; false when the geometry or flags need another form.
template <typename S, int R, int RPT>
bool launch3(const step_params& p, int n_rb, int nbx, int want_ns, cudaStream_t s, cudaError_t* err) {
  const int f = p.flags;
  if (!(f & SF_HOP) || !(f & SF_WRITE) || !p.err) return false;
  const int nc = ((p.Lx * (R / RPT) + 31) / 32) * 32;
  if (nc + 32 > max_threads<RPT>() || p.V % p.Lx != 0) return false;
  // bulk copies need 16-byte aligned rows
  if ((reinterpret_cast<uintptr_t>(p.in) | reinterpret_cast<uintptr_t>(p.links)) & 15) return false;
  const bool aux = (f & SF_AUX) != 0;
  int acc = ACC_NONE;
  if (f & SF_BIL_CODES) acc = ACC_CODES;
  else if (f & SF_YACC) acc = ACC_Y;
  else if (f & SF_BIL_LEFT) acc = ACC_LEFT;
  if ((f & SF_DAGGER) && (aux || acc != ACC_NONE)) return false;
  const bool bil = acc == ACC_CODES || acc == ACC_LEFT;
  int dev = 0, nsm = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int ns = want_ns > 0 ? want_ns : 6;
  const size_t budget = size_t(maxsm) - 1024;
  while (ns >= 2 && smem_bytes(p.Lx, R, sizeof(S), ns) > budget) --ns;
  if (ns < 2) return false;
  const size_t sm = smem_bytes(p.Lx, R, sizeof(S), ns);
  const int n_items = (p.V / p.Lx) * n_rb;
  void (*kern)(step_params, int, int) = nullptr;
  if (f & SF_DAGGER) {
    kern = step3_kernel<S, R, RPT, -1, false, ACC_NONE>;
  } else if (!aux) {
    switch (acc) {
      case ACC_NONE: kern = step3_kernel<S, R, RPT, 1, false, ACC_NONE>; break;
      case ACC_CODES: kern = step3_kernel<S, R, RPT, 1, false, ACC_CODES>; break;
      case ACC_Y: kern = step3_kernel<S, R, RPT, 1, false, ACC_Y>; break;
      default: kern = step3_kernel<S, R, RPT, 1, false, ACC_LEFT>; break;
    }
  } else {
    switch (acc) {
      case ACC_NONE: kern = step3_kernel<S, R, RPT, 1, true, ACC_NONE>; break;
      case ACC_CODES: kern = step3_kernel<S, R, RPT, 1, true, ACC_CODES>; break;
      case ACC_Y: kern = step3_kernel<S, R, RPT, 1, true, ACC_Y>; break;
      default: kern = step3_kernel<S, R, RPT, 1, true, ACC_LEFT>; break;
    }
  }
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nc + 32, sm) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return false;
  }
  int grid = std::min(nsm * per_sm, n_items);
  if (bil) grid = std::min(grid, nbx / (nc / 32));  // one partial row per compute warp
  if (grid < 1) return false;
  kern<<<grid, nc + 32, sm, s>>>(p, ns, nc);
  count_launch();
  *err = cudaGetLastError();
  return true;
}

}  // namespace sten3
}  // namespace mmc
