// Fused Wilson step kernel, third form: lattice rows staged in shared memory by
// bulk asynchronous copies.  Same arithmetic and operand conventions as
// step_kernel (stencil.cu) and step2_kernel (stencil2.cuh).
//
// Work item = one x-row (Lx sites) of one right-hand-side block: in the blocked
// layout [rb][site][c][R] that row is one contiguous run of Lx*12*R words, and so
// are its FP32 links [site][mu][10].  A persistent CTA of Lx*R threads (one site and
// one right-hand side each) walks items blockIdx.x, blockIdx.x + gridDim.x, ...; for
// each item one thread issues cp.async.bulk copies of
//   - the item's own row and its links into one of two "own" buffers (the own row
//     serves the +-x hops, whose neighbours lie in the same row, and the epilogue),
//   - the six rows y+-1, z+-1, t+-1 (with links for the backward ones) into a ring
//     of ns slots, in that order,
// each completing on its slot's mbarrier.  The copies run ns rows (plus the next own
// row) ahead of the arithmetic, so the memory system sees ~ns x 45 KB per SM in
// flight instead of the one neighbour per thread of the register-staged forms.
// A slot is refilled after a CTA barrier that ends its use.  Every mbarrier wait is
// bounded; a CTA whose wait gives up records it in *p.err, waits (bounded) for the
// copies it has in flight and leaves, so the host reads an error instead of a hang.
#pragma once
#include "kernels.h"
#include "stencil_ops.cuh"

namespace mmc {
namespace sten3 {
using namespace sten;

enum Acc { ACC_NONE = 0, ACC_CODES = 1, ACC_Y = 2, ACC_LEFT = 3 };

constexpr long long kWait = 1ll << 22;  // bounded try_wait loop (well over a second)
constexpr int kMaxThreads = 512;

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ bool bar_wait(uint32_t addr, uint32_t parity) {
  for (long long i = 0; i < kWait; ++i) {
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

// sgn-weighted hop of direction MU from a neighbour spinor in shared memory
// (component c at nb[c * R]); same projector algebra as sten::hop_dir with one rhs.
template <typename S, int R, int MU, bool DAGU, int SG>
__device__ __forceinline__ void hop_sm(const S* nb, const Link<float>& L, cx<float> (&acc)[12]) {
  const float sg = SG;
  cx<float> h0[3], h1[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const cx<float> s0 = to_cx(nb[(0 * 3 + b) * R]);
    const cx<float> s1 = to_cx(nb[(1 * 3 + b) * R]);
    const cx<float> s2 = to_cx(nb[(2 * 3 + b) * R]);
    const cx<float> s3 = to_cx(nb[(3 * 3 + b) * R]);
    if (MU == 0) {
      h0[b] = cadd(s0, cscale(ctimes_i(s3), sg));
      h1[b] = cadd(s1, cscale(ctimes_i(s2), sg));
    } else if (MU == 1) {
      h0[b] = cadd(s0, cscale(s3, sg));
      h1[b] = csub(s1, cscale(s2, sg));
    } else if (MU == 2) {
      h0[b] = cadd(s0, cscale(ctimes_i(s2), sg));
      h1[b] = csub(s1, cscale(ctimes_i(s3), sg));
    } else {
      h0[b] = csub(s0, cscale(s2, sg));
      h1[b] = csub(s1, cscale(s3, sg));
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cx<float> v0 = cmake(0.f, 0.f), v1 = cmake(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (DAGU) {
        v0 = cfmac(L.u[b * 3 + a], h0[b], v0);
        v1 = cfmac(L.u[b * 3 + a], h1[b], v1);
      } else {
        v0 = cfma(L.u[a * 3 + b], h0[b], v0);
        v1 = cfma(L.u[a * 3 + b], h1[b], v1);
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
    acc[0 * 3 + a] = cadd(acc[0 * 3 + a], v0);
    acc[1 * 3 + a] = cadd(acc[1 * 3 + a], v1);
    acc[2 * 3 + a] = cadd(acc[2 * 3 + a], r2);
    acc[3 * 3 + a] = cadd(acc[3 * 3 + a], r3);
  }
}

// Per-CTA stream of rows: item sequence (active rhs blocks only) and, per item, six
// ring entries (roles y+, y-, z+, z-, t+, t-).
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

template <typename S, int R, int KD, bool AUX, int ACC>
__global__ void __launch_bounds__(kMaxThreads, 1) step3_kernel(step_params p, int ns) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr bool BIL = (ACC == ACC_CODES || ACC == ACC_LEFT);
  const int Lx = p.Lx;
  const uint32_t rowB = uint32_t(Lx) * 12 * R * sizeof(S);
  const uint32_t linkB = uint32_t(Lx) * 4 * 10 * sizeof(float2);
  const uint32_t slotB = rowB + linkB;
  unsigned char* ownb = smem;                 // 2 slots
  unsigned char* ring = smem + 2 * slotB;     // ns slots
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + size_t(2 + ns) * slotB);  // own[2], ring[ns]
  const uint32_t bar0 = su32(bars);
  const int tid = threadIdx.x;
  const int sx = tid / R, r = tid % R;
  const bool lane_ok = sx < Lx;
  Walk w;
  w.n_rows = p.V / Lx;
  w.n_items = w.n_rows * (p.npad / R);
  const size_t rb_elems = size_t(p.V) * 12 * R;
  const S* in = reinterpret_cast<const S*>(p.in);
  const float2* links = reinterpret_cast<const float2*>(p.links);
  const bool bil_out = (p.flags & SF_BIL_OUT) != 0;

  if (tid == 0) {
    for (int b = 0; b < 2 + ns; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * b));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // producer state (thread 0): next own item to issue, next ring entry (item, role, count)
  int o_item = 0, o_j = 0;        // own copies issued: for local item index o_j
  int q_item = 0, q_role = 0;     // next ring entry to issue
  long long q_issued = 0;
  auto issue_own = [&](int item, int j) {
    const int rb = item / w.n_rows, row = item % w.n_rows;
    unsigned char* dst = ownb + (j & 1) * slotB;
    const uint32_t bar = bar0 + 8 * (j & 1);
    bar_expect(bar, slotB);
    bulk_load(su32(dst), in + size_t(rb) * rb_elems + size_t(row) * Lx * 12 * R, rowB, bar);
    bulk_load(su32(dst + rowB), links + size_t(row) * Lx * 40, linkB, bar);
  };
  auto issue_ring = [&]() {  // entry q_issued for (q_item, q_role)
    const int slot = int(q_issued % ns);
    const int rb = q_item / w.n_rows, row = q_item % w.n_rows;
    const int nr = nbr_row(p, row, q_role);
    unsigned char* dst = ring + size_t(slot) * slotB;
    const uint32_t bar = bar0 + 8 * (2 + slot);
    const bool bwd = (q_role & 1) != 0;
    bar_expect(bar, rowB + (bwd ? linkB : 0u));
    bulk_load(su32(dst), in + size_t(rb) * rb_elems + size_t(nr) * Lx * 12 * R, rowB, bar);
    if (bwd) bulk_load(su32(dst + rowB), links + size_t(nr) * Lx * 40, linkB, bar);
    ++q_issued;
    if (++q_role == 6) {
      q_role = 0;
      q_item = w.next(p, q_item + gridDim.x);
    }
  };

  int item = w.next(p, blockIdx.x);
  if (tid == 0) {
    o_item = item;
    q_item = item;
    if (item < w.n_items) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_own(o_item, 0);
      o_j = 1;
      o_item = w.next(p, o_item + gridDim.x);
      for (int e = 0; e < ns && q_item < w.n_items; ++e) issue_ring();
    }
  }

  cx<float> ca = cmake(0.f, 0.f), cb = ca, cg = ca, cwi = ca, cwo = ca;
  int cur_rb = -1;
  double bre = 0.0, bim = 0.0;
  bool bad = false;
  long long q = 0;  // ring entries consumed
  int j = 0;        // local item index
  __shared__ double2 red[kMaxThreads / 32][16];

  auto flush_bil = [&](int rb) {
    // sum over the threads sharing r, then one read-modify-write per rhs of this CTA's partial row
    double sr = bre, si = bim;
#pragma unroll
    for (int off = R; off < 32; off <<= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, off);
      si += __shfl_xor_sync(0xffffffffu, si, off);
    }
    const int warp = tid >> 5, wl = tid & 31;
    if (wl < R) red[warp][wl] = make_double2(sr, si);
    __syncthreads();
    if (tid < R) {
      double a = 0, b = 0;
      for (int k = 0; k < int(blockDim.x >> 5); ++k) {
        a += red[k][tid].x;
        b += red[k][tid].y;
      }
      double2* dst = p.partial + size_t(blockIdx.x) * p.npad + rb * R + tid;
      double2 cur = *dst;
      cur.x += a;
      cur.y += b;
      *dst = cur;
    }
    __syncthreads();
    bre = bim = 0.0;
  };

  while (item < w.n_items) {
    const int rb = item / w.n_rows, row = item % w.n_rows;
    if (BIL && cur_rb >= 0 && rb != cur_rb) flush_bil(cur_rb);
    if (rb != cur_rb) {
      cur_rb = rb;
      const int rg = rb * R + r;
      double2 v = p.coef[0 * p.npad + rg];
      ca = cmake(float(v.x), float(v.y));
      v = p.coef[1 * p.npad + rg];
      cb = cmake(float(v.x), float(v.y));
      if (AUX) {
        v = p.coef[2 * p.npad + rg];
        cg = cmake(float(v.x), float(v.y));
      }
      if (ACC != ACC_NONE) {
        v = p.coef[3 * p.npad + rg];
        cwi = cmake(float(v.x), float(v.y));
        v = p.coef[4 * p.npad + rg];
        cwo = cmake(float(v.x), float(v.y));
      }
    }
    // next item's own row: its buffer was released by the barrier that ended item j - 1
    if (tid == 0 && o_item < w.n_items) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_own(o_item, o_j);
      ++o_j;
      o_item = w.next(p, o_item + gridDim.x);
    }
    const int site = row * Lx + (lane_ok ? sx : 0);
    const size_t fofs = size_t(rb) * rb_elems + size_t(site) * 12 * R + r;  // component 0 of this (site, rhs)
    // epilogue operands from global memory, requested before the waits
    uint32_t code = 0;
    if (ACC == ACC_CODES && lane_ok) code = __ldg(p.codes + (size_t(rb) * p.V + site) * R + r);
    cx<float> ax[12];
    if (AUX) {
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        cx<float> t[1];
        load_rpt<S, 1>(reinterpret_cast<const S*>(p.aux) + fofs + c * R, t);
        ax[c] = t[0];
      }
    }

    const unsigned char* own = ownb + (j & 1) * slotB;
    const S* orow = reinterpret_cast<const S*>(own);
    const unsigned char* olk = own + rowB;
    bad |= !bar_wait(bar0 + 8 * (j & 1), uint32_t((j >> 1) & 1));

    cx<float> acc[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = cmake(0.f, 0.f);
    const int xs = lane_ok ? sx : 0;
    {
      Link<float> L;
      const int xp = (xs + 1 == Lx) ? 0 : xs + 1, xm = (xs == 0) ? Lx - 1 : xs - 1;
      link_sm(olk, xs, 0, L);
      hop_sm<S, R, 0, false, KD>(orow + size_t(xp) * 12 * R + r, L, acc);
      link_sm(olk, xm, 0, L);
      hop_sm<S, R, 0, true, -KD>(orow + size_t(xm) * 12 * R + r, L, acc);
    }
#pragma unroll 1
    for (int k = 0; k < 6; ++k) {
      const int slot = int(q % ns);
      const unsigned char* sb = ring + size_t(slot) * slotB;
      const S* nrow = reinterpret_cast<const S*>(sb) + size_t(xs) * 12 * R + r;
      bad |= !bar_wait(bar0 + 8 * (2 + slot), uint32_t((q / ns) & 1));
      Link<float> L;
      switch (k) {
        case 0: link_sm(olk, xs, 1, L); hop_sm<S, R, 1, false, KD>(nrow, L, acc); break;
        case 1: link_sm(sb + rowB, xs, 1, L); hop_sm<S, R, 1, true, -KD>(nrow, L, acc); break;
        case 2: link_sm(olk, xs, 2, L); hop_sm<S, R, 2, false, KD>(nrow, L, acc); break;
        case 3: link_sm(sb + rowB, xs, 2, L); hop_sm<S, R, 2, true, -KD>(nrow, L, acc); break;
        case 4: link_sm(olk, xs, 3, L); hop_sm<S, R, 3, false, KD>(nrow, L, acc); break;
        default: link_sm(sb + rowB, xs, 3, L); hop_sm<S, R, 3, true, -KD>(nrow, L, acc); break;
      }
      ++q;
      // every thread is done with this slot: refill it (or leave together after a failed wait)
      if (__syncthreads_or(bad)) goto fail;
      if (tid == 0 && q_item < w.n_items) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue_ring();
      }
    }

    if (lane_ok) {
      // epilogue: out = a in + b D in (+ g aux), accumulations
      cx<float> si = cmake(0.f, 0.f), so = si;
      const S* vin_p = orow + size_t(xs) * 12 * R + r;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        const cx<float> vin = to_cx(vin_p[c * R]);
        cx<float> vout = cfma(cb, acc[c], cmul(ca, vin));
        if (AUX) vout = cfma(cg, ax[c], vout);
        cx<float> o1[1] = {vout};
        store_rpt<S, 1>(reinterpret_cast<S*>(p.out) + fofs + c * R, o1);
        if (ACC == ACC_Y) {
          float2* yp = reinterpret_cast<float2*>(p.y) + fofs + c * R;
          const float2 yv = *yp;
          cx<float> a = cmake(yv.x, yv.y);
          a = cfma(cwi, vin, a);
          if (bil_out) a = cfma(cwo, vout, a);
          *yp = make_float2(a.re, a.im);
        }
        if (BIL) {
          const int cp = (p.theta == 1) ? (c + 6) % 12 : c;
          const float sg = (p.theta == 2 && c >= 6) ? -1.f : 1.f;
          if (ACC == ACC_CODES) {
            const uint32_t kq = (code >> (2 * cp)) & 3u;
            const float f = (kq & 2u) ? -sg : sg;
            const bool odd = (kq & 1u) != 0;
            si.re = fmaf(f, odd ? vin.im : vin.re, si.re);
            si.im = fmaf(f, odd ? -vin.re : vin.im, si.im);
            if (bil_out) {
              so.re = fmaf(f, odd ? vout.im : vout.re, so.re);
              so.im = fmaf(f, odd ? -vout.re : vout.im, so.im);
            }
          } else {
            cx<float> eta[1];
            load_rpt<S, 1>(reinterpret_cast<const S*>(p.left) + fofs + size_t(cp) * R, eta);
            si = cfmac(eta[0], cscale(vin, sg), si);
            if (bil_out) so = cfmac(eta[0], cscale(vout, sg), so);
          }
        }
      }
      if (BIL) {
        cx<float> contrib = cmul(cwi, si);
        if (bil_out) contrib = cfma(cwo, so, contrib);
        bre += double(contrib.re);
        bim += double(contrib.im);
      }
    }
    // the own buffer of this item is reused by item j + 2, issued at the start of item j + 1
    if (__syncthreads_or(bad)) goto fail;
    item = w.next(p, item + gridDim.x);
    ++j;
  }
  if (BIL && cur_rb >= 0) flush_bil(cur_rb);
  return;

fail:
  // a wait gave up: record it, let the copies in flight land (bounded), leave
  if (tid == 0) {
    atomicExch(p.err, 1);
    for (long long e = q; e < q_issued; ++e) bar_wait(bar0 + 8 * (2 + int(e % ns)), uint32_t((e / ns) & 1));
    for (int jj = j; jj < o_j; ++jj) bar_wait(bar0 + 8 * (jj & 1), uint32_t((jj >> 1) & 1));
  }
  __syncthreads();
}

// Shared memory of one CTA for ns ring slots.
inline size_t smem_bytes(int Lx, int R, int elem, int ns) {
  const size_t slot = size_t(Lx) * 12 * R * elem + size_t(Lx) * 4 * 10 * 8;
  return slot * (2 + ns) + 8 * (2 + ns);
}

// Launch for one (S, R) family; false when the geometry or flags need another form.
template <typename S, int R>
bool launch3(const step_params& p, int n_rb, int nbx, int want_ns, cudaStream_t s, cudaError_t* err) {
  const int f = p.flags;
  if (!(f & SF_HOP) || !(f & SF_WRITE) || !p.err) return false;
  const int nt = p.Lx * R;
  if (nt % 32 != 0 || nt > kMaxThreads || p.V % p.Lx != 0) return false;
  // bulk copies need 16-byte aligned rows
  const uintptr_t al = reinterpret_cast<uintptr_t>(p.in) | reinterpret_cast<uintptr_t>(p.links);
  if (al & 15) return false;
  const bool aux = (f & SF_AUX) != 0;
  int acc = ACC_NONE;
  if (f & SF_BIL_CODES) acc = ACC_CODES;
  else if (f & SF_YACC) acc = ACC_Y;
  else if (f & SF_BIL_LEFT) acc = ACC_LEFT;
  if ((f & SF_DAGGER) && (aux || acc != ACC_NONE)) return false;
  const bool bil = acc == ACC_CODES || acc == ACC_LEFT;
  if (bil && nbx <= 0) return false;
  int dev = 0, nsm = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int ns = want_ns > 0 ? want_ns : 6;
  const size_t budget = size_t(maxsm) - 8192;  // static shared memory (reduction buffer) and margin
  while (ns >= 2 && smem_bytes(p.Lx, R, sizeof(S), ns) > budget) --ns;
  if (ns < 2) return false;
  const size_t sm = smem_bytes(p.Lx, R, sizeof(S), ns);
  const int n_items = (p.V / p.Lx) * n_rb;
  void (*kern)(step_params, int) = nullptr;
  if (f & SF_DAGGER) {
    kern = step3_kernel<S, R, -1, false, ACC_NONE>;
  } else if (!aux) {
    switch (acc) {
      case ACC_NONE: kern = step3_kernel<S, R, 1, false, ACC_NONE>; break;
      case ACC_CODES: kern = step3_kernel<S, R, 1, false, ACC_CODES>; break;
      case ACC_Y: kern = step3_kernel<S, R, 1, false, ACC_Y>; break;
      default: kern = step3_kernel<S, R, 1, false, ACC_LEFT>; break;
    }
  } else {
    switch (acc) {
      case ACC_NONE: kern = step3_kernel<S, R, 1, true, ACC_NONE>; break;
      case ACC_CODES: kern = step3_kernel<S, R, 1, true, ACC_CODES>; break;
      case ACC_Y: kern = step3_kernel<S, R, 1, true, ACC_Y>; break;
      default: kern = step3_kernel<S, R, 1, true, ACC_LEFT>; break;
    }
  }
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, sm) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return false;
  }
  int grid = std::min(nsm * per_sm, n_items);
  if (bil) grid = std::min(grid, nbx);
  if (grid < 1) return false;
  kern<<<grid, nt, sm, s>>>(p, ns);
  count_launch();
  *err = cudaGetLastError();
  return true;
}

}  // namespace sten3
}  // namespace mmc
