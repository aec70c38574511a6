// Fused Wilson step kernel, fifth form (same arithmetic and operand conventions as
// step_kernel and step2_kernel).  It keeps the fourth form's persistent grid and
// compact front of work items (a pass of SPP sites of one rhs block) and stages every
// global operand of the eight hops in shared memory with asynchronous copies
// (cp.async, one 8-byte FP32 or 4-byte BF16 complex word per lane and component, the
// links by five lanes of a site in 16-byte pieces), D stages deep:
//
//   stage s of the CTA's stream = (its k-th item, step d), k = s / 9, d = s % 9;
//   d = 0..7: the neighbour spinor and link of hop d, d = 8: the site's own spinor.
//
// While stage s computes, the copies of stage s + D - 1 are in flight (also across
// item boundaries), each in its own commit group; cp.async.wait_group D-1 then
// guarantees stage s.  The data in flight occupy shared memory, not registers, so the
// kernel keeps 16 warps per SM with up to D-1 hops of loads outstanding per thread.
// A thread waits only for its own copies (they always complete), and a site's 16 (or
// 8) lanes, which share its link, sit in one warp and meet at __syncwarp before the
// link is read and before its slot is refilled.  No wait depends on another CTA.
#pragma once
#include <algorithm>

#include "kernels.h"
#include "stencil_ops.cuh"

namespace mmc {
namespace sten5 {
using namespace sten;

enum Acc { ACC_NONE = 0, ACC_CODES = 1, ACC_Y = 2, ACC_LEFT = 3 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t dst, const void* src) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// upper half-spinor h = P psi of the projector (1 - sg gamma_MU) in the chiral basis
template <int MU, int SG>
__device__ __forceinline__ void project(const cx<float> (&s)[12], cx<float> (&h0)[3], cx<float> (&h1)[3]) {
  const float sg = SG;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const cx<float> s0 = s[b], s1 = s[3 + b], s2 = s[6 + b], s3 = s[9 + b];
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
}

// acc += (1 - sg gamma_MU) W h, W = U (DAGU false) or U^+ (DAGU true)
template <int MU, bool DAGU, int SG>
__device__ __forceinline__ void multiply_add(const Link<float>& L, const cx<float> (&h0)[3], const cx<float> (&h1)[3],
                                             cx<float> (&acc)[12]) {
  const float sg = SG;
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
    acc[a] = cadd(acc[a], v0);
    acc[3 + a] = cadd(acc[3 + a], v1);
    acc[6 + a] = cadd(acc[6 + a], r2);
    acc[9 + a] = cadd(acc[9 + a], r3);
  }
}

__device__ __forceinline__ cx<float> lds_cx(const float2* p) {
  const float2 v = *p;
  return cmake(v.x, v.y);
}
__device__ __forceinline__ cx<float> lds_cx(const __nv_bfloat162* p) {
  const float2 v = __bfloat1622float2(*p);
  return cmake(v.x, v.y);
}

// Where this thread's copies of one stage go and come from.
template <typename S, int R, int D>
struct Ring {
  static constexpr int L = R;            // lanes per site (one rhs each)
  static constexpr int SPP = 128 / L;    // sites per item
  S* spin;                               // [D][12][128] elements: thread-private columns
  float4* link;                          // [D][SPP][5] 16-byte pieces of a site's link
  __device__ S* spin_at(int slot, int c) const { return spin + (slot * 12 + c) * 128 + threadIdx.x; }
  __device__ float4* link_at(int slot, int site_local) const { return link + (slot * SPP + site_local) * 5; }
};

// Per-item coordinates of this thread: site, its neighbours, rhs block, validity.
struct ItemPos {
  int item = -1, rb = 0, site = 0;
  int4 nf, nb;
  bool live = false;  // the item exists, its rhs block is still active, and this lane's site is in the lattice
};

template <int SPP, int L>
__device__ __forceinline__ void locate(const step_params& p, int n_chunks, int n_items, int item, ItemPos& ip,
                                       bool want_nbr) {
  ip.item = item;
  ip.live = false;
  if (item >= n_items) return;
  ip.rb = item / n_chunks;
  if (p.rb_len && p.step >= p.rb_len[ip.rb]) return;
  const int pos = (item - ip.rb * n_chunks) * SPP + int(threadIdx.x) / L;
  if (pos >= p.V) return;
  ip.site = p.order ? __ldg(p.order + pos) : pos;
  if (want_nbr) {
    ip.nf = __ldg(reinterpret_cast<const int4*>(p.nbr) + 2 * size_t(ip.site));
    ip.nb = __ldg(reinterpret_cast<const int4*>(p.nbr) + 2 * size_t(ip.site) + 1);
  }
  ip.live = true;
}

// Issue the copies of step d (0..7: hop d's neighbour spinor and link; 8: the own
// spinor) of the item at `ip` into ring slot `slot`, then close the commit group
// (an empty group when the lane has nothing to copy).
template <typename S, int R, int D>
__device__ __forceinline__ void issue(const step_params& p, const Ring<S, R, D>& ring, const ItemPos& ip, int d,
                                      int slot) {
  constexpr int L = R;
  if (ip.live) {
    const int lane = int(threadIdx.x) % L;
    const S* base = reinterpret_cast<const S*>(p.in) + size_t(ip.rb) * p.V * 12 * R + lane;
    int nsite = ip.site, lsite = ip.site, mu = 0;
    if (d < 8) {
      mu = d >> 1;
      const bool bwd = (d & 1) != 0;
      const int f = mu == 0 ? ip.nf.x : mu == 1 ? ip.nf.y : mu == 2 ? ip.nf.z : ip.nf.w;
      const int b = mu == 0 ? ip.nb.x : mu == 1 ? ip.nb.y : mu == 2 ? ip.nb.z : ip.nb.w;
      nsite = bwd ? b : f;
      lsite = bwd ? b : ip.site;
    }
    const S* src = base + size_t(nsite) * 12 * R;
#pragma unroll
    for (int c = 0; c < 12; ++c) cp_async<sizeof(S)>(smem_u32(ring.spin_at(slot, c)), src + c * R);
    if (d < 8 && lane < 5) {
      const float4* lsrc = reinterpret_cast<const float4*>(p.links) + (size_t(lsite) * 4 + mu) * 5 + lane;
      cp_async<16>(smem_u32(ring.link_at(slot, int(threadIdx.x) / L) + lane), lsrc);
    }
  }
  cp_commit();
}

// TH: the insertion Theta of the code bilinear when fixed at compile time (0: the
// identity), -1 when read from p.theta.
template <typename S, int R, int MINB, int KD, bool AUX, int ACC, int TH, int D>
__global__ void __launch_bounds__(128, MINB) step5_kernel(step_params p, int n_chunks, int n_items) {
  using T = float;
  constexpr int L = R;
  constexpr int SPP = 128 / L;
  constexpr bool BIL = (ACC == ACC_CODES || ACC == ACC_LEFT);
  extern __shared__ __align__(16) unsigned char smem[];
  Ring<S, R, D> ring;
  ring.link = reinterpret_cast<float4*>(smem);
  ring.spin = reinterpret_cast<S*>(smem + size_t(D) * SPP * 5 * sizeof(float4));
  const int lane = int(threadIdx.x) % L;
  const bool bil_out = (p.flags & SF_BIL_OUT) != 0;
  const uint32_t srkey = sr_key(p);
  __shared__ double2 red[4][32];
  const int warp = threadIdx.x >> 5;
  const int wl = threadIdx.x & 31;
  const int site_local = int(threadIdx.x) / L;

  cx<T> ca, cb, cg, cwi, cwo;
  double bre = 0.0, bim = 0.0;
  int cur_rb = -1;

  auto flush = [&](int rb) {  // block-uniform: this CTA's bilinear sums of rhs block rb
#pragma unroll
    for (int off = L; off < 32; off <<= 1) {
      bre += __shfl_xor_sync(0xffffffffu, bre, off);
      bim += __shfl_xor_sync(0xffffffffu, bim, off);
    }
    if (wl < L) red[warp][wl] = make_double2(bre, bim);
    __syncthreads();
    if (threadIdx.x < R) {
      double sr = 0, sim = 0;
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        sr += red[w][threadIdx.x].x;
        sim += red[w][threadIdx.x].y;
      }
      double2* dst = p.partial + size_t(blockIdx.x) * p.npad + rb * R + threadIdx.x;
      double2 cur = *dst;
      cur.x += sr;
      cur.y += sim;
      *dst = cur;
    }
    __syncthreads();
  };

  // prologue: stages 0 .. D-2 (all in the first item, D <= 9)
  ItemPos is;  // the item the copies are issued for
  locate<SPP, L>(p, n_chunks, n_items, int(blockIdx.x), is, true);
#pragma unroll
  for (int d = 0; d < D - 1; ++d) issue<S, R, D>(p, ring, is, d, d % D);

  for (int k = 0;; ++k) {
    const int item = int(blockIdx.x) + k * int(gridDim.x);
    if (item >= n_items) break;  // uniform over the CTA
    const int rb = item / n_chunks;
    if (rb != cur_rb) {
      if (BIL && cur_rb >= 0) flush(cur_rb);
      cur_rb = rb;
      const int r = rb * R + lane;
      double2 v;
      v = p.coef[0 * p.npad + r];
      ca = cmake(T(v.x), T(v.y));
      v = p.coef[1 * p.npad + r];
      cb = cmake(T(v.x), T(v.y));
      if (AUX) {
        v = p.coef[2 * p.npad + r];
        cg = cmake(T(v.x), T(v.y));
      }
      if (ACC != ACC_NONE) {
        v = p.coef[3 * p.npad + r];
        cwi = cmake(T(v.x), T(v.y));
        v = p.coef[4 * p.npad + r];
        cwo = cmake(T(v.x), T(v.y));
      }
      bre = bim = 0.0;
    }
    ItemPos ic;  // the item computed now (no neighbour table needed: the copies carry it)
    locate<SPP, L>(p, n_chunks, n_items, item, ic, false);
    uint32_t code = 0;
    if (ACC == ACC_CODES && ic.live) code = __ldg(p.codes + (size_t(rb) * p.V + ic.site) * R + lane);
    cx<T> acc[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = cmake(T(0), T(0));
    cx<T> vin[12];

#pragma unroll
    for (int d = 0; d < 9; ++d) {
      // refill the slot of stage s - 1 with stage s + D - 1 once every lane of the
      // site is done with it
      __syncwarp();
      const int dn = d + D - 1;  // step of the stage to issue, in this item (< 9) or the next
      if (dn < 9) {
        issue<S, R, D>(p, ring, is, dn, (k * 9 + dn) % D);
      } else {
        if (dn == 9) locate<SPP, L>(p, n_chunks, n_items, item + int(gridDim.x), is, true);
        issue<S, R, D>(p, ring, is, dn - 9, ((k + 1) * 9 + dn - 9) % D);
      }
      cp_wait<D - 1>();
      __syncwarp();
      const int slot = (k * 9 + d) % D;
      if (!ic.live) continue;
      cx<T> sp[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) sp[c] = lds_cx(ring.spin_at(slot, c));
      if (d == 8) {
#pragma unroll
        for (int c = 0; c < 12; ++c) vin[c] = sp[c];
        continue;
      }
      Link<T> lk;
      const float4* lp = ring.link_at(slot, site_local);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 v = lp[q];
        lk.u[2 * q] = cmake(v.x, v.y);
        lk.u[2 * q + 1] = cmake(v.z, v.w);
      }
      {
        const float4 v = lp[4];
        lk.u[8] = cmake(v.x, v.y);
      }
      cx<T> h0[3], h1[3];
      switch (d) {
        case 0: project<0, KD>(sp, h0, h1); multiply_add<0, false, KD>(lk, h0, h1, acc); break;
        case 1: project<0, -KD>(sp, h0, h1); multiply_add<0, true, -KD>(lk, h0, h1, acc); break;
        case 2: project<1, KD>(sp, h0, h1); multiply_add<1, false, KD>(lk, h0, h1, acc); break;
        case 3: project<1, -KD>(sp, h0, h1); multiply_add<1, true, -KD>(lk, h0, h1, acc); break;
        case 4: project<2, KD>(sp, h0, h1); multiply_add<2, false, KD>(lk, h0, h1, acc); break;
        case 5: project<2, -KD>(sp, h0, h1); multiply_add<2, true, -KD>(lk, h0, h1, acc); break;
        case 6: project<3, KD>(sp, h0, h1); multiply_add<3, false, KD>(lk, h0, h1, acc); break;
        default: project<3, -KD>(sp, h0, h1); multiply_add<3, true, -KD>(lk, h0, h1, acc); break;
      }
    }
    if (!ic.live) continue;

    const size_t boff = size_t(rb) * p.V * 12 * R + size_t(ic.site) * 12 * R + lane;
    cx<T> si = cmake(T(0), T(0)), so = cmake(T(0), T(0));
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      cx<T> vout = cfma(cb, acc[c], cmul(ca, vin[c]));
      if (AUX) {
        cx<T> ax[1];
        load_rpt<S, 1>(reinterpret_cast<const S*>(p.aux) + boff + c * R, ax);
        vout = cfma(cg, ax[0], vout);
      }
      {
        cx<T> o[1] = {vout};
        if (std::is_same<S, __nv_bfloat162>::value && p.salt)
          store_rpt_sr<S, 1>(reinterpret_cast<S*>(p.out) + boff + c * R, o, srkey, uint32_t(boff + c * R));
        else
          store_rpt<S, 1>(reinterpret_cast<S*>(p.out) + boff + c * R, o);
      }
      if (ACC == ACC_Y) {
        float2* yp = reinterpret_cast<float2*>(p.y) + boff + c * R;
        const float2 yv = *yp;
        cx<T> a = cmake(yv.x, yv.y);
        a = cfma(cwi, vin[c], a);
        if (bil_out) a = cfma(cwo, vout, a);
        *yp = make_float2(a.re, a.im);
      }
      if (BIL) {
        const int theta = TH >= 0 ? TH : p.theta;
        const int cp = (theta == 1) ? (c + 6) % 12 : c;
        const T sg = (theta == 2 && c >= 6) ? T(-1) : T(1);
        if (ACC == ACC_CODES) {
          // conj(i^k) v: k odd swaps (re, im) -> (im, -re), k >= 2 negates (gamma_5 sign folded in)
          const uint32_t kk = (code >> (2 * cp)) & 3u;
          const T f = (kk & 2u) ? -sg : sg;
          const bool odd = (kk & 1u) != 0;
          si.re = fmaf(f, odd ? vin[c].im : vin[c].re, si.re);
          si.im = fmaf(f, odd ? -vin[c].re : vin[c].im, si.im);
          if (bil_out) {
            so.re = fmaf(f, odd ? vout.im : vout.re, so.re);
            so.im = fmaf(f, odd ? -vout.re : vout.im, so.im);
          }
        } else {
          cx<T> eta[1];
          load_rpt<S, 1>(reinterpret_cast<const S*>(p.left) + boff + size_t(cp) * R, eta);
          si = cfmac(eta[0], cscale(vin[c], sg), si);
          if (bil_out) so = cfmac(eta[0], cscale(vout, sg), so);
        }
      }
    }
    if (BIL) {
      cx<T> contrib = cmul(cwi, si);
      if (bil_out) contrib = cfma(cwo, so, contrib);
      bre += double(contrib.re);
      bim += double(contrib.im);
    }
  }
  if (BIL && cur_rb >= 0) flush(cur_rb);
  cp_wait<0>();  // nothing of this thread's is still being copied when it leaves
}

template <typename S, int R, int D>
constexpr size_t smem_bytes() {
  return size_t(D) * (128 / R) * 5 * sizeof(float4) + size_t(D) * 12 * 128 * sizeof(S);
}

// Dispatch of one (S, R, D) family over the epilogue modes; false when the flags or
// the operands' alignment need another form.  nbx: rows of the bilinear partials.
template <typename S, int R, int MINB, int D>
bool launch5(const step_params& p, int n_rb, int nbx, cudaStream_t s, cudaError_t* err) {
  const int f = p.flags;
  if (!(f & SF_HOP) || !(f & SF_WRITE)) return false;
  // cp.async needs every source word aligned to its size, the link pieces to 16 bytes
  if ((reinterpret_cast<uintptr_t>(p.in) % sizeof(S)) || (reinterpret_cast<uintptr_t>(p.links) & 15)) return false;
  const bool aux = (f & SF_AUX) != 0;
  int acc = ACC_NONE;
  if (f & SF_BIL_CODES) acc = ACC_CODES;
  else if (f & SF_YACC) acc = ACC_Y;
  else if (f & SF_BIL_LEFT) acc = ACC_LEFT;
  if ((f & SF_DAGGER) && (aux || acc != ACC_NONE)) return false;
  void (*kern)(step_params, int, int) = nullptr;
  if (f & SF_DAGGER) {
    kern = step5_kernel<S, R, MINB, -1, false, ACC_NONE, -1, D>;
  } else if (!aux) {
    switch (acc) {
      case ACC_NONE: kern = step5_kernel<S, R, MINB, 1, false, ACC_NONE, -1, D>; break;
      case ACC_CODES:
        kern = p.theta == 0 ? step5_kernel<S, R, MINB, 1, false, ACC_CODES, 0, D>
                            : step5_kernel<S, R, MINB, 1, false, ACC_CODES, -1, D>;
        break;
      case ACC_Y: kern = step5_kernel<S, R, MINB, 1, false, ACC_Y, -1, D>; break;
      default: kern = step5_kernel<S, R, MINB, 1, false, ACC_LEFT, -1, D>; break;
    }
  } else {
    switch (acc) {
      case ACC_NONE: kern = step5_kernel<S, R, MINB, 1, true, ACC_NONE, -1, D>; break;
      case ACC_CODES: kern = step5_kernel<S, R, MINB, 1, true, ACC_CODES, -1, D>; break;
      case ACC_Y: kern = step5_kernel<S, R, MINB, 1, true, ACC_Y, -1, D>; break;
      default: kern = step5_kernel<S, R, MINB, 1, true, ACC_LEFT, -1, D>; break;
    }
  }
  constexpr size_t sm = smem_bytes<S, R, D>();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  constexpr int SPP = 128 / R;
  const int n_chunks = (p.V + SPP - 1) / SPP;
  const int n_items = n_chunks * n_rb;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, sm) != cudaSuccess || per_sm < 1 ||
      nsm < 1) {
    cudaGetLastError();
    return false;
  }
  int grid = std::min(nsm * per_sm, n_items);
  if (acc == ACC_CODES || acc == ACC_LEFT) grid = std::min(grid, nbx);  // one partial row per CTA
  if (grid < 1) return false;
  kern<<<grid, 128, sm, s>>>(p, n_chunks, n_items);
  count_launch();
  *err = cudaGetLastError();
  return true;
}

}  // namespace sten5
}  // namespace mmc
