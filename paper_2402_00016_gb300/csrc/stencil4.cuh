// Fused Wilson step kernel, fourth form (same arithmetic and operand conventions
// as step_kernel and step2_kernel: out = a in + b D in + g aux with the epilogues
// of step_params).  Two changes against the second form, both aimed at the HBM
// roofline of the stencil:
//
//  * A persistent grid (one wave of resident CTAs) takes work items round-robin.
//    An item is one pass of SPP sites of one rhs block; items run rhs block by
//    rhs block and, within a block, in site traversal order.  The sites in flight
//    on the whole GPU therefore form one compact front of (CTAs x SPP) sites that
//    advances through the lattice, so a spinor read as the t+1 neighbour is still
//    in L2 when it is read again as its own site and as the t-1 neighbour (about
//    two t-slices of one rhs block later) instead of being evicted by the reads of
//    CTAs spread over several slices.
//  * Software pipelining over the eight hops: the neighbour spinor and link of hop
//    d+1 are loaded while hop d does its SU(3) products, and the own site's spinor
//    while the last hop computes; the second form waits for every hop's loads.
//
// Optionally (p.hint & 1) the result is stored with an L2 evict-first policy: it is
// not read again by this launch, so L2 keeps the inputs instead.
//
// Reconstructed links (RC, with 3 resident CTAs per SM, special unitary gauge fields
// only): a hop loads the first two rows of its link (three 16-byte pieces instead of
// five) and rebuilds the third as the complex conjugate of their cross product, negated
// on the time links that carry the antiperiodic phase.  With 8-rhs blocks the launch is
// bound by the L1 data pipe, and the link loads are a third of its requests; with 16-rhs
// blocks a link's loads are shared by twice the rhs.
//
// Paired-component layout (PAIRED, FP32, one rhs per lane, no accumulator or bilinear: the
// Horner chains of the solves): fields [rb][site][c/2][R][c%2], so a lane loads and stores
// components 2q and 2q+1 of its rhs in one 16-byte access; with 8-rhs blocks a site's lanes
// then read a whole 128-byte line per instruction instead of half of one, and the launch is
// no longer bound by the L1 data pipe.
//
// Link staging (SL, with 4 resident CTAs per SM): the eight links of each
// site of an item are copied into shared memory (cp.async, 16-byte pieces, issued by the
// site's own lanes at the start of the item, together with the first hop's spinor
// loads) and every hop reads its link from there right before its products, so no
// registers hold a link in flight and the prefetch of the next hop's spinor fits the
// 128-register budget of 16 warps per SM.
#pragma once
#include <algorithm>

#include "kernels.h"
#include "stencil_ops.cuh"

namespace mmc {
namespace sten4 {
using namespace sten;

enum Acc { ACC_NONE = 0, ACC_CODES = 1, ACC_Y = 2, ACC_LEFT = 3 };

// the 12 spin-colour components of a site for RPT right-hand sides; PAIRED: one rhs per
// lane in the paired-component layout, components 2q and 2q+1 adjacent (one 16-byte load)
template <typename S, int R, int RPT, bool PAIRED = false>
__device__ __forceinline__ void load_spinor(const S* p, cx<typename StoreTraits<S>::R> (&v)[12][RPT]) {
  if constexpr (PAIRED) {
    static_assert(std::is_same<S, float2>::value && RPT == 1, "paired layout: FP32, one rhs per lane");
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      cx<float> pr[2];
      load_rpt<S, 2>(p + q * 2 * R, pr);
      v[2 * q][0] = pr[0];
      v[2 * q + 1][0] = pr[1];
    }
  } else {
#pragma unroll
    for (int c = 0; c < 12; ++c) load_rpt<S, RPT>(p + c * R, v[c]);
  }
}

// upper half-spinor h = P psi of the projector (1 - sg gamma_MU) in the chiral basis
template <typename T, int RPT, int MU, int SG>
__device__ __forceinline__ void project(const cx<T> (&s)[12][RPT], cx<T> (&h0)[3][RPT], cx<T> (&h1)[3][RPT]) {
  const T sg = SG;
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      const cx<T> s0 = s[b][j], s1 = s[3 + b][j], s2 = s[6 + b][j], s3 = s[9 + b][j];
      if (MU == 0) {
        h0[b][j] = cadd(s0, cscale(ctimes_i(s3), sg));
        h1[b][j] = cadd(s1, cscale(ctimes_i(s2), sg));
      } else if (MU == 1) {
        h0[b][j] = cadd(s0, cscale(s3, sg));
        h1[b][j] = csub(s1, cscale(s2, sg));
      } else if (MU == 2) {
        h0[b][j] = cadd(s0, cscale(ctimes_i(s2), sg));
        h1[b][j] = csub(s1, cscale(ctimes_i(s3), sg));
      } else {
        h0[b][j] = csub(s0, cscale(s2, sg));
        h1[b][j] = csub(s1, cscale(s3, sg));
      }
    }
}

// acc += (1 - sg gamma_MU) W h with W = U (DAGU false) or U^+ (DAGU true): the colour
// products of the two upper components and the lower half rebuilt from them
template <typename T, int RPT, int MU, bool DAGU, int SG>
__device__ __forceinline__ void multiply_add(const Link<T>& L, const cx<T> (&h0)[3][RPT], const cx<T> (&h1)[3][RPT],
                                             cx<T> (&acc)[12][RPT]) {
  const T sg = SG;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      cx<T> v0 = cmake(T(0), T(0)), v1 = cmake(T(0), T(0));
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
      cx<T> r2, r3;
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
      acc[a][j] = cadd(acc[a][j], v0);
      acc[3 + a][j] = cadd(acc[3 + a][j], v1);
      acc[6 + a][j] = cadd(acc[6 + a][j], r2);
      acc[9 + a][j] = cadd(acc[9 + a][j], r3);
    }
}

// compiler fences (see fence_acc) on the accumulators and on a pair of half-spinors
template <typename T, int RPT>
__device__ __forceinline__ void fence_arr(cx<T> (&v)[12][RPT]) {
#pragma unroll
  for (int c = 0; c < 12; c += 2)
#pragma unroll
    for (int j = 0; j < RPT; ++j) fence_acc(v[c][j].re, v[c][j].im, v[c + 1][j].re, v[c + 1][j].im);
}
template <typename T, int RPT>
__device__ __forceinline__ void fence_half(cx<T> (&h0)[3][RPT], cx<T> (&h1)[3][RPT]) {
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int j = 0; j < RPT; ++j) fence_acc(h0[b][j].re, h0[b][j].im, h1[b][j].re, h1[b][j].im);
}

// stores, optionally with an L2 evict-first cache policy
template <typename S, int RPT>
__device__ __forceinline__ void store_hint(S* p, const cx<typename StoreTraits<S>::R> (&v)[RPT], bool ef,
                                           uint64_t pol) {
  if (!ef) {
    store_rpt<S, RPT>(p, v);
    return;
  }
  S tmp[RPT];
#pragma unroll
  for (int j = 0; j < RPT; ++j) from_cx(v[j], tmp[j]);
  if constexpr (sizeof(S) * RPT == 16) {
    const uint4 w = *reinterpret_cast<const uint4*>(tmp);
    asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(p), "r"(w.x), "r"(w.y), "r"(w.z),
                 "r"(w.w), "l"(pol)
                 : "memory");
  } else if constexpr (sizeof(S) * RPT == 8) {
    const uint2 w = *reinterpret_cast<const uint2*>(tmp);
    asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1,%2}, %3;" ::"l"(p), "r"(w.x), "r"(w.y), "l"(pol)
                 : "memory");
  } else if constexpr (sizeof(S) * RPT == 4) {
    const uint32_t w = *reinterpret_cast<const uint32_t*>(tmp);
    asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(w), "l"(pol) : "memory");
  } else {
    store_rpt<S, RPT>(p, v);
  }
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit_wait_all() {
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// A link from its five 16-byte pieces in shared memory (the FP32 link layout).
__device__ __forceinline__ void load_link_shared(const float4* p, Link<float>& L) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 v = p[k];
    L.u[2 * k] = cmake(v.x, v.y);
    L.u[2 * k + 1] = cmake(v.z, v.w);
  }
  const float4 v = p[4];
  L.u[8] = cmake(v.x, v.y);
}

// The first two rows of the link (site, mu) (u[0..5]; u[6..8] are rebuilt by complete_link).
__device__ __forceinline__ void load_link_rows(const void* links, int site, int mu, Link<float>& L) {
  const float4* p = reinterpret_cast<const float4*>(links) + (size_t(site) * 4 + mu) * 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uint4 raw = ldv4(p + k);
    float4 v = *reinterpret_cast<const float4*>(&raw);
    L.u[2 * k] = cmake(v.x, v.y);
    L.u[2 * k + 1] = cmake(v.z, v.w);
  }
}

// Third row of a special unitary link from the first two: conj(row0 x row1), times -1
// for a link that carries the antiperiodic phase (all of its rows were negated).
__device__ __forceinline__ void complete_link(Link<float>& L, bool neg) {
  const cx<float>*a = &L.u[0], *b = &L.u[3];
  cx<float> c0 = csub(cmul(a[1], b[2]), cmul(a[2], b[1]));
  cx<float> c1 = csub(cmul(a[2], b[0]), cmul(a[0], b[2]));
  cx<float> c2 = csub(cmul(a[0], b[1]), cmul(a[1], b[0]));
  const float sg = neg ? -1.f : 1.f;
  L.u[6] = cmake(sg * c0.re, -sg * c0.im);
  L.u[7] = cmake(sg * c1.re, -sg * c1.im);
  L.u[8] = cmake(sg * c2.re, -sg * c2.im);
}

// Hop D of the eight (0: x+, 1: x-, 2: y+, ..., 7: t-): project the spinor in `sp`,
// start the loads of hop D+1 (or, after the last hop, of the own site) into `sp`
// and `lk`, then multiply with the link of hop D and accumulate.
// LATE: load the next link after the products (18 registers fewer, its latency not hidden).
// SL: the link of hop D comes from this site's staged links `sl` (8 x 5 pieces).
// RC: `lk` holds the first two rows of hop D's link; the third is rebuilt here.
template <typename S, int R, int RPT, int KD, int D, bool LATE, bool SL, bool RC, bool PAIRED>
__device__ __forceinline__ void hop_pipelined(const step_params& p, const S* in, int site, const int4& nf,
                                              const int4& nb, cx<typename StoreTraits<S>::R> (&sp)[12][RPT],
                                              Link<typename StoreTraits<S>::R>& lk, const float4* sl,
                                              cx<typename StoreTraits<S>::R> (&acc)[12][RPT]) {
  using T = typename StoreTraits<S>::R;
  constexpr int MU = D / 2;
  constexpr bool BWD = (D & 1) != 0;
  constexpr int SG = BWD ? -KD : KD;
  cx<T> h0[3][RPT], h1[3][RPT];
  project<T, RPT, MU, SG>(sp, h0, h1);
  fence_half<T, RPT>(h0, h1);
  constexpr int NMU = (D + 1) / 2;
  constexpr bool NBWD = ((D + 1) & 1) != 0;
  const int nsite = D == 7 ? site
                           : NBWD ? (NMU == 0 ? nb.x : NMU == 1 ? nb.y : NMU == 2 ? nb.z : nb.w)
                                  : (NMU == 0 ? nf.x : NMU == 1 ? nf.y : NMU == 2 ? nf.z : nf.w);
  if constexpr (SL) {
    Link<T> lc;
    load_link_shared(sl + D * 5, lc);
    load_spinor<S, R, RPT, PAIRED>(in + size_t(nsite) * 12 * R, sp);  // after the last hop: the own site
    multiply_add<T, RPT, MU, BWD, SG>(lc, h0, h1, acc);
    fence_arr<T, RPT>(acc);
  } else if constexpr (LATE) {
    load_spinor<S, R, RPT, PAIRED>(in + size_t(nsite) * 12 * R, sp);  // after the last hop: the own site
    multiply_add<T, RPT, MU, BWD, SG>(lk, h0, h1, acc);
    fence_arr<T, RPT>(acc);
    if constexpr (D < 7) load_link(p.links, NBWD ? nsite : site, NMU, lk);
  } else if constexpr (RC) {
    Link<T> lc = lk;
    // the time link at t = Lt - 1 (forward from there, backward from t = 0) carries the phase
    const int lsite = BWD ? (MU == 0 ? nb.x : MU == 1 ? nb.y : MU == 2 ? nb.z : nb.w) : site;
    const bool neg = MU == 3 && p.tap && lsite >= (p.Lt - 1) * p.Lx * p.Ly * p.Lz;
    load_spinor<S, R, RPT, PAIRED>(in + size_t(nsite) * 12 * R, sp);
    if constexpr (D < 7) load_link_rows(p.links, NBWD ? nsite : site, NMU, lk);
    complete_link(lc, neg);
    multiply_add<T, RPT, MU, BWD, SG>(lc, h0, h1, acc);
    fence_arr<T, RPT>(acc);
  } else {
    const Link<T> lc = lk;
    load_spinor<S, R, RPT, PAIRED>(in + size_t(nsite) * 12 * R, sp);
    if constexpr (D < 7) load_link(p.links, NBWD ? nsite : site, NMU, lk);
    multiply_add<T, RPT, MU, BWD, SG>(lc, h0, h1, acc);
    fence_arr<T, RPT>(acc);
  }
}

// TH: the insertion Theta of the code bilinear when fixed at compile time (0: the
// identity), -1 when read from p.theta.
template <typename S, int R, int RPT, int MINB, int KD, bool AUX, int ACC, int TH, bool SL, bool RC,
          bool PAIRED = false>
__global__ void __launch_bounds__(128, MINB) step4_kernel(step_params p, int n_chunks, int n_items) {
  using T = float;
  static_assert(!PAIRED || (std::is_same<S, float2>::value && RPT == 1 && ACC == ACC_NONE),
                "paired layout: FP32 Horner steps (no accumulator, no bilinear)");
  constexpr int L = R / RPT;    // lanes per site
  constexpr int SPP = 128 / L;  // sites per item
  // staged links: [site of the item][hop][piece]; a site's slot is written and read by
  // its own L lanes only (one warp), so a warp-level barrier over them orders it
  __shared__ __align__(16) float4 slink[SL ? SPP : 1][8][5];
  const unsigned site_mask = (L == 32 ? 0xffffffffu : ((1u << L) - 1u)) << ((threadIdx.x & 31) / L * L);
  constexpr bool BIL = (ACC == ACC_CODES || ACC == ACC_LEFT);
  const int lane = threadIdx.x % L;
  const int r0 = lane * RPT;
  const bool bil_out = (p.flags & SF_BIL_OUT) != 0;
  const bool ef = (p.hint & 1) != 0;
  const uint32_t srkey = sr_key(p);
  uint64_t pol = 0;
  if (ef) asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  __shared__ double2 red[4][32];
  const int warp = threadIdx.x >> 5;
  const int wl = threadIdx.x & 31;

  cx<T> ca[RPT], cb[RPT], cg[RPT], cwi[RPT], cwo[RPT];
  double bre[RPT], bim[RPT];
  int cur_rb = -1;

  // bilinear sums of this CTA for rhs block rb into its partial row (block-uniform call)
  auto flush = [&](int rb) {
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
#pragma unroll
      for (int off = L; off < 32; off <<= 1) {
        bre[j] += __shfl_xor_sync(0xffffffffu, bre[j], off);
        bim[j] += __shfl_xor_sync(0xffffffffu, bim[j], off);
      }
    }
    if (wl < L) {
#pragma unroll
      for (int j = 0; j < RPT; ++j) red[warp][wl * RPT + j] = make_double2(bre[j], bim[j]);
    }
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

  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int rb = item / n_chunks;
    if (rb != cur_rb) {  // uniform over the CTA: every thread takes the same items
      if (BIL && cur_rb >= 0) flush(cur_rb);
      cur_rb = rb;
      const int rglob = rb * R + r0;
#pragma unroll
      for (int j = 0; j < RPT; ++j) {
        double2 v;
        v = p.coef[0 * p.npad + rglob + j];
        ca[j] = cmake(T(v.x), T(v.y));
        v = p.coef[1 * p.npad + rglob + j];
        cb[j] = cmake(T(v.x), T(v.y));
        if (AUX) {
          v = p.coef[2 * p.npad + rglob + j];
          cg[j] = cmake(T(v.x), T(v.y));
        }
        if (ACC != ACC_NONE) {
          v = p.coef[3 * p.npad + rglob + j];
          cwi[j] = cmake(T(v.x), T(v.y));
          v = p.coef[4 * p.npad + rglob + j];
          cwo[j] = cmake(T(v.x), T(v.y));
        }
        bre[j] = bim[j] = 0.0;
      }
    }
    if (p.rb_len && p.step >= p.rb_len[rb]) continue;
    const int pos = (item - rb * n_chunks) * SPP + threadIdx.x / L;
    if (pos >= p.V) continue;
    const size_t rb_off = size_t(rb) * p.V * 12 * R;
    const int lane_off = PAIRED ? 2 * r0 : r0;  // a lane's first element in a site's block
    const S* in = reinterpret_cast<const S*>(p.in) + rb_off + lane_off;
    const int site = p.order ? __ldg(p.order + pos) : pos;
    const int4 nf = __ldg(reinterpret_cast<const int4*>(p.nbr) + 2 * size_t(site));
    const int4 nb = __ldg(reinterpret_cast<const int4*>(p.nbr) + 2 * size_t(site) + 1);
    uint32_t code[RPT];
    if (ACC == ACC_CODES) {
#pragma unroll
      for (int j = 0; j < RPT; ++j) code[j] = __ldg(p.codes + (size_t(rb) * p.V + site) * R + r0 + j);
    }
    cx<T> acc[12][RPT];
#pragma unroll
    for (int c = 0; c < 12; ++c)
#pragma unroll
      for (int j = 0; j < RPT; ++j) acc[c][j] = cmake(T(0), T(0));
    cx<T> sp[12][RPT];
    Link<T> lk;
    const float4* sl = &slink[SL ? threadIdx.x / L : 0][0][0];
    if constexpr (SL) {
      // the site's 8 links (forward at this site, backward at the neighbours) as 40
      // pieces over its L lanes; the previous item's reads of the slot end first
      __syncwarp(site_mask);
      const float4* lsrc = reinterpret_cast<const float4*>(p.links);
      for (int q = lane; q < 40; q += L) {
        const int d = q / 5, k = q - 5 * (q / 5), mu = d >> 1;
        const int nbs = mu == 0 ? nb.x : mu == 1 ? nb.y : mu == 2 ? nb.z : nb.w;
        const int src = (d & 1) ? nbs : site;
        cp_async16(smem_addr(sl + q), lsrc + (size_t(src) * 4 + mu) * 5 + k);
      }
    }
    load_spinor<S, R, RPT, PAIRED>(in + size_t(nf.x) * 12 * R, sp);
    if constexpr (SL) {
      cp_commit_wait_all();
      __syncwarp(site_mask);
    } else if constexpr (RC) {
      load_link_rows(p.links, site, 0, lk);
    } else {
      load_link(p.links, site, 0, lk);
    }
    constexpr bool LT = (MINB >= 4) && !SL;
    hop_pipelined<S, R, RPT, KD, 0, LT, SL, RC, PAIRED>(p, in, site, nf, nb, sp, lk, sl, acc);
    hop_pipelined<S, R, RPT, KD, 1, LT, SL, RC, PAIRED>(p, in, site, nf, nb, sp, lk, sl, acc);
    hop_pipelined<S, R, RPT, KD, 2, LT, SL, RC, PAIRED>(p, in, site, nf, nb, sp, lk, sl, acc);
    hop_pipelined<S, R, RPT, KD, 3, LT, SL, RC, PAIRED>(p, in, site, nf, nb, sp, lk, sl, acc);
    hop_pipelined<S, R, RPT, KD, 4, LT, SL, RC, PAIRED>(p, in, site, nf, nb, sp, lk, sl, acc);
    hop_pipelined<S, R, RPT, KD, 5, LT, SL, RC, PAIRED>(p, in, site, nf, nb, sp, lk, sl, acc);
    hop_pipelined<S, R, RPT, KD, 6, LT, SL, RC, PAIRED>(p, in, site, nf, nb, sp, lk, sl, acc);
    hop_pipelined<S, R, RPT, KD, 7, LT, SL, RC, PAIRED>(p, in, site, nf, nb, sp, lk, sl, acc);  // leaves the own spinor in sp

    const size_t boff = rb_off + size_t(site) * 12 * R + lane_off;
    cx<T> si[RPT], so[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) si[j] = so[j] = cmake(T(0), T(0));
    // the aux operand's and the accumulator's 12 components, all loaded before the first
    // store of the pass (the compiler keeps loads that may alias the stores behind them,
    // one memory latency per component)
    cx<T> yv[ACC == ACC_Y ? 12 : 1][RPT];
    cx<T> axv[AUX ? 12 : 1][RPT];
    if constexpr (AUX) load_spinor<S, R, RPT, PAIRED>(reinterpret_cast<const S*>(p.aux) + boff, axv);
    if (ACC == ACC_Y) {
      const float2* yp = reinterpret_cast<const float2*>(p.y) + boff;
#pragma unroll
      for (int c = 0; c < 12; ++c)
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
          const float2 t = yp[c * R + j];
          yv[c][j] = cmake(t.x, t.y);
        }
    }
    cx<T> vprev = cmake(T(0), T(0));
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      cx<T> vout[RPT];
#pragma unroll
      for (int j = 0; j < RPT; ++j) vout[j] = cfma(cb[j], acc[c][j], cmul(ca[j], sp[c][j]));
      if (AUX) {
#pragma unroll
        for (int j = 0; j < RPT; ++j) vout[j] = cfma(cg[j], axv[AUX ? c : 0][j], vout[j]);
      }
      if constexpr (PAIRED) {
        // components 2q and 2q+1 of the lane's rhs are adjacent: one 16-byte store a pair
        if (c & 1) {
          const cx<T> pr[2] = {vprev, vout[0]};
          store_hint<S, 2>(reinterpret_cast<S*>(p.out) + boff + (c >> 1) * 2 * R, pr, ef, pol);
        } else {
          vprev = vout[0];
        }
      } else if (std::is_same<S, __nv_bfloat162>::value && p.salt)
        store_rpt_sr<S, RPT>(reinterpret_cast<S*>(p.out) + boff + c * R, vout, srkey, uint32_t(boff + c * R));
      else
        store_hint<S, RPT>(reinterpret_cast<S*>(p.out) + boff + c * R, vout, ef, pol);
      if (ACC == ACC_Y) {
        float2* yp = reinterpret_cast<float2*>(p.y) + boff + c * R;
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
          cx<T> a = yv[ACC == ACC_Y ? c : 0][j];
          a = cfma(cwi[j], sp[c][j], a);
          if (bil_out) a = cfma(cwo[j], vout[j], a);
          yp[j] = make_float2(a.re, a.im);
        }
      }
      if (BIL) {
        const int theta = TH >= 0 ? TH : p.theta;
        const int cp = (theta == 1) ? (c + 6) % 12 : c;
        const T sg = (theta == 2 && c >= 6) ? T(-1) : T(1);
        if (ACC == ACC_CODES) {
          // conj(i^k) v: k odd swaps (re, im) -> (im, -re), k >= 2 negates (gamma_5 sign folded in)
#pragma unroll
          for (int j = 0; j < RPT; ++j) {
            const uint32_t k = (code[j] >> (2 * cp)) & 3u;
            const T f = (k & 2u) ? -sg : sg;
            const bool odd = (k & 1u) != 0;
            si[j].re = fmaf(f, odd ? sp[c][j].im : sp[c][j].re, si[j].re);
            si[j].im = fmaf(f, odd ? -sp[c][j].re : sp[c][j].im, si[j].im);
            if (bil_out) {
              so[j].re = fmaf(f, odd ? vout[j].im : vout[j].re, so[j].re);
              so[j].im = fmaf(f, odd ? -vout[j].re : vout[j].im, so[j].im);
            }
          }
        } else {
          cx<T> eta[RPT];
          load_rpt<S, RPT>(reinterpret_cast<const S*>(p.left) + boff + size_t(cp) * R, eta);
#pragma unroll
          for (int j = 0; j < RPT; ++j) {
            si[j] = cfmac(eta[j], cscale(sp[c][j], sg), si[j]);
            if (bil_out) so[j] = cfmac(eta[j], cscale(vout[j], sg), so[j]);
          }
        }
      }
    }
    if (BIL) {
#pragma unroll
      for (int j = 0; j < RPT; ++j) {
        cx<T> contrib = cmul(cwi[j], si[j]);
        if (bil_out) contrib = cfma(cwo[j], so[j], contrib);
        bre[j] += double(contrib.re);
        bim[j] += double(contrib.im);
      }
    }
  }
  if (BIL && cur_rb >= 0) flush(cur_rb);
}

template <typename K>
inline int resident_ctas(K kern) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm;
}

// Dispatch of one (S, R) family over the epilogue modes (one rhs per lane); false
// when the flags need another form.  nbx: rows of the bilinear partials (grid bound).
template <typename S, int R, int MINB, bool SL, bool RC, bool PAIRED = false>
bool launch4(const step_params& p, int n_rb, int nbx, cudaStream_t s, cudaError_t* err) {
  constexpr int RPT = 1;
  const int f = p.flags;
  if (!(f & SF_HOP) || !(f & SF_WRITE)) return false;
  const bool aux = (f & SF_AUX) != 0;
  int acc = ACC_NONE;
  if (f & SF_BIL_CODES) acc = ACC_CODES;
  else if (f & SF_YACC) acc = ACC_Y;
  else if (f & SF_BIL_LEFT) acc = ACC_LEFT;
  if ((f & SF_DAGGER) && (aux || acc != ACC_NONE)) return false;
  void (*kern)(step_params, int, int) = nullptr;
  if constexpr (PAIRED) {
    // the paired-component layout: the two steps of a Horner chain only
    if ((f & SF_DAGGER) || acc != ACC_NONE) return false;
    kern = aux ? step4_kernel<S, R, RPT, MINB, 1, true, ACC_NONE, -1, SL, RC, true>
               : step4_kernel<S, R, RPT, MINB, 1, false, ACC_NONE, -1, SL, RC, true>;
  } else if (f & SF_DAGGER) {
    kern = step4_kernel<S, R, RPT, MINB, -1, false, ACC_NONE, -1, SL, RC>;
  } else if (!aux) {
    switch (acc) {
      case ACC_NONE: kern = step4_kernel<S, R, RPT, MINB, 1, false, ACC_NONE, -1, SL, RC>; break;
      case ACC_CODES:
        kern = p.theta == 0 ? step4_kernel<S, R, RPT, MINB, 1, false, ACC_CODES, 0, SL, RC>
                            : step4_kernel<S, R, RPT, MINB, 1, false, ACC_CODES, -1, SL, RC>;
        break;
      case ACC_Y: kern = step4_kernel<S, R, RPT, MINB, 1, false, ACC_Y, -1, SL, RC>; break;
      default: kern = step4_kernel<S, R, RPT, MINB, 1, false, ACC_LEFT, -1, SL, RC>; break;
    }
  } else {
    switch (acc) {
      case ACC_NONE: kern = step4_kernel<S, R, RPT, MINB, 1, true, ACC_NONE, -1, SL, RC>; break;
      case ACC_CODES: kern = step4_kernel<S, R, RPT, MINB, 1, true, ACC_CODES, -1, SL, RC>; break;
      case ACC_Y: kern = step4_kernel<S, R, RPT, MINB, 1, true, ACC_Y, -1, SL, RC>; break;
      default: kern = step4_kernel<S, R, RPT, MINB, 1, true, ACC_LEFT, -1, SL, RC>; break;
    }
  }
  constexpr int SPP = 128 / (R / RPT);
  const int n_chunks = (p.V + SPP - 1) / SPP;
  const int n_items = n_chunks * n_rb;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = resident_ctas(kern);
  if (per_sm < 1 || nsm < 1) return false;
  int grid = std::min(nsm * per_sm, n_items);
  const bool bil = acc == ACC_CODES || acc == ACC_LEFT;
  if (bil) grid = std::min(grid, nbx);  // one partial row per CTA
  if (grid < 1) return false;
  kern<<<grid, 128, 0, s>>>(p, n_chunks, n_items);
  count_launch();
  *err = cudaGetLastError();
  return true;
}

}  // namespace sten4
}  // namespace mmc
