// The fused multi-right-hand-side Wilson-Dirac step kernel.
//
// One launch computes, for every site x and every right-hand side r of the
// active rhs blocks,
//     out = a * in + b * (D in) + g * aux,
// where D is the Wilson hop (M = 1 - kappa D, Sec. 1 Eq. 1's matrix), plus
// optional epilogues: a bilinear eta^H Theta in (and of out) accumulated per
// CTA in FP64 (the noise bilinears of Eq. 2 and Sec. 6), and a vector
// accumulation y += w_in in + w_out out (the sum over u_k of Sec. 3).  With
// a = 1, b = -kappa it is M; with the coefficients of one Leja step it is one
// degree of the GMRES polynomial recurrence (Sec. 3, Sec. 5).
//
// Layout: fields are [rb][site][c][R] complex with c = 3*spin + colour; a
// lane handles RPT consecutive right-hand sides of one site, 2^logL lanes
// share a site, so a warp reads 32*RPT consecutive complex words per
// component (coalesced) and the links of a site are broadcast to its lanes.
// Dirac matrices: chiral basis, gamma_mu = [[0, A_mu], [A_mu^+, 0]] with
// A_x = -i s1, A_y = -i s2, A_z = -i s3, A_t = 1; the projector (1 - sg gamma)
// has upper half h = psi_u - sg A psi_d and lower half -sg A^+ h.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace mmc {
namespace {

// ------------------------------------------------------------ load / store
// Read-only loads as volatile PTX: they stay in program order with respect to the
// per-hop compiler barriers, which bounds the loads in flight per thread to one
// neighbour (and the register footprint with it).
__device__ __forceinline__ uint4 ldv4(const void* p) {
  uint4 r;
  asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
  return r;
}
__device__ __forceinline__ uint2 ldv2(const void* p) {
  uint2 r;
  asm volatile("ld.global.nc.v2.u32 {%0,%1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
  return r;
}
__device__ __forceinline__ uint32_t ldv1(const void* p) {
  uint32_t r;
  asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(r) : "l"(p));
  return r;
}

template <typename S>
struct StoreTraits;

template <>
struct StoreTraits<double2> {
  using R = double;
};
template <>
struct StoreTraits<float2> {
  using R = float;
};
template <>
struct StoreTraits<__nv_bfloat162> {
  using R = float;
};

__device__ __forceinline__ cx<double> to_cx(double2 v) { return cmake(v.x, v.y); }
__device__ __forceinline__ cx<float> to_cx(float2 v) { return cmake(v.x, v.y); }
__device__ __forceinline__ cx<float> to_cx(__nv_bfloat162 v) {
  float2 f = __bfloat1622float2(v);
  return cmake(f.x, f.y);
}

template <typename S, int RPT>
__device__ __forceinline__ void load_rpt(const S* p, cx<typename StoreTraits<S>::R> (&v)[RPT]) {
  if constexpr (sizeof(S) * RPT == 16) {
    uint4 raw = ldv4(p);
    const S* s = reinterpret_cast<const S*>(&raw);
#pragma unroll
    for (int j = 0; j < RPT; ++j) v[j] = to_cx(s[j]);
  } else if constexpr (sizeof(S) * RPT == 8) {
    uint2 raw = ldv2(p);
    const S* s = reinterpret_cast<const S*>(&raw);
#pragma unroll
    for (int j = 0; j < RPT; ++j) v[j] = to_cx(s[j]);
  } else if constexpr (sizeof(S) * RPT == 4) {
    uint32_t raw = ldv1(p);
    const S* s = reinterpret_cast<const S*>(&raw);
#pragma unroll
    for (int j = 0; j < RPT; ++j) v[j] = to_cx(s[j]);
  } else {
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      uint4 raw = ldv4(p + j);
      v[j] = to_cx(*reinterpret_cast<const S*>(&raw));
    }
  }
}

__device__ __forceinline__ void from_cx(cx<double> c, double2& s) { s = make_double2(c.re, c.im); }
__device__ __forceinline__ void from_cx(cx<float> c, float2& s) { s = make_float2(c.re, c.im); }
__device__ __forceinline__ void from_cx(cx<float> c, __nv_bfloat162& s) {
  s = __float22bfloat162_rn(make_float2(c.re, c.im));
}

template <typename S, int RPT>
__device__ __forceinline__ void store_rpt(S* p, const cx<typename StoreTraits<S>::R> (&v)[RPT]) {
  S tmp[RPT];
#pragma unroll
  for (int j = 0; j < RPT; ++j) from_cx(v[j], tmp[j]);
  if constexpr (sizeof(S) * RPT == 16) {
    *reinterpret_cast<uint4*>(p) = *reinterpret_cast<const uint4*>(tmp);
  } else if constexpr (sizeof(S) * RPT == 8) {
    *reinterpret_cast<uint2*>(p) = *reinterpret_cast<const uint2*>(tmp);
  } else if constexpr (sizeof(S) * RPT == 4) {
    *reinterpret_cast<unsigned int*>(p) = *reinterpret_cast<const unsigned int*>(tmp);
  } else {
#pragma unroll
    for (int j = 0; j < RPT; ++j) p[j] = tmp[j];
  }
}

// ------------------------------------------------------------ complex ops
template <typename T>
__device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return cmake(a.re + b.re, a.im + b.im); }
template <typename T>
__device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return cmake(a.re - b.re, a.im - b.im); }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return cmake(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>  // a * conj(b)
__device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return cmake(a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im);
}
template <typename T>  // acc + a * b
__device__ __forceinline__ cx<T> cfma(cx<T> a, cx<T> b, cx<T> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
template <typename T>  // acc + conj(a) * b
__device__ __forceinline__ cx<T> cfmac(cx<T> a, cx<T> b, cx<T> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
template <typename T>
__device__ __forceinline__ cx<T> ctimes_i(cx<T> a) { return cmake(-a.im, a.re); }
template <typename T>
__device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return cmake(a.re * s, a.im * s); }

// -------------------------------------------------------------- links
template <typename R>
struct Link {
  cx<R> u[9];
};

__device__ __forceinline__ void load_link(const void* links, int site, int mu, Link<double>& L) {
  const double2* p = reinterpret_cast<const double2*>(links) + (size_t(site) * 4 + mu) * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    uint4 raw = ldv4(p + k);
    double2 v = *reinterpret_cast<const double2*>(&raw);
    L.u[k] = cmake(v.x, v.y);
  }
}
__device__ __forceinline__ void load_link(const void* links, int site, int mu, Link<float>& L) {
  const float4* p = reinterpret_cast<const float4*>(links) + (size_t(site) * 4 + mu) * 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint4 raw = ldv4(p + k);
    float4 v = *reinterpret_cast<const float4*>(&raw);
    L.u[2 * k] = cmake(v.x, v.y);
    L.u[2 * k + 1] = cmake(v.z, v.w);
  }
  uint4 raw = ldv4(p + 4);
  float4 v = *reinterpret_cast<const float4*>(&raw);
  L.u[8] = cmake(v.x, v.y);
}

// ------------------------------------------------- one hop direction
// Adds sgn * (1 - sg gamma_MU) W h(nbr) to acc, W = U (FWD) or U^+ (backward),
// for RPT right-hand sides.  sg = +1 forward / -1 backward for M; flipped for M^+.
template <typename S, int RPT, int MU, bool DAGU, int SG>
__device__ __forceinline__ void hop_dir(const S* nb, int R, const Link<typename StoreTraits<S>::R>& L,
                                        cx<typename StoreTraits<S>::R> (&acc)[12][RPT]) {
  const typename StoreTraits<S>::R sg = SG;
  using T = typename StoreTraits<S>::R;
  cx<T> h0[3][RPT], h1[3][RPT];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    cx<T> s0[RPT], s1[RPT], s2[RPT], s3[RPT];
    load_rpt<S, RPT>(nb + (0 * 3 + b) * R, s0);
    load_rpt<S, RPT>(nb + (1 * 3 + b) * R, s1);
    load_rpt<S, RPT>(nb + (2 * 3 + b) * R, s2);
    load_rpt<S, RPT>(nb + (3 * 3 + b) * R, s3);
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      if (MU == 0) {  // A psi_d = (-i s3, -i s2); h = psi_u - sg A psi_d
        h0[b][j] = cadd(s0[j], cscale(ctimes_i(s3[j]), sg));
        h1[b][j] = cadd(s1[j], cscale(ctimes_i(s2[j]), sg));
      } else if (MU == 1) {  // A psi_d = (-s3, s2)
        h0[b][j] = cadd(s0[j], cscale(s3[j], sg));
        h1[b][j] = csub(s1[j], cscale(s2[j], sg));
      } else if (MU == 2) {  // A psi_d = (-i s2, i s3)
        h0[b][j] = cadd(s0[j], cscale(ctimes_i(s2[j]), sg));
        h1[b][j] = csub(s1[j], cscale(ctimes_i(s3[j]), sg));
      } else {  // A = 1
        h0[b][j] = csub(s0[j], cscale(s2[j], sg));
        h1[b][j] = csub(s1[j], cscale(s3[j], sg));
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
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
      // lower half r = -sg A^+ v
      cx<T> r2, r3;
      if (MU == 0) {  // A^+ v = (i v1, i v0)
        r2 = cscale(ctimes_i(v1), -sg);
        r3 = cscale(ctimes_i(v0), -sg);
      } else if (MU == 1) {  // A^+ v = (v1, -v0)
        r2 = cscale(v1, -sg);
        r3 = cscale(v0, sg);
      } else if (MU == 2) {  // A^+ v = (i v0, -i v1)
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

// Compiler fence on the hop accumulators: the empty volatile asm reads and writes
// every accumulator, so the arithmetic of one hop finishes before the (volatile)
// loads of the next hop are issued.  This bounds the live registers to one hop.
__device__ __forceinline__ void fence_acc(float& a, float& b, float& c, float& d) {
  asm volatile("" : "+f"(a), "+f"(b), "+f"(c), "+f"(d));
}
__device__ __forceinline__ void fence_acc(double& a, double& b, double& c, double& d) {
  asm volatile("" : "+d"(a), "+d"(b), "+d"(c), "+d"(d));
}
template <typename T, int RPT>
__device__ __forceinline__ void fence(cx<T> (&acc)[12][RPT]) {
#pragma unroll
  for (int c = 0; c < 12; c += 2)
#pragma unroll
    for (int j = 0; j < RPT; ++j) fence_acc(acc[c][j].re, acc[c][j].im, acc[c + 1][j].re, acc[c + 1][j].im);
}

// Both hops of direction MU.  The antiperiodic time phase is folded into the stored
// links (U_t at t = Lt-1 carries the factor -1), so every hop across the boundary
// gets it from the link itself.  KD = +1 for M, -1 for M^+ (projector signs flipped).
template <typename S, int RPT, int MU, int KD>
__device__ __forceinline__ void hop_mu(const step_params& p, const S* base, int site, int coord, int stride,
                                       int extent, cx<typename StoreTraits<S>::R> (&acc)[12][RPT]) {
  using T = typename StoreTraits<S>::R;
  Link<T> L;
  const int fwd = (coord == extent - 1) ? site - (extent - 1) * stride : site + stride;
  load_link(p.links, site, MU, L);
  hop_dir<S, RPT, MU, false, KD>(base + size_t(fwd) * 12 * p.R, p.R, L, acc);
  // one neighbour's loads in flight per thread: occupancy, not hoisting, hides latency
  fence<T, RPT>(acc);
  const int bwd = (coord == 0) ? site + (extent - 1) * stride : site - stride;
  load_link(p.links, bwd, MU, L);
  hop_dir<S, RPT, MU, true, -KD>(base + size_t(bwd) * 12 * p.R, p.R, L, acc);
  fence<T, RPT>(acc);
}

template <typename S, int RPT, int KD, int MINB>
__global__ void __launch_bounds__(128, MINB) step_kernel(step_params p) {
  using T = typename StoreTraits<S>::R;
  using Y = typename std::conditional<std::is_same<T, double>::value, double2, float2>::type;
  const int rb = blockIdx.y;
  if (p.rb_len && p.step >= p.rb_len[rb]) return;
  const int L = 1 << p.logL;
  const int lane = threadIdx.x & (L - 1);
  const int sites_per_pass = blockDim.x >> p.logL;
  const int r0 = lane * RPT;
  const int rglob = rb * p.R + r0;
  const S* in = reinterpret_cast<const S*>(p.in) + size_t(rb) * p.V * 12 * p.R;
  const int flags = p.flags;

  cx<T> ca[RPT], cb[RPT], cg[RPT], cwi[RPT], cwo[RPT];
#pragma unroll
  for (int j = 0; j < RPT; ++j) {
    double2 v;
    v = p.coef[0 * p.npad + rglob + j]; ca[j] = cmake(T(v.x), T(v.y));
    v = p.coef[1 * p.npad + rglob + j]; cb[j] = cmake(T(v.x), T(v.y));
    v = p.coef[2 * p.npad + rglob + j]; cg[j] = cmake(T(v.x), T(v.y));
    v = p.coef[3 * p.npad + rglob + j]; cwi[j] = cmake(T(v.x), T(v.y));
    v = p.coef[4 * p.npad + rglob + j]; cwo[j] = cmake(T(v.x), T(v.y));
  }
  double bre[RPT], bim[RPT];
#pragma unroll
  for (int j = 0; j < RPT; ++j) bre[j] = bim[j] = 0.0;

  const int site_begin = blockIdx.x * p.spc;
  const int site_end = min(p.V, site_begin + p.spc);
  for (int s0 = site_begin; s0 < site_end; s0 += sites_per_pass) {
    const int site = s0 + (threadIdx.x >> p.logL);
    if (site >= site_end) continue;
    cx<T> acc[12][RPT];
#pragma unroll
    for (int c = 0; c < 12; ++c)
#pragma unroll
      for (int j = 0; j < RPT; ++j) acc[c][j] = cmake(T(0), T(0));
    const S* base = in + r0;
    if (flags & SF_HOP) {
      int x = site % p.Lx;
      int rest = site / p.Lx;
      int y = rest % p.Ly;
      rest /= p.Ly;
      int z = rest % p.Lz;
      int t = rest / p.Lz;
      const int sx = 1, sy = p.Lx, sz = p.Lx * p.Ly, st = p.Lx * p.Ly * p.Lz;
      hop_mu<S, RPT, 0, KD>(p, base, site, x, sx, p.Lx, acc);
      hop_mu<S, RPT, 1, KD>(p, base, site, y, sy, p.Ly, acc);
      hop_mu<S, RPT, 2, KD>(p, base, site, z, sz, p.Lz, acc);
      hop_mu<S, RPT, 3, KD>(p, base, site, t, st, p.Lt, acc);
    }
    const size_t off = (size_t(site) * 12) * p.R + r0;  // within rhs block
    const size_t boff = size_t(rb) * p.V * 12 * p.R + off;
    const bool bil = (flags & (SF_BIL_CODES | SF_BIL_LEFT)) != 0;
    uint32_t code[RPT];
    if (flags & SF_BIL_CODES) {
#pragma unroll
      for (int j = 0; j < RPT; ++j) code[j] = __ldg(p.codes + (size_t(rb) * p.V + site) * p.R + r0 + j);
    }
    // epilogue streamed one spin-colour component at a time: out_c = a in_c + b (D in)_c + g aux_c
    cx<T> si[RPT], so[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) si[j] = so[j] = cmake(T(0), T(0));
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      cx<T> vin[RPT], vout[RPT];
      load_rpt<S, RPT>(in + off + size_t(c) * p.R, vin);
#pragma unroll
      for (int j = 0; j < RPT; ++j) vout[j] = cfma(cb[j], acc[c][j], cmul(ca[j], vin[j]));
      if (flags & SF_AUX) {
        cx<T> ax[RPT];
        load_rpt<S, RPT>(reinterpret_cast<const S*>(p.aux) + boff + size_t(c) * p.R, ax);
#pragma unroll
        for (int j = 0; j < RPT; ++j) vout[j] = cfma(cg[j], ax[j], vout[j]);
      }
      if (flags & SF_WRITE) store_rpt<S, RPT>(reinterpret_cast<S*>(p.out) + boff + size_t(c) * p.R, vout);
      if (flags & SF_YACC) {
        Y* yp = reinterpret_cast<Y*>(p.y) + boff + size_t(c) * p.R;
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
          Y yv = yp[j];
          cx<T> a = cmake(T(yv.x), T(yv.y));
          a = cfma(cwi[j], vin[j], a);
          if (flags & SF_BIL_OUT) a = cfma(cwo[j], vout[j], a);
          yv.x = a.re;
          yv.y = a.im;
          yp[j] = yv;
        }
      }
      if (bil) {
        // conj(eta_c') (Theta v)_c' with c' the component that Theta maps c to:
        // gamma_4 swaps upper and lower spins (c' = c +- 6), gamma_5 flips the lower sign.
        const int cp = (p.theta == 1) ? (c + 6) % 12 : c;
        const T sg = (p.theta == 2 && c >= 6) ? T(-1) : T(1);
        cx<T> eta[RPT];
        if (flags & SF_BIL_CODES) {
#pragma unroll
          for (int j = 0; j < RPT; ++j) {
            const uint32_t k = (code[j] >> (2 * cp)) & 3u;
            eta[j] = cmake(k == 0 ? T(1) : (k == 2 ? T(-1) : T(0)), k == 1 ? T(1) : (k == 3 ? T(-1) : T(0)));
          }
        } else {
          load_rpt<S, RPT>(reinterpret_cast<const S*>(p.left) + boff + size_t(cp) * p.R, eta);
        }
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
          si[j] = cfmac(eta[j], cscale(vin[j], sg), si[j]);
          if (flags & SF_BIL_OUT) so[j] = cfmac(eta[j], cscale(vout[j], sg), so[j]);
        }
      }
    }
    if (bil) {
#pragma unroll
      for (int j = 0; j < RPT; ++j) {
        cx<T> contrib = cmul(cwi[j], si[j]);
        if (flags & SF_BIL_OUT) contrib = cfma(cwo[j], so[j], contrib);
        bre[j] += double(contrib.re);
        bim[j] += double(contrib.im);
      }
    }
  }
  if (flags & (SF_BIL_CODES | SF_BIL_LEFT)) {
    // reduce over the lanes that hold the same right-hand sides (lane bits above logL)
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      for (int off = L; off < 32; off <<= 1) {
        bre[j] += __shfl_xor_sync(0xffffffffu, bre[j], off);
        bim[j] += __shfl_xor_sync(0xffffffffu, bim[j], off);
      }
    }
    __shared__ double2 red[4][32];
    const int warp = threadIdx.x >> 5;
    const int wl = threadIdx.x & 31;
    if (wl < L) {
#pragma unroll
      for (int j = 0; j < RPT; ++j) red[warp][wl * RPT + j] = make_double2(bre[j], bim[j]);
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (threadIdx.x < L * RPT) {
      double sr = 0, si = 0;
      for (int w = 0; w < nw; ++w) {
        sr += red[w][threadIdx.x].x;
        si += red[w][threadIdx.x].y;
      }
      double2* dst = p.partial + size_t(blockIdx.x) * p.npad + rb * p.R + threadIdx.x;
      double2 cur = *dst;
      cur.x += sr;
      cur.y += si;
      *dst = cur;
    }
  }
}

}  // namespace

static long long g_launches = 0;
long long launch_count() { return g_launches; }
void count_launch(int n) { g_launches += n; }

template <typename S, int RPT, int MINB>
static cudaError_t launch_t(const step_params& p, int n_rb, cudaStream_t s) {
  dim3 grid((p.V + p.spc - 1) / p.spc, n_rb);
  if (p.flags & SF_DAGGER)
    step_kernel<S, RPT, -1, MINB><<<grid, 128, 0, s>>>(p);
  else
    step_kernel<S, RPT, 1, MINB><<<grid, 128, 0, s>>>(p);
  count_launch();
  return cudaGetLastError();
}

// variant: rhs per lane (1, 2, 4) and minimum resident CTAs per SM (register cap)
cudaError_t launch_step(int prec, int rpt, int minb, const step_params& p, int n_rb, cudaStream_t s) {
  if (prec == 0) return minb >= 3 ? launch_t<double2, 1, 3>(p, n_rb, s) : launch_t<double2, 1, 1>(p, n_rb, s);
  if (prec == 1) {
    if (rpt == 2) return minb >= 3 ? launch_t<float2, 2, 3>(p, n_rb, s) : launch_t<float2, 2, 1>(p, n_rb, s);
    return minb >= 4 ? launch_t<float2, 1, 4>(p, n_rb, s) : launch_t<float2, 1, 1>(p, n_rb, s);
  }
  if (rpt == 2) return minb >= 3 ? launch_t<__nv_bfloat162, 2, 3>(p, n_rb, s) : launch_t<__nv_bfloat162, 2, 1>(p, n_rb, s);
  return minb >= 4 ? launch_t<__nv_bfloat162, 1, 4>(p, n_rb, s) : launch_t<__nv_bfloat162, 1, 1>(p, n_rb, s);
}

}  // namespace mmc
