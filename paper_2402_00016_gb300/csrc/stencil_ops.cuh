// Device helpers of the fused Wilson step kernels (stencil.cu, stencil2_*.cu):
// storage conversion, complex arithmetic, link loads and one hop of the stencil
// with the chiral-basis spin projection.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace mmc {
namespace sten {

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

// ------------------------------------------------------- stochastic rounding
// 32 random bits for element `idx` of the rounding stream `key`: a 32-bit integer
// hash (multiply-xorshift finaliser) of idx * golden-ratio constant + key.  The key
// mixes a per-chain salt read from device memory with the step index, so the bits
// are fresh for every element, step and chain application and do not depend on the
// data being rounded.
__device__ __forceinline__ uint32_t sr_bits(uint32_t idx, uint32_t key) {
  uint32_t x = idx * 0x9E3779B1u + key;
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}
// FP32 -> BF16 rounding the magnitude up with probability (discarded bits) / 2^16:
// adding a uniform 16-bit r to the bit pattern carries into the kept half exactly
// then, so E[result] = v (for finite v away from the overflow threshold).
__device__ __forceinline__ uint32_t bf16_bits_sr(float v, uint32_t r16) {
  const uint32_t u = __float_as_uint(v);
  if ((u & 0x7f800000u) == 0x7f800000u) {  // Inf, NaN: as round to nearest
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    return uint32_t(*reinterpret_cast<const unsigned short*>(&b));
  }
  return (u + (r16 & 0xffffu)) >> 16;
}

// store_rpt with stochastic rounding of BF16 storage: element idx0 + j takes the random
// bits sr_bits(idx0 + j, key) (FP32 and FP64 storage are stored exactly as store_rpt).
template <typename S, int RPT>
__device__ __forceinline__ void store_rpt_sr(S* p, const cx<typename StoreTraits<S>::R> (&v)[RPT], uint32_t key,
                                             uint32_t idx0) {
  if constexpr (std::is_same<S, __nv_bfloat162>::value) {
    uint32_t w[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      const uint32_t r = sr_bits(idx0 + uint32_t(j), key);
      w[j] = bf16_bits_sr(v[j].re, r) | (bf16_bits_sr(v[j].im, r >> 16) << 16);
    }
    if constexpr (RPT == 4) {
      *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    } else if constexpr (RPT == 2) {
      *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
    } else {
#pragma unroll
      for (int j = 0; j < RPT; ++j) reinterpret_cast<uint32_t*>(p)[j] = w[j];
    }
  } else {
    store_rpt<S, RPT>(p, v);
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

}  // namespace sten
}  // namespace mmc

namespace mmc {
namespace sten {
// Key of the stochastic-rounding stream of one step launch (0 when rounding to nearest).
__device__ __forceinline__ uint32_t sr_key(const step_params& p) {
  return p.salt ? (__ldg(p.salt) ^ (uint32_t(p.step) * 0x85EBCA6Bu)) : 0u;
}
}  // namespace sten
}  // namespace mmc
