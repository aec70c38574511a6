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
    uint4 raw = __ldg(reinterpret_cast<const uint4*>(p));
    const S* s = reinterpret_cast<const S*>(&raw);
#pragma unroll
    for (int j = 0; j < RPT; ++j) v[j] = to_cx(s[j]);
  } else if constexpr (sizeof(S) * RPT == 8) {
    uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
    const S* s = reinterpret_cast<const S*>(&raw);
#pragma unroll
    for (int j = 0; j < RPT; ++j) v[j] = to_cx(s[j]);
  } else if constexpr (sizeof(S) * RPT == 4) {
    uint32_t raw = __ldg(reinterpret_cast<const unsigned int*>(p));
    const S* s = reinterpret_cast<const S*>(&raw);
#pragma unroll
    for (int j = 0; j < RPT; ++j) v[j] = to_cx(s[j]);
  } else {
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      uint4 raw = __ldg(reinterpret_cast<const uint4*>(p + j));
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
    double2 v = __ldg(p + k);
    L.u[k] = cmake(v.x, v.y);
  }
}
__device__ __forceinline__ void load_link(const void* links, int site, int mu, Link<float>& L) {
  const float4* p = reinterpret_cast<const float4*>(links) + (size_t(site) * 4 + mu) * 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float4 v = __ldg(p + k);
    L.u[2 * k] = cmake(v.x, v.y);
    L.u[2 * k + 1] = cmake(v.z, v.w);
  }
  float4 v = __ldg(p + 4);
  L.u[8] = cmake(v.x, v.y);
}

// ------------------------------------------------- one hop direction
// Adds sgn * (1 - sg gamma_MU) W h(nbr) to acc, W = U (FWD) or U^+ (backward),
// for RPT right-hand sides.  sg = +1 forward / -1 backward for M; flipped for M^+.
template <typename S, int RPT, int MU>
__device__ __forceinline__ void hop_dir(const S* nb, int R, const Link<typename StoreTraits<S>::R>& L,
                                        bool dagU, typename StoreTraits<S>::R sg,
                                        typename StoreTraits<S>::R bsign,
                                        cx<typename StoreTraits<S>::R> (&acc)[12][RPT]) {
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
        if (dagU) {
          v0 = cfmac(L.u[b * 3 + a], h0[b][j], v0);
          v1 = cfmac(L.u[b * 3 + a], h1[b][j], v1);
        } else {
          v0 = cfma(L.u[a * 3 + b], h0[b][j], v0);
          v1 = cfma(L.u[a * 3 + b], h1[b][j], v1);
        }
      }
      v0 = cscale(v0, bsign);
      v1 = cscale(v1, bsign);
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

template <typename S, int RPT, int MU>
__device__ __forceinline__ void hop_mu(const step_params& p, const S* base, int site, int coord,
                                       int stride, int extent, int sgn_dag,
                                       cx<typename StoreTraits<S>::R> (&acc)[12][RPT]) {
  using T = typename StoreTraits<S>::R;
  Link<T> L;
  // forward neighbour x + mu
  int fwd = (coord == extent - 1) ? site - (extent - 1) * stride : site + stride;
  T bf = (MU == 3 && p.tap && coord == extent - 1) ? T(-1) : T(1);
  load_link(p.links, site, MU, L);
  hop_dir<S, RPT, MU>(base + size_t(fwd) * 12 * p.R, p.R, L, false, T(sgn_dag), bf, acc);
  // backward neighbour x - mu
  int bwd = (coord == 0) ? site + (extent - 1) * stride : site - stride;
  T bb = (MU == 3 && p.tap && coord == 0) ? T(-1) : T(1);
  load_link(p.links, bwd, MU, L);
  hop_dir<S, RPT, MU>(base + size_t(bwd) * 12 * p.R, p.R, L, true, T(-sgn_dag), bb, acc);
}

// conj(eta_c) * (Theta psi)_c summed over the 12 components, eta = i^code.
template <typename T>
__device__ __forceinline__ cx<T> bil_codes(uint32_t code, int theta, const cx<T> (&v)[12]) {
  cx<T> s = cmake(T(0), T(0));
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    int src = c;
    T sgn = T(1);
    if (theta == 1) src = (c + 6) % 12;                   // gamma_4 swaps upper and lower spins
    if (theta == 2 && c >= 6) sgn = T(-1);                // gamma_5 = diag(1,1,-1,-1)
    cx<T> w = v[src];
    uint32_t k = (code >> (2 * c)) & 3u;                  // conj(i^k) * w
    cx<T> t;
    if (k == 0) t = w;
    else if (k == 1) t = cmake(w.im, -w.re);
    else if (k == 2) t = cmake(-w.re, -w.im);
    else t = cmake(-w.im, w.re);
    s.re += sgn * t.re;
    s.im += sgn * t.im;
  }
  return s;
}

template <typename T>
__device__ __forceinline__ cx<T> bil_left(const cx<T> (&l)[12], int theta, const cx<T> (&v)[12]) {
  cx<T> s = cmake(T(0), T(0));
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    int src = (theta == 1) ? (c + 6) % 12 : c;
    T sgn = (theta == 2 && c >= 6) ? T(-1) : T(1);
    s = cfmac(l[c], cscale(v[src], sgn), s);
  }
  return s;
}

template <typename S, int RPT>
__global__ void __launch_bounds__(128) step_kernel(step_params p) {
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
  const T kd = (flags & SF_DAGGER) ? T(-1) : T(1);

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
      hop_mu<S, RPT, 0>(p, base, site, x, sx, p.Lx, int(kd), acc);
      hop_mu<S, RPT, 1>(p, base, site, y, sy, p.Ly, int(kd), acc);
      hop_mu<S, RPT, 2>(p, base, site, z, sz, p.Lz, int(kd), acc);
      hop_mu<S, RPT, 3>(p, base, site, t, st, p.Lt, int(kd), acc);
    }
    const size_t off = (size_t(site) * 12) * p.R + r0;  // within rhs block
    const size_t boff = size_t(rb) * p.V * 12 * p.R + off;
    cx<T> vin[12][RPT];
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      cx<T> tmp[RPT];
      load_rpt<S, RPT>(in + off + size_t(c) * p.R, tmp);
#pragma unroll
      for (int j = 0; j < RPT; ++j) vin[c][j] = tmp[j];
    }
    cx<T> vout[12][RPT];
#pragma unroll
    for (int c = 0; c < 12; ++c)
#pragma unroll
      for (int j = 0; j < RPT; ++j) vout[c][j] = cfma(cb[j], acc[c][j], cmul(ca[j], vin[c][j]));
    if (flags & SF_AUX) {
      const S* aux = reinterpret_cast<const S*>(p.aux) + boff;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        cx<T> tmp[RPT];
        load_rpt<S, RPT>(aux + size_t(c) * p.R, tmp);
#pragma unroll
        for (int j = 0; j < RPT; ++j) vout[c][j] = cfma(cg[j], tmp[j], vout[c][j]);
      }
    }
    if (flags & SF_WRITE) {
      S* out = reinterpret_cast<S*>(p.out) + boff;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        cx<T> tmp[RPT];
#pragma unroll
        for (int j = 0; j < RPT; ++j) tmp[j] = vout[c][j];
        store_rpt<S, RPT>(out + size_t(c) * p.R, tmp);
      }
    }
    if (flags & SF_YACC) {
      Y* yp = reinterpret_cast<Y*>(p.y) + boff;
#pragma unroll
      for (int c = 0; c < 12; ++c)
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
          Y yv = yp[size_t(c) * p.R + j];
          cx<T> a = cmake(T(yv.x), T(yv.y));
          a = cfma(cwi[j], vin[c][j], a);
          if (flags & SF_BIL_OUT) a = cfma(cwo[j], vout[c][j], a);
          yv.x = a.re;
          yv.y = a.im;
          yp[size_t(c) * p.R + j] = yv;
        }
    }
    if (flags & (SF_BIL_CODES | SF_BIL_LEFT)) {
#pragma unroll
      for (int j = 0; j < RPT; ++j) {
        cx<T> vi[12], vo[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          vi[c] = vin[c][j];
          vo[c] = vout[c][j];
        }
        cx<T> si, so = cmake(T(0), T(0));
        if (flags & SF_BIL_CODES) {
          uint32_t code = p.codes[(size_t(rb) * p.V + site) * p.R + r0 + j];
          si = bil_codes(code, p.theta, vi);
          if (flags & SF_BIL_OUT) so = bil_codes(code, p.theta, vo);
        } else {
          const S* lp = reinterpret_cast<const S*>(p.left) + boff;
          cx<T> l[12];
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            cx<T> tmp[RPT];
            load_rpt<S, RPT>(lp + size_t(c) * p.R, tmp);
            l[c] = tmp[j];
          }
          si = bil_left(l, p.theta, vi);
          if (flags & SF_BIL_OUT) so = bil_left(l, p.theta, vo);
        }
        cx<T> contrib = cmul(cwi[j], si);
        if (flags & SF_BIL_OUT) contrib = cfma(cwo[j], so, contrib);
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

template <typename S, int RPT>
static cudaError_t launch_t(const step_params& p, int n_rb, cudaStream_t s) {
  dim3 grid((p.V + p.spc - 1) / p.spc, n_rb);
  step_kernel<S, RPT><<<grid, 128, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_step(int prec, int rpt, const step_params& p, int n_rb, cudaStream_t s) {
  if (prec == 0) return launch_t<double2, 1>(p, n_rb, s);
  if (prec == 1) {
    if (rpt == 2) return launch_t<float2, 2>(p, n_rb, s);
    return launch_t<float2, 1>(p, n_rb, s);
  }
  if (rpt == 4) return launch_t<__nv_bfloat162, 4>(p, n_rb, s);
  if (rpt == 2) return launch_t<__nv_bfloat162, 2>(p, n_rb, s);
  return launch_t<__nv_bfloat162, 1>(p, n_rb, s);
}

}  // namespace mmc
