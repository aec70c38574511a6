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

#include "stencil_ops.cuh"

namespace mmc {
namespace {
using namespace sten;

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
  const uint32_t srkey = sr_key(p);

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
      if (flags & SF_WRITE) {
        if (std::is_same<S, __nv_bfloat162>::value && p.salt)
          store_rpt_sr<S, RPT>(reinterpret_cast<S*>(p.out) + boff + size_t(c) * p.R, vout, srkey,
                               uint32_t(boff + size_t(c) * p.R));
        else
          store_rpt<S, RPT>(reinterpret_cast<S*>(p.out) + boff + size_t(c) * p.R, vout);
      }
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
