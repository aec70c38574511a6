// Fused Wilson step kernel, second form: right-hand-side block R, rhs per lane
// RPT and the epilogue mode are template parameters, so every operand offset is
// an immediate, each mode compiles to a small kernel (instruction cache), and
// neighbour sites come from a precomputed table instead of integer division.
// Same arithmetic and operand conventions as step_kernel (stencil.cu).
#pragma once
#include "kernels.h"
#include "stencil_ops.cuh"

namespace mmc {
namespace sten2 {
using namespace sten;

enum Acc { ACC_NONE = 0, ACC_CODES = 1, ACC_Y = 2, ACC_LEFT = 3 };

// MINB resident CTAs of 128 threads per SM cap the registers: RPT = 2 uses 3 (168
// registers), RPT = 1 uses 4 (128) or 6 (80, more warps to hide memory latency).
template <typename S, int R, int RPT, int MINB, int KD, bool AUX, int ACC>
__global__ void __launch_bounds__(128, MINB) step2_kernel(step_params p) {
  using T = float;
  constexpr int L = R / RPT;      // lanes per site
  constexpr int SPP = 128 / L;    // sites per pass of the CTA
  constexpr bool BIL = (ACC == ACC_CODES || ACC == ACC_LEFT);
  const int rb = blockIdx.y;
  if (p.rb_len && p.step >= p.rb_len[rb]) return;
  const int lane = threadIdx.x % L;
  const int r0 = lane * RPT;
  const int rglob = rb * R + r0;
  const size_t rb_off = size_t(rb) * p.V * 12 * R;
  const S* in = reinterpret_cast<const S*>(p.in) + rb_off + r0;
  const bool bil_out = (p.flags & SF_BIL_OUT) != 0;
  const uint32_t srkey = sr_key(p);

  cx<T> ca[RPT], cb[RPT], cg[RPT], cwi[RPT], cwo[RPT];
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
  }
  double bre[RPT], bim[RPT];
#pragma unroll
  for (int j = 0; j < RPT; ++j) bre[j] = bim[j] = 0.0;

  const int site_begin = blockIdx.x * p.spc;
  const int site_end = min(p.V, site_begin + p.spc);
  for (int s0 = site_begin; s0 < site_end; s0 += SPP) {
    const int pos = s0 + threadIdx.x / L;
    if (pos >= site_end) continue;
    const int site = p.order ? __ldg(p.order + pos) : pos;
    const int4 nf = __ldg(reinterpret_cast<const int4*>(p.nbr) + 2 * size_t(site));
    const int4 nb = __ldg(reinterpret_cast<const int4*>(p.nbr) + 2 * size_t(site) + 1);
    cx<T> acc[12][RPT];
#pragma unroll
    for (int c = 0; c < 12; ++c)
#pragma unroll
      for (int j = 0; j < RPT; ++j) acc[c][j] = cmake(T(0), T(0));
    Link<T> Lk;
    load_link(p.links, site, 0, Lk);
    hop_dir<S, RPT, 0, false, KD>(in + size_t(nf.x) * 12 * R, R, Lk, acc);
    load_link(p.links, nb.x, 0, Lk);
    hop_dir<S, RPT, 0, true, -KD>(in + size_t(nb.x) * 12 * R, R, Lk, acc);
    load_link(p.links, site, 1, Lk);
    hop_dir<S, RPT, 1, false, KD>(in + size_t(nf.y) * 12 * R, R, Lk, acc);
    load_link(p.links, nb.y, 1, Lk);
    hop_dir<S, RPT, 1, true, -KD>(in + size_t(nb.y) * 12 * R, R, Lk, acc);
    load_link(p.links, site, 2, Lk);
    hop_dir<S, RPT, 2, false, KD>(in + size_t(nf.z) * 12 * R, R, Lk, acc);
    load_link(p.links, nb.z, 2, Lk);
    hop_dir<S, RPT, 2, true, -KD>(in + size_t(nb.z) * 12 * R, R, Lk, acc);
    load_link(p.links, site, 3, Lk);
    hop_dir<S, RPT, 3, false, KD>(in + size_t(nf.w) * 12 * R, R, Lk, acc);
    load_link(p.links, nb.w, 3, Lk);
    hop_dir<S, RPT, 3, true, -KD>(in + size_t(nb.w) * 12 * R, R, Lk, acc);

    const size_t off = size_t(site) * 12 * R;  // within the rhs block, lane offset included in `in`
    const size_t boff = rb_off + off + r0;
    uint32_t code[RPT];
    if (ACC == ACC_CODES) {
#pragma unroll
      for (int j = 0; j < RPT; ++j) code[j] = __ldg(p.codes + (size_t(rb) * p.V + site) * R + r0 + j);
    }
    cx<T> si[RPT], so[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) si[j] = so[j] = cmake(T(0), T(0));
    // the aux operand's and the accumulator's 12 components, all loaded before the first
    // store of the pass (the compiler keeps loads that may alias the stores behind them,
    // one memory latency per component)
    cx<T> axv[AUX ? 12 : 1][RPT];
    if (AUX) {
#pragma unroll
      for (int c = 0; c < 12; ++c) load_rpt<S, RPT>(reinterpret_cast<const S*>(p.aux) + boff + c * R, axv[c]);
    }
    cx<T> yv[ACC == ACC_Y ? 12 : 1][RPT];
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
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      cx<T> vin[RPT], vout[RPT];
      load_rpt<S, RPT>(in + off + c * R, vin);
#pragma unroll
      for (int j = 0; j < RPT; ++j) vout[j] = cfma(cb[j], acc[c][j], cmul(ca[j], vin[j]));
      if (AUX) {
#pragma unroll
        for (int j = 0; j < RPT; ++j) vout[j] = cfma(cg[j], axv[AUX ? c : 0][j], vout[j]);
      }
      if (std::is_same<S, __nv_bfloat162>::value && p.salt)
        store_rpt_sr<S, RPT>(reinterpret_cast<S*>(p.out) + boff + c * R, vout, srkey, uint32_t(boff + c * R));
      else
        store_rpt<S, RPT>(reinterpret_cast<S*>(p.out) + boff + c * R, vout);
      if (ACC == ACC_Y) {
        float2* yp = reinterpret_cast<float2*>(p.y) + boff + c * R;
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
          cx<T> a = yv[ACC == ACC_Y ? c : 0][j];
          a = cfma(cwi[j], vin[j], a);
          if (bil_out) a = cfma(cwo[j], vout[j], a);
          yp[j] = make_float2(a.re, a.im);
        }
      }
      if (BIL) {
        const int cp = (p.theta == 1) ? (c + 6) % 12 : c;
        const T sg = (p.theta == 2 && c >= 6) ? T(-1) : T(1);
        if (ACC == ACC_CODES) {
          // conj(i^k) v is v turned by -k quarter turns: k odd swaps (re, im) -> (im, -re),
          // k >= 2 negates; the gamma_5 sign folds into the same factor
#pragma unroll
          for (int j = 0; j < RPT; ++j) {
            const uint32_t k = (code[j] >> (2 * cp)) & 3u;
            const T f = (k & 2u) ? -sg : sg;
            const bool odd = (k & 1u) != 0;
            si[j].re = fmaf(f, odd ? vin[j].im : vin[j].re, si[j].re);
            si[j].im = fmaf(f, odd ? -vin[j].re : vin[j].im, si[j].im);
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
            si[j] = cfmac(eta[j], cscale(vin[j], sg), si[j]);
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
  if (BIL) {
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
#pragma unroll
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
  }
}

// Dispatch of one (S, R, RPT) family over the epilogue modes; returns false when
// the flags need the generic kernel.
template <typename S, int R, int RPT, int MINB>
bool launch2(const step_params& p, int n_rb, cudaStream_t s, cudaError_t* err) {
  const int f = p.flags;
  if (!(f & SF_HOP) || !(f & SF_WRITE)) return false;
  const bool aux = (f & SF_AUX) != 0;
  int acc = ACC_NONE;
  if (f & SF_BIL_CODES) acc = ACC_CODES;
  else if (f & SF_YACC) acc = ACC_Y;
  else if (f & SF_BIL_LEFT) acc = ACC_LEFT;
  dim3 grid((p.V + p.spc - 1) / p.spc, n_rb);
  if (f & SF_DAGGER) {
    if (aux || acc != ACC_NONE) return false;
    step2_kernel<S, R, RPT, MINB, -1, false, ACC_NONE><<<grid, 128, 0, s>>>(p);
  } else if (!aux) {
    switch (acc) {
      case ACC_NONE: step2_kernel<S, R, RPT, MINB, 1, false, ACC_NONE><<<grid, 128, 0, s>>>(p); break;
      case ACC_CODES: step2_kernel<S, R, RPT, MINB, 1, false, ACC_CODES><<<grid, 128, 0, s>>>(p); break;
      case ACC_Y: step2_kernel<S, R, RPT, MINB, 1, false, ACC_Y><<<grid, 128, 0, s>>>(p); break;
      default: step2_kernel<S, R, RPT, MINB, 1, false, ACC_LEFT><<<grid, 128, 0, s>>>(p); break;
    }
  } else {
    switch (acc) {
      case ACC_NONE: step2_kernel<S, R, RPT, MINB, 1, true, ACC_NONE><<<grid, 128, 0, s>>>(p); break;
      case ACC_CODES: step2_kernel<S, R, RPT, MINB, 1, true, ACC_CODES><<<grid, 128, 0, s>>>(p); break;
      case ACC_Y: step2_kernel<S, R, RPT, MINB, 1, true, ACC_Y><<<grid, 128, 0, s>>>(p); break;
      default: step2_kernel<S, R, RPT, MINB, 1, true, ACC_LEFT><<<grid, 128, 0, s>>>(p); break;
    }
  }
  count_launch();
  *err = cudaGetLastError();
  return true;
}

}  // namespace sten2
}  // namespace mmc
