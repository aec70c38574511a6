// Kernels of the gauge-covariant linear stencil network (learned subtraction
// operator and preconditioner; the method's paper has no learned part).
//
// A layer maps C_in to C_out channels (each a colour 3-vector) per site:
//   out[x,o] = sum_i W0[o,i] in[x,i] + sum_mu sum_i ( Wf[mu][o,i] U_mu(x) in[x+mu,i]
//                                                  + Wb[mu][o,i] U_mu(x-mu)^+ in[x-mu,i] ).
// Activations use the blocked field layout [rb][site][3*C][R] with complex FP32
// (float2) or BF16 (two bfloat16) storage, weights FP32 or BF16, arithmetic and
// accumulation in FP32; the FP32 links carry the antiperiodic time phase, like M's.
// The adjoint of a layer is the same layer with weights W0^+, Wf[mu] <- Wb[mu]^+,
// Wb[mu] <- Wf[mu]^+, so the backward data pass reuses the forward kernel.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace mmc {
namespace {

constexpr int kMaxC = 8;

__device__ __forceinline__ float2 ld2(const float2* p) { return *p; }
__device__ __forceinline__ float2 ld2(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
__device__ __forceinline__ void st2(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void st2(__nv_bfloat162* p, float2 v) { *p = __float22bfloat162_rn(v); }

__device__ __forceinline__ void load_link32(const float2* links, int site, int mu, float2 (&u)[9]) {
  const float4* p = reinterpret_cast<const float4*>(links) + (size_t(site) * 4 + mu) * 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float4 v = __ldg(p + k);
    u[2 * k] = make_float2(v.x, v.y);
    u[2 * k + 1] = make_float2(v.z, v.w);
  }
  float4 v = __ldg(p + 4);
  u[8] = make_float2(v.x, v.y);
}

// feature w of the layer input at this site: f[i][a] for i < CI
template <int CI, typename SI>
__device__ __forceinline__ void feature(const SI* in, const float2* links, const net_geom& g, int rb, int site,
                                        int r, int w, float2 (&f)[CI][3]) {
  int src = site;
  int mu = 0;
  bool fwd = true;
  if (w > 0) {
    mu = (w - 1) & 3;
    fwd = w <= 4;
    int c[4] = {site % g.L[0], (site / g.L[0]) % g.L[1], (site / (g.L[0] * g.L[1])) % g.L[2],
                site / (g.L[0] * g.L[1] * g.L[2])};
    int stride = 1;
    for (int m = 0; m < mu; ++m) stride *= g.L[m];
    if (fwd)
      src = (c[mu] == g.L[mu] - 1) ? site - (g.L[mu] - 1) * stride : site + stride;
    else
      src = (c[mu] == 0) ? site + (g.L[mu] - 1) * stride : site - stride;
  }
  const SI* base = in + ((size_t(rb) * g.V + src) * (3 * CI)) * g.R + r;
  float2 v[CI][3];
#pragma unroll
  for (int i = 0; i < CI; ++i)
#pragma unroll
    for (int a = 0; a < 3; ++a) v[i][a] = ld2(base + size_t(3 * i + a) * g.R);
  if (w == 0) {
#pragma unroll
    for (int i = 0; i < CI; ++i)
#pragma unroll
      for (int a = 0; a < 3; ++a) f[i][a] = v[i][a];
    return;
  }
  float2 u[9];
  load_link32(links, fwd ? site : src, mu, u);
#pragma unroll
  for (int i = 0; i < CI; ++i)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float re = 0.f, im = 0.f;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        float2 m = fwd ? u[a * 3 + b] : make_float2(u[b * 3 + a].x, -u[b * 3 + a].y);
        re = fmaf(m.x, v[i][b].x, fmaf(-m.y, v[i][b].y, re));
        im = fmaf(m.x, v[i][b].y, fmaf(m.y, v[i][b].x, im));
      }
      f[i][a] = make_float2(re, im);
    }
}

template <int CI, int CO, typename SI, typename SO, typename WT>
__global__ void __launch_bounds__(128) layer_fwd_kernel(net_geom g, const SI* in, const WT* W, SO* out) {
  __shared__ float2 sw[9 * kMaxC * kMaxC];
  for (int k = threadIdx.x; k < 9 * CO * CI; k += blockDim.x) sw[k] = ld2(W + k);
  __syncthreads();
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int site = (blockIdx.x * blockDim.x + threadIdx.x) / g.R;
  if (site >= g.V) return;
  float2 acc[CO][3];
#pragma unroll
  for (int o = 0; o < CO; ++o)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[o][a] = make_float2(0.f, 0.f);
#pragma unroll 1
  for (int w = 0; w < 9; ++w) {
    float2 f[CI][3];
    feature<CI, SI>(in, reinterpret_cast<const float2*>(g.links), g, rb, site, r, w, f);
#pragma unroll
    for (int o = 0; o < CO; ++o)
#pragma unroll
      for (int i = 0; i < CI; ++i) {
        const float2 m = sw[(w * CO + o) * CI + i];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          acc[o][a].x = fmaf(m.x, f[i][a].x, fmaf(-m.y, f[i][a].y, acc[o][a].x));
          acc[o][a].y = fmaf(m.x, f[i][a].y, fmaf(m.y, f[i][a].x, acc[o][a].y));
        }
      }
  }
  SO* ob = out + ((size_t(rb) * g.V + site) * (3 * CO)) * g.R + r;
#pragma unroll
  for (int o = 0; o < CO; ++o)
#pragma unroll
    for (int a = 0; a < 3; ++a) st2(ob + size_t(3 * o + a) * g.R, acc[o][a]);
}

// Weight gradient partials: G[w][o][i] = sum_{x,a,r} delta[x,o,a] conj(f_w[x,i,a]) for
// w = blockIdx.z / (CO/OC), output channels o in the chunk (blockIdx.z % (CO/OC)) * OC ...
template <int CI, int CO, int OC, typename SI>
__global__ void __launch_bounds__(128) layer_wgrad_kernel(net_geom g, const SI* in, const float2* delta, int spc,
                                                          double2* partial) {
  const int nchunk = CO / OC;
  const int w = blockIdx.z / nchunk;
  const int o0 = (blockIdx.z % nchunk) * OC;
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int spp = blockDim.x / g.R;
  const int s_begin = blockIdx.x * spc, s_end = min(g.V, s_begin + spc);
  float2 acc[OC][CI];
#pragma unroll
  for (int o = 0; o < OC; ++o)
#pragma unroll
    for (int i = 0; i < CI; ++i) acc[o][i] = make_float2(0.f, 0.f);
  for (int s0 = s_begin; s0 < s_end; s0 += spp) {
    const int site = s0 + threadIdx.x / g.R;
    if (site >= s_end) continue;
    float2 f[CI][3];
    feature<CI, SI>(in, reinterpret_cast<const float2*>(g.links), g, rb, site, r, w, f);
    const float2* db = delta + ((size_t(rb) * g.V + site) * (3 * CO)) * g.R + r;
#pragma unroll
    for (int o = 0; o < OC; ++o)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float2 d = db[size_t(3 * (o0 + o) + a) * g.R];
#pragma unroll
        for (int i = 0; i < CI; ++i) {  // d * conj(f)
          acc[o][i].x = fmaf(d.x, f[i][a].x, fmaf(d.y, f[i][a].y, acc[o][i].x));
          acc[o][i].y = fmaf(d.y, f[i][a].x, fmaf(-d.x, f[i][a].y, acc[o][i].y));
        }
      }
  }
  // CTA reduction over all threads (every rhs contributes to the same weight)
  __shared__ double2 red[4][OC * CI];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 0; o < OC; ++o)
#pragma unroll
    for (int i = 0; i < CI; ++i) {
      double re = acc[o][i].x, im = acc[o][i].y;
      for (int off = 16; off > 0; off >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, off);
        im += __shfl_xor_sync(0xffffffffu, im, off);
      }
      if (lane == 0) red[warp][o * CI + i] = make_double2(re, im);
    }
  __syncthreads();
  for (int k = threadIdx.x; k < OC * CI; k += blockDim.x) {
    double re = 0, im = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      re += red[q][k].x;
      im += red[q][k].y;
    }
    const int o = k / CI, i = k % CI;
    const size_t bx = size_t(blockIdx.y) * gridDim.x + blockIdx.x;
    partial[bx * (9 * CO * CI) + (size_t(w) * CO + o0 + o) * CI + i] = make_double2(re, im);
  }
}

template <int CI, int CO, typename SI, typename SO, typename WT>
cudaError_t fwd_t(const net_geom& g, const void* in, const void* W, void* out, cudaStream_t s) {
  dim3 grid(unsigned((size_t(g.V) * g.R + 127) / 128), unsigned(g.nrb));
  layer_fwd_kernel<CI, CO, SI, SO, WT><<<grid, 128, 0, s>>>(g, static_cast<const SI*>(in),
                                                            static_cast<const WT*>(W), static_cast<SO*>(out));
  count_launch();
  return cudaGetLastError();
}

template <int CI, int CO, typename SI>
cudaError_t wgrad_t(const net_geom& g, const void* in, const float2* delta, int spc, double2* partial,
                    cudaStream_t s) {
  constexpr int OC = 2;
  dim3 grid(unsigned((g.V + spc - 1) / spc), unsigned(g.nrb), unsigned(9 * (CO / OC)));
  layer_wgrad_kernel<CI, CO, OC, SI><<<grid, 128, 0, s>>>(g, static_cast<const SI*>(in), delta, spc, partial);
  count_launch();
  return cudaGetLastError();
}

template <int CI, int CO>
cudaError_t fwd_any(const net_geom& g, const void* in, bool in_bf16, const void* W, bool w_bf16, void* out,
                    bool out_bf16, cudaStream_t s) {
  using B = __nv_bfloat162;
  using F = float2;
  if (!w_bf16) {
    if (!in_bf16 && !out_bf16) return fwd_t<CI, CO, F, F, F>(g, in, W, out, s);
    return cudaErrorInvalidValue;  // FP32 weights go with FP32 activations
  }
  if (!in_bf16 && !out_bf16) return fwd_t<CI, CO, F, F, B>(g, in, W, out, s);
  if (!in_bf16 && out_bf16) return fwd_t<CI, CO, F, B, B>(g, in, W, out, s);
  if (in_bf16 && out_bf16) return fwd_t<CI, CO, B, B, B>(g, in, W, out, s);
  return fwd_t<CI, CO, B, F, B>(g, in, W, out, s);
}

}  // namespace

cudaError_t launch_net_layer(const net_geom& g, int ci, int co, const void* in, bool in_bf16, const void* W,
                             bool w_bf16, void* out, bool out_bf16, cudaStream_t s) {
  if (ci == 4 && co == 8) return fwd_any<4, 8>(g, in, in_bf16, W, w_bf16, out, out_bf16, s);
  if (ci == 8 && co == 8) return fwd_any<8, 8>(g, in, in_bf16, W, w_bf16, out, out_bf16, s);
  if (ci == 8 && co == 4) return fwd_any<8, 4>(g, in, in_bf16, W, w_bf16, out, out_bf16, s);
  if (ci == 4 && co == 4) return fwd_any<4, 4>(g, in, in_bf16, W, w_bf16, out, out_bf16, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_net_wgrad(const net_geom& g, int ci, int co, const void* in, bool in_bf16, const float2* delta,
                             int spc, double2* partial, cudaStream_t s) {
  if (ci == 4 && co == 8)
    return in_bf16 ? wgrad_t<4, 8, __nv_bfloat162>(g, in, delta, spc, partial, s)
                   : wgrad_t<4, 8, float2>(g, in, delta, spc, partial, s);
  if (ci == 8 && co == 8)
    return in_bf16 ? wgrad_t<8, 8, __nv_bfloat162>(g, in, delta, spc, partial, s)
                   : wgrad_t<8, 8, float2>(g, in, delta, spc, partial, s);
  if (ci == 8 && co == 4)
    return in_bf16 ? wgrad_t<8, 4, __nv_bfloat162>(g, in, delta, spc, partial, s)
                   : wgrad_t<8, 4, float2>(g, in, delta, spc, partial, s);
  if (ci == 4 && co == 4)
    return in_bf16 ? wgrad_t<4, 4, __nv_bfloat162>(g, in, delta, spc, partial, s)
                   : wgrad_t<4, 4, float2>(g, in, delta, spc, partial, s);
  return cudaErrorInvalidValue;
}

}  // namespace mmc
