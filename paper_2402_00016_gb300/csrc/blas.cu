// Field kernels around the stencil: Z(4) noise from Philox4x32-10, probe
// vectors, layout conversion, and the batched dot products / updates that
// the CGS2 Arnoldi process, the solves and the deflation projections use.
// Every reduction is two-stage (per-CTA partial, then a fixed-order sum over
// CTAs) so results do not depend on scheduling.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "stencil_ops.cuh"

namespace mmc {
namespace {

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): per round, words 0 and 2 are
// multiplied by two 32-bit constants; the high halves are mixed with words 1
// and 3 and the round key, the low halves become words 1 and 3; the key gets
// two Weyl increments between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

template <typename T>
__device__ __forceinline__ void put(T* f, size_t i, double re, double im);
template <>
__device__ __forceinline__ void put<double2>(double2* f, size_t i, double re, double im) {
  f[i] = make_double2(re, im);
}
template <>
__device__ __forceinline__ void put<float2>(float2* f, size_t i, double re, double im) {
  f[i] = make_float2(float(re), float(im));
}
template <>
__device__ __forceinline__ void put<__nv_bfloat162>(__nv_bfloat162* f, size_t i, double re, double im) {
  f[i] = __float22bfloat162_rn(make_float2(float(re), float(im)));
}

template <typename T>
__device__ __forceinline__ double2 get(const T* f, size_t i);
template <>
__device__ __forceinline__ double2 get<double2>(const double2* f, size_t i) {
  return f[i];
}
template <>
__device__ __forceinline__ double2 get<float2>(const float2* f, size_t i) {
  float2 v = f[i];
  return make_double2(v.x, v.y);
}
template <>
__device__ __forceinline__ double2 get<__nv_bfloat162>(const __nv_bfloat162* f, size_t i) {
  float2 v = __bfloat1622float2(f[i]);
  return make_double2(v.x, v.y);
}

// Arithmetic precision of a field type: FP64 fields compute in FP64; FP32 and BF16
// fields in FP32 (GB300 runs FP64 at a small fraction of the FP32 rate).
template <typename T>
struct Arith {
  using R = float;
  using C = float2;
};
template <>
struct Arith<double2> {
  using R = double;
  using C = double2;
};

template <typename T>
__device__ __forceinline__ typename Arith<T>::C getc(const T* f, size_t i);
template <>
__device__ __forceinline__ double2 getc<double2>(const double2* f, size_t i) {
  return f[i];
}
template <>
__device__ __forceinline__ float2 getc<float2>(const float2* f, size_t i) {
  return f[i];
}
template <>
__device__ __forceinline__ float2 getc<__nv_bfloat162>(const __nv_bfloat162* f, size_t i) {
  return __bfloat1622float2(f[i]);
}

// store in the field's own precision from its arithmetic type (no FP64 round trip)
__device__ __forceinline__ void putc(double2* f, size_t i, double2 v) { f[i] = v; }
__device__ __forceinline__ void putc(float2* f, size_t i, float2 v) { f[i] = v; }
__device__ __forceinline__ void putc(__nv_bfloat162* f, size_t i, float2 v) { f[i] = __float22bfloat162_rn(v); }

__device__ __forceinline__ size_t fidx(const geom& g, int rb, int site, int c, int r) {
  return ((size_t(rb) * g.V + site) * 12 + c) * g.R + r;
}

// thread -> (rb = blockIdx.y, site, r) with R lanes per site
template <typename T>
__global__ void noise_kernel(geom g, const uint2* ids, uint32_t tag, uint32_t k0, uint32_t k1, T* field,
                             uint32_t* codes) {
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int site = (blockIdx.x * blockDim.x + threadIdx.x) / g.R;
  if (site >= g.V) return;
  const uint2 id = ids[rb * g.R + r];
  uint32_t w0 = 0;
  const bool live = id.x != 0xffffffffu;
  if (live) w0 = philox10(make_uint4(uint32_t(site), id.y, id.x, tag), k0, k1).x;
  if (codes) codes[(size_t(rb) * g.V + site) * g.R + r] = w0;
  if (field) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      uint32_t k = (w0 >> (2 * c)) & 3u;
      double re = (k == 0) ? 1.0 : (k == 2 ? -1.0 : 0.0);
      double im = (k == 1) ? 1.0 : (k == 3 ? -1.0 : 0.0);
      if (!live) re = im = 0.0;
      put<T>(field, fidx(g, rb, site, c, r), re, im);
    }
  }
}

template <typename T>
__global__ void probe_kernel(geom g, const int* site_colour, const int2* probe, T* field) {
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int site = (blockIdx.x * blockDim.x + threadIdx.x) / g.R;
  if (site >= g.V) return;
  const int2 pr = probe[rb * g.R + r];  // (colour, component); colour < 0: padding
  const bool on = pr.x >= 0 && site_colour[site] == pr.x;
#pragma unroll
  for (int c = 0; c < 12; ++c) put<T>(field, fidx(g, rb, site, c, r), (on && c == pr.y) ? 1.0 : 0.0, 0.0);
}

template <typename T>
__global__ void pack_kernel(geom g, int nrhs, const double2* canon, T* field) {
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int site = (blockIdx.x * blockDim.x + threadIdx.x) / g.R;
  if (site >= g.V) return;
  const int rg = rb * g.R + r;
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    double2 v = (rg < nrhs) ? canon[(size_t(rg) * g.V + site) * 12 + c] : make_double2(0.0, 0.0);
    put<T>(field, fidx(g, rb, site, c, r), v.x, v.y);
  }
}

template <typename T>
__global__ void unpack_kernel(geom g, int nrhs, const T* field, double2* canon) {
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int site = (blockIdx.x * blockDim.x + threadIdx.x) / g.R;
  if (site >= g.V) return;
  const int rg = rb * g.R + r;
  if (rg >= nrhs) return;
#pragma unroll
  for (int c = 0; c < 12; ++c) canon[(size_t(rg) * g.V + site) * 12 + c] = get<T>(field, fidx(g, rb, site, c, r));
}

template <typename D, typename S>
__global__ void convert_kernel(size_t n, D* dst, const S* src) {
  size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  size_t stride = size_t(gridDim.x) * blockDim.x;
  for (; i < n; i += stride) {
    double2 v = get<S>(src, i);
    put<D>(dst, i, v.x, v.y);
  }
}

// Reduce (re, im) over the threads of the CTA that share r = threadIdx.x % R;
// thread r < R of the CTA returns the total in (re, im).
__device__ __forceinline__ void cta_reduce_r(double& re, double& im, int R, double2* sh) {
  for (int off = R; off < 32; off <<= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, off);
    im += __shfl_xor_sync(0xffffffffu, im, off);
  }
  const int warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  __syncthreads();
  if (wl < R && wl < 32) sh[warp * 32 + wl] = make_double2(re, im);
  __syncthreads();
  if (threadIdx.x < R) {
    double sr = 0, si = 0;
    for (int w = 0; w < nw; ++w) {
      sr += sh[w * 32 + threadIdx.x].x;
      si += sh[w * 32 + threadIdx.x].y;
    }
    re = sr;
    im = si;
  }
}

// conj(a) * (Theta w) accumulated over 12 components
__device__ __forceinline__ void theta_dot(const double2 (&a)[12], const double2 (&w)[12], int theta, double& re,
                                          double& im) {
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    int src = (theta == 1) ? (c + 6) % 12 : c;
    double sg = (theta == 2 && c >= 6) ? -1.0 : 1.0;
    double2 x = w[src];
    re += sg * (a[c].x * x.x + a[c].y * x.y);
    im += sg * (a[c].x * x.y - a[c].y * x.x);
  }
}

// partial[bx][i][npad] = sum over the CTA's sites of conj(A_i) . Theta w, for i < nvec.
// Basis vectors are processed NB at a time: w is read once per chunk and the NB
// sums stay in registers (FP32 for FP32/BF16 fields, FP64 for FP64 fields).
template <typename T, int NB>
__global__ void multidot_kernel(geom g, const T* A, size_t a_stride, int nvec, const T* w, int theta, int spc,
                                double2* partial) {
  using R = typename Arith<T>::R;
  using C = typename Arith<T>::C;
  __shared__ double2 sh[8 * 32];
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int spp = blockDim.x / g.R;
  const int s_begin = blockIdx.x * spc, s_end = min(g.V, s_begin + spc);
  for (int i0 = 0; i0 < nvec; i0 += NB) {
    R re[NB], im[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) re[q] = im[q] = R(0);
    for (int s0 = s_begin; s0 < s_end; s0 += spp) {
      const int site = s0 + threadIdx.x / g.R;
      if (site >= s_end) continue;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        const int src = (theta == 1) ? (c + 6) % 12 : c;
        const R sg = (theta == 2 && c >= 6) ? R(-1) : R(1);
        const C x = getc<T>(w, fidx(g, rb, site, src, r));
        const size_t e = fidx(g, rb, site, c, r);
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          if (i0 + q < nvec) {
            const C a = getc<T>(A + size_t(i0 + q) * a_stride, e);
            re[q] += sg * (a.x * x.x + a.y * x.y);
            im[q] += sg * (a.x * x.y - a.y * x.x);
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      if (i0 + q >= nvec) break;
      double dre = re[q], dim = im[q];
      cta_reduce_r(dre, dim, g.R, sh);
      if (threadIdx.x < g.R)
        partial[(size_t(blockIdx.x) * nvec + i0 + q) * g.npad + rb * g.R + threadIdx.x] = make_double2(dre, dim);
    }
  }
}

// out[idx] (+)= sum_b partial[b][idx] in a fixed order: a CTA of 32 x 32 threads takes 32
// consecutive outputs; thread row j sums rows b = j, j + 32, ... with eight independent
// accumulators (loads in flight), then the 32 row sums are added in order.
constexpr int kRedRows = 32;
__global__ void __launch_bounds__(1024) reduce_kernel(const double2* partial, int nbx, int nvec, int npad,
                                                      double2* out, int accumulate) {
  __shared__ double2 rs[kRedRows][33];
  const int n = nvec * npad;
  const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
  const int idx = blockIdx.x * 32 + lane;
  double re[8], im[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) re[u] = im[u] = 0.0;
  if (idx < n) {
    int b = row;
    for (; b + 7 * kRedRows < nbx; b += 8 * kRedRows) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const double2 v = partial[size_t(b + u * kRedRows) * n + idx];
        re[u] += v.x;
        im[u] += v.y;
      }
    }
    for (; b < nbx; b += kRedRows) {
      const double2 v = partial[size_t(b) * n + idx];
      re[0] += v.x;
      im[0] += v.y;
    }
  }
  double tr = 0, ti = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    tr += re[u];
    ti += im[u];
  }
  rs[row][lane] = make_double2(tr, ti);
  __syncthreads();
  if (row == 0 && idx < n) {
    double a = 0, c = 0;
    for (int j = 0; j < kRedRows; ++j) {
      a += rs[j][lane].x;
      c += rs[j][lane].y;
    }
    if (accumulate) {
      a += out[idx].x;
      c += out[idx].y;
    }
    out[idx] = make_double2(a, c);
  }
}

template <typename T>
__global__ void basis_update_kernel(geom g, const T* A, size_t a_stride, int nvec, const double2* h, T* w) {
  using R = typename Arith<T>::R;
  using C = typename Arith<T>::C;
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int site = (blockIdx.x * blockDim.x + threadIdx.x) / g.R;
  if (site >= g.V) return;
  const int rg = rb * g.R + r;
  C acc[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = getc<T>(w, fidx(g, rb, site, c, r));
  for (int i = 0; i < nvec; ++i) {
    const double2 hd = h[size_t(i) * g.npad + rg];
    const R hx = R(hd.x), hy = R(hd.y);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      C a = getc<T>(A + size_t(i) * a_stride, fidx(g, rb, site, c, r));
      acc[c].x -= a.x * hx - a.y * hy;
      acc[c].y -= a.x * hy + a.y * hx;
    }
  }
#pragma unroll
  for (int c = 0; c < 12; ++c) put<T>(w, fidx(g, rb, site, c, r), acc[c].x, acc[c].y);
}

// The basis update of a Gram-Schmidt pass fused with the dot products that follow it:
// w <- w - sum_i h_i A_i (nvec <= 8 basis fields), then, from the updated w still in
// registers, either partial[b][i] = sum A_i^H w (the next pass's projections, NORM
// false) or partial[b][0] = w^H w (NORM true), per CTA of spc sites as multidot_kernel
// lays them out.  One read of A and w instead of two.
template <bool NORM>
__global__ void update_dot_kernel(geom g, const float2* A, size_t a_stride, int nvec, const double2* h, float2* w,
                                  int spc, double2* partial) {
  constexpr int NB = 8;
  __shared__ double2 sh[8 * 32];
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int spp = blockDim.x / g.R;
  const int rg = rb * g.R + r;
  float hx[NB], hy[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const double2 hd = q < nvec ? h[size_t(q) * g.npad + rg] : make_double2(0.0, 0.0);
    hx[q] = float(hd.x);
    hy[q] = float(hd.y);
  }
  float re[NB], im[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) re[q] = im[q] = 0.f;
  const int s_begin = blockIdx.x * spc, s_end = min(g.V, s_begin + spc);
  for (int s0 = s_begin; s0 < s_end; s0 += spp) {
    const int site = s0 + threadIdx.x / g.R;
    if (site >= s_end) continue;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const size_t e = fidx(g, rb, site, c, r);
      float2 x = w[e];
      float2 a[NB];
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        if (q < nvec) {
          a[q] = A[size_t(q) * a_stride + e];
          x.x -= a[q].x * hx[q] - a[q].y * hy[q];
          x.y -= a[q].x * hy[q] + a[q].y * hx[q];
        }
      }
      w[e] = x;
      if (NORM) {
        re[0] += x.x * x.x + x.y * x.y;
      } else {
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          if (q < nvec) {
            re[q] += a[q].x * x.x + a[q].y * x.y;
            im[q] += a[q].x * x.y - a[q].y * x.x;
          }
        }
      }
    }
  }
  const int nout = NORM ? 1 : nvec;
  for (int q = 0; q < nout; ++q) {
    double dre = re[q], dim = im[q];
    cta_reduce_r(dre, dim, g.R, sh);
    if (threadIdx.x < g.R) partial[(size_t(blockIdx.x) * nout + q) * g.npad + rb * g.R + threadIdx.x] = make_double2(dre, dim);
  }
}

template <typename T>
__global__ void normalise_kernel(geom g, const T* src, const double2* nrm2, T* dst) {
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int site = (blockIdx.x * blockDim.x + threadIdx.x) / g.R;
  if (site >= g.V) return;
  using R = typename Arith<T>::R;
  using C = typename Arith<T>::C;
  const double n2 = nrm2[rb * g.R + r].x;
  const R sc = R(n2 > 0 ? 1.0 / sqrt(n2) : 0.0);  // in the field's arithmetic precision
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    size_t e = fidx(g, rb, site, c, r);
    C v = getc<T>(src, e);
    v.x *= sc;
    v.y *= sc;
    putc(dst, e, v);
  }
}

template <typename T>
__global__ void axpby_kernel(geom g, const double2* a, const T* x, const double2* b, T* y) {
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int site = (blockIdx.x * blockDim.x + threadIdx.x) / g.R;
  if (site >= g.V) return;
  const int rg = rb * g.R + r;
  // in the field's arithmetic precision (FP32 for FP32 and BF16 fields)
  using R = typename Arith<T>::R;
  using C = typename Arith<T>::C;
  const double2 da = a ? a[rg] : make_double2(0, 0), db = b ? b[rg] : make_double2(0, 0);
  const R ax = R(da.x), ay = R(da.y), bx = R(db.x), by = R(db.y);
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    size_t e = fidx(g, rb, site, c, r);
    C xv = x ? getc<T>(x, e) : C{R(0), R(0)};
    C yv = b ? getc<T>(y, e) : C{R(0), R(0)};
    C o;
    o.x = ax * xv.x - ay * xv.y + bx * yv.x - by * yv.y;
    o.y = ax * xv.y + ay * xv.x + bx * yv.y + by * yv.x;
    putc(y, e, o);
  }
}

template <typename T>
__global__ void gamma_kernel(geom g, int theta, const T* src, T* dst) {
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int site = (blockIdx.x * blockDim.x + threadIdx.x) / g.R;
  if (site >= g.V) return;
  double2 v[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) v[c] = get<T>(src, fidx(g, rb, site, c, r));
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    int s = (theta == 1) ? (c + 6) % 12 : c;
    double sg = (theta == 2 && c >= 6) ? -1.0 : 1.0;
    put<T>(dst, fidx(g, rb, site, c, r), sg * v[s].x, sg * v[s].y);
  }
}

template <typename T>
__global__ void bilinear_codes_kernel(geom g, const uint32_t* codes, int theta, const T* x, int spc,
                                      double2* partial) {
  __shared__ double2 sh[8 * 32];
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int spp = blockDim.x / g.R;
  const int s_begin = blockIdx.x * spc, s_end = min(g.V, s_begin + spc);
  double re = 0, im = 0;
  for (int s0 = s_begin; s0 < s_end; s0 += spp) {
    int site = s0 + threadIdx.x / g.R;
    if (site >= s_end) continue;
    uint32_t code = codes[(size_t(rb) * g.V + site) * g.R + r];
    double2 a[12], xv[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      uint32_t k = (code >> (2 * c)) & 3u;
      a[c] = make_double2(k == 0 ? 1.0 : (k == 2 ? -1.0 : 0.0), k == 1 ? 1.0 : (k == 3 ? -1.0 : 0.0));
      xv[c] = get<T>(x, fidx(g, rb, site, c, r));
    }
    theta_dot(a, xv, theta, re, im);
  }
  cta_reduce_r(re, im, g.R, sh);
  if (threadIdx.x < g.R) {
    double2* d = partial + size_t(blockIdx.x) * g.npad + rb * g.R + threadIdx.x;
    double2 cur = *d;
    *d = make_double2(cur.x + re, cur.y + im);
  }
}

// a[i][r] = sum conj(eta_r) Theta z_i ; b[i][r] = sum conj(u_i) eta_r.  z_i, u_i are
// single-vector fields ([site][12], R = 1 layout) of type E (double2 or float2);
// the per-thread sums run in E's precision, the CTA reduction in FP64.
template <typename E>
__global__ void defl_proj_kernel(geom g, const uint32_t* codes, int theta, const E* Z, const E* U, int k, int spc,
                                 double2* pa, double2* pb) {
  using R = decltype(E().x);
  __shared__ double2 sh[8 * 32];
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int spp = blockDim.x / g.R;
  const int s_begin = blockIdx.x * spc, s_end = min(g.V, s_begin + spc);
  const size_t n = size_t(g.V) * 12;
  for (int i = 0; i < k; ++i) {
    R are = 0, aim = 0, bre = 0, bim = 0;
    for (int s0 = s_begin; s0 < s_end; s0 += spp) {
      int site = s0 + threadIdx.x / g.R;
      if (site >= s_end) continue;
      uint32_t code = codes[(size_t(rb) * g.V + site) * g.R + r];
      const E* zp = Z + size_t(i) * n + size_t(site) * 12;
      const E* up = U + size_t(i) * n + size_t(site) * 12;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        // a: conj(eta_c) (Theta z)_c ; b: conj(u_c) eta_c with eta_c = i^k
        const int src = (theta == 1) ? (c + 6) % 12 : c;
        const R sg = (theta == 2 && c >= 6) ? R(-1) : R(1);
        E zv = zp[src];
        E uv = up[c];
        const uint32_t kk = (code >> (2 * c)) & 3u;
        R er = (kk == 0) ? R(1) : (kk == 2 ? R(-1) : R(0));
        R ei = (kk == 1) ? R(1) : (kk == 3 ? R(-1) : R(0));
        are += sg * (er * zv.x + ei * zv.y);
        aim += sg * (er * zv.y - ei * zv.x);
        bre += uv.x * er + uv.y * ei;
        bim += uv.x * ei - uv.y * er;
      }
    }
    double dar = are, dai = aim, dbr = bre, dbi = bim;
    cta_reduce_r(dar, dai, g.R, sh);
    if (threadIdx.x < g.R) pa[(size_t(blockIdx.x) * k + i) * g.npad + rb * g.R + threadIdx.x] = make_double2(dar, dai);
    cta_reduce_r(dbr, dbi, g.R, sh);
    if (threadIdx.x < g.R) pb[(size_t(blockIdx.x) * k + i) * g.npad + rb * g.R + threadIdx.x] = make_double2(dbr, dbi);
  }
}

// c[i][r] (partial) = sum over the CTA's sites of conj(v_i) . f_r, v_i single-vector FP64 fields.
template <typename T>
__global__ void vec_proj_kernel(geom g, const double2* Vv, int k, const T* f, int spc, double2* partial) {
  __shared__ double2 sh[8 * 32];
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int spp = blockDim.x / g.R;
  const int s_begin = blockIdx.x * spc, s_end = min(g.V, s_begin + spc);
  const size_t n = size_t(g.V) * 12;
  for (int i = 0; i < k; ++i) {
    double re = 0, im = 0;
    for (int s0 = s_begin; s0 < s_end; s0 += spp) {
      int site = s0 + threadIdx.x / g.R;
      if (site >= s_end) continue;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        double2 v = Vv[size_t(i) * n + size_t(site) * 12 + c];
        double2 x = get<T>(f, fidx(g, rb, site, c, r));
        re += v.x * x.x + v.y * x.y;
        im += v.x * x.y - v.y * x.x;
      }
    }
    cta_reduce_r(re, im, g.R, sh);
    if (threadIdx.x < g.R) partial[(size_t(blockIdx.x) * k + i) * g.npad + rb * g.R + threadIdx.x] = make_double2(re, im);
  }
}

// f_r += sum_i v_i coef[i][r], v_i single-vector FP64 fields.
template <typename T>
__global__ void vec_update_kernel(geom g, const double2* Vv, int k, const double2* coef, T* f) {
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int site = (blockIdx.x * blockDim.x + threadIdx.x) / g.R;
  if (site >= g.V) return;
  const int rg = rb * g.R + r;
  const size_t n = size_t(g.V) * 12;
#pragma unroll 1
  for (int c = 0; c < 12; ++c) {
    size_t e = fidx(g, rb, site, c, r);
    double2 acc = get<T>(f, e);
    for (int i = 0; i < k; ++i) {
      double2 v = Vv[size_t(i) * n + size_t(site) * 12 + c];
      double2 h = coef[size_t(i) * g.npad + rg];
      acc.x += v.x * h.x - v.y * h.y;
      acc.y += v.x * h.y + v.y * h.x;
    }
    put<T>(f, e, acc.x, acc.y);
  }
}

// FP32 forms of the two kernels above for the corrections inside refined solves
// (the outer FP64 residual absorbs their rounding).  The vectors v_i are FP32
// copies; each thread owns one (site, rhs), keeps its 12 field components in
// registers, and takes the eigenvectors in chunks of kVc with one CTA reduction
// per chunk, so the field is read once per chunk from L1 and every v_i once.
constexpr int kVc = 8;

template <typename T>
__global__ void vec_proj32_kernel(geom g, const float2* Vv, int k, const T* f, int spc, double2* partial) {
  __shared__ double2 sh[8 * 32];
  const int rb = blockIdx.y;
  const int r = threadIdx.x % g.R;
  const int spp = blockDim.x / g.R;
  const int s_begin = blockIdx.x * spc, s_end = min(g.V, s_begin + spc);
  const size_t n = size_t(g.V) * 12;
  for (int i0 = 0; i0 < k; i0 += kVc) {
    float2 acc[kVc];
#pragma unroll
    for (int q = 0; q < kVc; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int s0 = s_begin; s0 < s_end; s0 += spp) {
      const int site = s0 + threadIdx.x / g.R;
      if (site >= s_end) continue;
      float2 x[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        const double2 v = get<T>(f, fidx(g, rb, site, c, r));
        x[c] = make_float2(float(v.x), float(v.y));
      }
#pragma unroll
      for (int q = 0; q < kVc; ++q) {
        if (i0 + q >= k) break;
        const float2* vi = Vv + size_t(i0 + q) * n + size_t(site) * 12;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          const float2 v = __ldg(vi + c);
          acc[q].x = fmaf(v.x, x[c].x, fmaf(v.y, x[c].y, acc[q].x));
          acc[q].y = fmaf(v.x, x[c].y, fmaf(-v.y, x[c].x, acc[q].y));
        }
      }
    }
#pragma unroll 1
    for (int q = 0; q < kVc && i0 + q < k; ++q) {
      double re = acc[q].x, im = acc[q].y;
      cta_reduce_r(re, im, g.R, sh);
      if (threadIdx.x < g.R)
        partial[(size_t(blockIdx.x) * k + i0 + q) * g.npad + rb * g.R + threadIdx.x] = make_double2(re, im);
    }
  }
}

template <typename T>
__global__ void vec_update32_kernel(geom g, const float2* Vv, int k, const double2* coef, T* f) {
  extern __shared__ float2 sc[];  // [k][R] coefficients of this rhs block
  const int rb = blockIdx.y;
  for (int e = threadIdx.x; e < k * g.R; e += blockDim.x) {
    const double2 h = coef[size_t(e / g.R) * g.npad + rb * g.R + e % g.R];
    sc[e] = make_float2(float(h.x), float(h.y));
  }
  __syncthreads();
  const int r = threadIdx.x % g.R;
  const int site = (blockIdx.x * blockDim.x + threadIdx.x) / g.R;
  if (site >= g.V) return;
  const size_t n = size_t(g.V) * 12;
  float2 acc[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = make_float2(0.f, 0.f);
#pragma unroll 2
  for (int i = 0; i < k; ++i) {
    const float2 h = sc[i * g.R + r];
    const float2* vi = Vv + size_t(i) * n + size_t(site) * 12;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const float2 v = __ldg(vi + c);
      acc[c].x = fmaf(v.x, h.x, fmaf(-v.y, h.y, acc[c].x));
      acc[c].y = fmaf(v.x, h.y, fmaf(v.y, h.x, acc[c].y));
    }
  }
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const size_t e = fidx(g, rb, site, c, r);
    const double2 y = get<T>(f, e);
    put<T>(f, e, y.x + double(acc[c].x), y.y + double(acc[c].y));
  }
}

__global__ void add2_kernel(const double2* a, const double2* b, double2* out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_double2(a[i].x + b[i].x, a[i].y + b[i].y);
}

inline dim3 site_grid(const geom& g, int threads) {
  size_t total = size_t(g.V) * g.R;
  return dim3(unsigned((total + threads - 1) / threads), unsigned(g.nrb));
}

}  // namespace

#define MMC_DISPATCH3(prec, F, ...)                          \
  do {                                                      \
    if ((prec) == 0) F<double2> __VA_ARGS__;                \
    else if ((prec) == 1) F<float2> __VA_ARGS__;            \
    else F<__nv_bfloat162> __VA_ARGS__;                     \
  } while (0)

cudaError_t launch_noise(int prec, geom g, const uint2* ids, uint32_t tag, uint64_t seed, void* field,
                         uint32_t* codes, cudaStream_t s) {
  const int th = 256;
  dim3 grid = site_grid(g, th);
  uint32_t k0 = uint32_t(seed & 0xffffffffu), k1 = uint32_t(seed >> 32);
  if (prec == 0)
    noise_kernel<double2><<<grid, th, 0, s>>>(g, ids, tag, k0, k1, (double2*)field, codes);
  else if (prec == 1)
    noise_kernel<float2><<<grid, th, 0, s>>>(g, ids, tag, k0, k1, (float2*)field, codes);
  else
    noise_kernel<__nv_bfloat162><<<grid, th, 0, s>>>(g, ids, tag, k0, k1, (__nv_bfloat162*)field, codes);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_probe(int prec, geom g, const int* site_colour, const int2* probe, void* field,
                         cudaStream_t s) {
  const int th = 256;
  dim3 grid = site_grid(g, th);
  if (prec == 0)
    probe_kernel<double2><<<grid, th, 0, s>>>(g, site_colour, probe, (double2*)field);
  else if (prec == 1)
    probe_kernel<float2><<<grid, th, 0, s>>>(g, site_colour, probe, (float2*)field);
  else
    probe_kernel<__nv_bfloat162><<<grid, th, 0, s>>>(g, site_colour, probe, (__nv_bfloat162*)field);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pack(int prec, geom g, int nrhs, const double2* canon, void* field, cudaStream_t s) {
  const int th = 256;
  dim3 grid = site_grid(g, th);
  if (prec == 0)
    pack_kernel<double2><<<grid, th, 0, s>>>(g, nrhs, canon, (double2*)field);
  else if (prec == 1)
    pack_kernel<float2><<<grid, th, 0, s>>>(g, nrhs, canon, (float2*)field);
  else
    pack_kernel<__nv_bfloat162><<<grid, th, 0, s>>>(g, nrhs, canon, (__nv_bfloat162*)field);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_unpack(int prec, geom g, int nrhs, const void* field, double2* canon, cudaStream_t s) {
  const int th = 256;
  dim3 grid = site_grid(g, th);
  if (prec == 0)
    unpack_kernel<double2><<<grid, th, 0, s>>>(g, nrhs, (const double2*)field, canon);
  else if (prec == 1)
    unpack_kernel<float2><<<grid, th, 0, s>>>(g, nrhs, (const float2*)field, canon);
  else
    unpack_kernel<__nv_bfloat162><<<grid, th, 0, s>>>(g, nrhs, (const __nv_bfloat162*)field, canon);
  count_launch();
  return cudaGetLastError();
}

template <typename D>
static void convert_from(int ps, size_t n, D* dst, const void* src, cudaStream_t s) {
  unsigned blocks = unsigned(std::min<size_t>((n + 255) / 256, 152 * 64));
  if (ps == 0)
    convert_kernel<D, double2><<<blocks, 256, 0, s>>>(n, dst, (const double2*)src);
  else if (ps == 1)
    convert_kernel<D, float2><<<blocks, 256, 0, s>>>(n, dst, (const float2*)src);
  else
    convert_kernel<D, __nv_bfloat162><<<blocks, 256, 0, s>>>(n, dst, (const __nv_bfloat162*)src);
}

// FP32 -> BF16 with stochastic rounding, stream key from *salt (a different stream
// from the step kernels' keys of the same salt)
__global__ void convert_sr_kernel(size_t n, __nv_bfloat162* dst, const float2* src, const uint32_t* salt) {
  const uint32_t key = __ldg(salt) ^ 0x5bd1e995u;
  size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t stride = size_t(gridDim.x) * blockDim.x;
  for (; i < n; i += stride) {
    const float2 v = src[i];
    const uint32_t r = sten::sr_bits(uint32_t(i), key);
    reinterpret_cast<uint32_t*>(dst)[i] = sten::bf16_bits_sr(v.x, r) | (sten::bf16_bits_sr(v.y, r >> 16) << 16);
  }
}

__global__ void salt_advance_kernel(uint32_t* salt) {
  // one step of a 32-bit linear congruential sequence (Numerical Recipes constants)
  *salt = *salt * 1664525u + 1013904223u;
}

cudaError_t launch_convert_sr(void* dst, const void* src, geom g, const uint32_t* salt, cudaStream_t s) {
  const size_t n = size_t(g.nrb) * g.V * 12 * g.R;
  const unsigned blocks = unsigned(std::min<size_t>((n + 255) / 256, 152 * 64));
  convert_sr_kernel<<<blocks, 256, 0, s>>>(n, (__nv_bfloat162*)dst, (const float2*)src, salt);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_salt_advance(uint32_t* salt, cudaStream_t s) {
  salt_advance_kernel<<<1, 1, 0, s>>>(salt);
  count_launch();
  return cudaGetLastError();
}

// FP32 field between the blocked layout [rb][site][c][R] and the paired-component layout
// [rb][site][c/2][R][c%2] (a permutation within each site's 12 R elements)
__global__ void pair_layout_kernel(size_t n, int R, int to_paired, float2* __restrict__ dst,
                                   const float2* __restrict__ src) {
  const size_t blk_elems = size_t(12) * R;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const size_t blk = i / blk_elems;
    const int w = int(i - blk * blk_elems);
    const int c = w / R, r = w - c * R;
    const size_t j = blk * blk_elems + size_t(c >> 1) * 2 * R + 2 * r + (c & 1);
    if (to_paired)
      dst[j] = src[i];
    else
      dst[i] = src[j];
  }
}

cudaError_t launch_pair_layout(void* dst, const void* src, geom g, int to_paired, cudaStream_t s) {
  const size_t n = size_t(g.nrb) * g.V * 12 * g.R;
  const unsigned blocks = unsigned(std::min<size_t>((n + 255) / 256, 152 * 64));
  pair_layout_kernel<<<blocks, 256, 0, s>>>(n, g.R, to_paired, (float2*)dst, (const float2*)src);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_convert(int pd, void* dst, int ps, const void* src, geom g, cudaStream_t s) {
  size_t n = size_t(g.nrb) * g.V * 12 * g.R;
  if (pd == 0)
    convert_from<double2>(ps, n, (double2*)dst, src, s);
  else if (pd == 1)
    convert_from<float2>(ps, n, (float2*)dst, src, s);
  else
    convert_from<__nv_bfloat162>(ps, n, (__nv_bfloat162*)dst, src, s);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_multidot(int prec, geom g, const void* A, size_t a_stride, int nvec, const void* w, int theta,
                            int spc, double2* partial, cudaStream_t s) {
  dim3 grid((g.V + spc - 1) / spc, g.nrb);
  if (prec == 0)
    multidot_kernel<double2, 4><<<grid, 256, 0, s>>>(g, (const double2*)A, a_stride, nvec, (const double2*)w, theta,
                                                     spc, partial);
  else
    multidot_kernel<float2, 8><<<grid, 256, 0, s>>>(g, (const float2*)A, a_stride, nvec, (const float2*)w, theta,
                                                    spc, partial);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double2* partial, int nbx, int nvec, int npad, double2* out, int accumulate,
                          cudaStream_t s) {
  int n = nvec * npad;
  reduce_kernel<<<(n + 31) / 32, 32 * kRedRows, 0, s>>>(partial, nbx, nvec, npad, out, accumulate);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_basis_update(int prec, geom g, const void* A, size_t a_stride, int nvec, const double2* h,
                                void* w, cudaStream_t s) {
  dim3 grid = site_grid(g, 256);
  if (prec == 0)
    basis_update_kernel<double2><<<grid, 256, 0, s>>>(g, (const double2*)A, a_stride, nvec, h, (double2*)w);
  else
    basis_update_kernel<float2><<<grid, 256, 0, s>>>(g, (const float2*)A, a_stride, nvec, h, (float2*)w);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_normalise(int prec, geom g, const void* src, const double2* nrm2, void* dst, cudaStream_t s) {
  dim3 grid = site_grid(g, 256);
  if (prec == 0)
    normalise_kernel<double2><<<grid, 256, 0, s>>>(g, (const double2*)src, nrm2, (double2*)dst);
  else
    normalise_kernel<float2><<<grid, 256, 0, s>>>(g, (const float2*)src, nrm2, (float2*)dst);
  count_launch();
  return cudaGetLastError();
}

// flag <- 1 if some FP64 link's third row differs by more than 1e-10 from the conjugate
// cross product of its first two rows (negated on the time links at t = Lt - 1 when the
// antiperiodic phase is folded in): the condition for rebuilding the third row.
__global__ void su3_rows_check_kernel(const double2* __restrict__ links, int V, int slice, int Lt, int tap,
                                      int* flag) {
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // link (site, mu)
  if (l >= 4ll * V) return;
  const int site = int(l / 4), mu = int(l % 4);
  const double2* u = links + l * 9;
  const double sg = (tap && mu == 3 && site >= (Lt - 1) * slice) ? -1.0 : 1.0;
  bool bad = false;
  for (int c = 0; c < 3; ++c) {
    const int a = (c + 1) % 3, b = (c + 2) % 3;
    const double2 x0 = u[a], y1 = u[3 + b], x1 = u[b], y0 = u[3 + a];
    // (row0 x row1)_c = r0[a] r1[b] - r0[b] r1[a], then conjugated and signed
    const double re = (x0.x * y1.x - x0.y * y1.y) - (x1.x * y0.x - x1.y * y0.y);
    const double im = (x0.x * y1.y + x0.y * y1.x) - (x1.x * y0.y + x1.y * y0.x);
    const double2 r2 = u[6 + c];
    if (fabs(sg * re - r2.x) > 1e-10 || fabs(-sg * im - r2.y) > 1e-10) bad = true;
  }
  if (bad) atomicOr(flag, 1);
}

cudaError_t launch_su3_rows_check(const double2* links, int V, int slice, int Lt, int tap, int* flag,
                                  cudaStream_t s) {
  const long long n = 4ll * V;
  su3_rows_check_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(links, V, slice, Lt, tap, flag);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_update_dot(geom g, const float2* A, size_t a_stride, int nvec, const double2* h, float2* w,
                              bool norm, int spc, double2* partial, cudaStream_t s) {
  if (nvec < 1 || nvec > 8) return cudaErrorInvalidValue;
  dim3 grid((g.V + spc - 1) / spc, g.nrb);
  if (norm)
    update_dot_kernel<true><<<grid, 256, 0, s>>>(g, A, a_stride, nvec, h, w, spc, partial);
  else
    update_dot_kernel<false><<<grid, 256, 0, s>>>(g, A, a_stride, nvec, h, w, spc, partial);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_axpby(int prec, geom g, const double2* a, const void* x, const double2* b, void* y,
                         cudaStream_t s) {
  dim3 grid = site_grid(g, 256);
  if (prec == 0)
    axpby_kernel<double2><<<grid, 256, 0, s>>>(g, a, (const double2*)x, b, (double2*)y);
  else if (prec == 1)
    axpby_kernel<float2><<<grid, 256, 0, s>>>(g, a, (const float2*)x, b, (float2*)y);
  else
    axpby_kernel<__nv_bfloat162><<<grid, 256, 0, s>>>(g, a, (const __nv_bfloat162*)x, b, (__nv_bfloat162*)y);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_gamma(int prec, geom g, int theta, const void* src, void* dst, cudaStream_t s) {
  dim3 grid = site_grid(g, 256);
  if (prec == 0)
    gamma_kernel<double2><<<grid, 256, 0, s>>>(g, theta, (const double2*)src, (double2*)dst);
  else if (prec == 1)
    gamma_kernel<float2><<<grid, 256, 0, s>>>(g, theta, (const float2*)src, (float2*)dst);
  else
    gamma_kernel<__nv_bfloat162><<<grid, 256, 0, s>>>(g, theta, (const __nv_bfloat162*)src, (__nv_bfloat162*)dst);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_bilinear_codes(int prec, geom g, const uint32_t* codes, int theta, const void* x, int spc,
                                  double2* partial, cudaStream_t s) {
  dim3 grid((g.V + spc - 1) / spc, g.nrb);
  if (prec == 0)
    bilinear_codes_kernel<double2><<<grid, 256, 0, s>>>(g, codes, theta, (const double2*)x, spc, partial);
  else if (prec == 1)
    bilinear_codes_kernel<float2><<<grid, 256, 0, s>>>(g, codes, theta, (const float2*)x, spc, partial);
  else
    bilinear_codes_kernel<__nv_bfloat162><<<grid, 256, 0, s>>>(g, codes, theta, (const __nv_bfloat162*)x, spc,
                                                               partial);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_defl_proj(int prec, geom g, const uint32_t* codes, int theta, const void* Z, const void* U, int k,
                             int spc, double2* pa, double2* pb, cudaStream_t s) {
  dim3 grid((g.V + spc - 1) / spc, g.nrb);
  if (prec == 0)
    defl_proj_kernel<double2><<<grid, 256, 0, s>>>(g, codes, theta, (const double2*)Z, (const double2*)U, k, spc, pa,
                                                   pb);
  else
    defl_proj_kernel<float2><<<grid, 256, 0, s>>>(g, codes, theta, (const float2*)Z, (const float2*)U, k, spc, pa,
                                                  pb);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_vec_proj(int prec, geom g, const double2* Vv, int k, const void* f, int spc, double2* partial,
                            cudaStream_t s) {
  dim3 grid((g.V + spc - 1) / spc, g.nrb);
  if (prec == 0)
    vec_proj_kernel<double2><<<grid, 256, 0, s>>>(g, Vv, k, (const double2*)f, spc, partial);
  else
    vec_proj_kernel<float2><<<grid, 256, 0, s>>>(g, Vv, k, (const float2*)f, spc, partial);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_vec_update(int prec, geom g, const double2* Vv, int k, const double2* coef, void* f,
                              cudaStream_t s) {
  dim3 grid = site_grid(g, 256);
  if (prec == 0)
    vec_update_kernel<double2><<<grid, 256, 0, s>>>(g, Vv, k, coef, (double2*)f);
  else
    vec_update_kernel<float2><<<grid, 256, 0, s>>>(g, Vv, k, coef, (float2*)f);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_vec_proj32(int prec, geom g, const float2* Vv, int k, const void* f, int spc, double2* partial,
                              cudaStream_t s) {
  dim3 grid((g.V + spc - 1) / spc, g.nrb);
  if (prec == 0)
    vec_proj32_kernel<double2><<<grid, 256, 0, s>>>(g, Vv, k, (const double2*)f, spc, partial);
  else
    vec_proj32_kernel<float2><<<grid, 256, 0, s>>>(g, Vv, k, (const float2*)f, spc, partial);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_vec_update32(int prec, geom g, const float2* Vv, int k, const double2* coef, void* f,
                                cudaStream_t s) {
  dim3 grid = site_grid(g, 256);
  const size_t sm = size_t(k) * g.R * sizeof(float2);
  if (sm > 48 * 1024) return cudaErrorInvalidValue;
  if (prec == 0)
    vec_update32_kernel<double2><<<grid, 256, sm, s>>>(g, Vv, k, coef, (double2*)f);
  else
    vec_update32_kernel<float2><<<grid, 256, sm, s>>>(g, Vv, k, coef, (float2*)f);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_add2(const double2* a, const double2* b, double2* out, int n, cudaStream_t s) {
  add2_kernel<<<(n + 127) / 128, 128, 0, s>>>(a, b, out, n);
  count_launch();
  return cudaGetLastError();
}

}  // namespace mmc
