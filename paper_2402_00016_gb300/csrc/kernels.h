// Host-side declarations of the library's CUDA kernels (launch wrappers).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace mmc {

// Geometry of a blocked field batch: [rb][site][c][R], rb < nrb, npad = nrb * R.
struct geom {
  int V, R, nrb, npad;
};

// Number of kernels the library has launched in this process (every launch_* call).
long long launch_count();
void count_launch(int n = 1);

// Fused stencil step (stencil.cu).  prec: 0 F64, 1 F32, 2 BF16; rpt: rhs per lane;
// minb: minimum resident CTAs per SM asked of the compiler (caps registers).
cudaError_t launch_step(int prec, int rpt, int minb, const step_params& p, int n_rb, cudaStream_t s);

// Step kernel v2 (stencil2_*.cu): compile-time rhs block R (8 or 16) and epilogue
// mode; returns false (nothing launched) when the flags or R need step_kernel.
// minb (RPT = 1 only): 6 caps registers at 80 (24 warps per SM), else 128 (16 warps).
bool launch_step2_f32(int R, int rpt, int minb, const step_params& p, int n_rb, cudaStream_t s, cudaError_t* err);
bool launch_step2_bf16(int R, int rpt, int minb, const step_params& p, int n_rb, cudaStream_t s, cudaError_t* err);
// Fourth form (stencil4.cuh): persistent grid over (rhs block, site pass) items with a
// compact front, loads of the next hop issued before the current hop's products; one
// rhs per lane, R = 8 or 16; minb 3 (168 registers), 4 (128) or 5 (128, the links of
// each pass staged in shared memory).  nbx: rows of the
// bilinear partials.  Returns false when the flags need another form.
bool launch_step4_f32(int R, int minb, const step_params& p, int n_rb, int nbx, cudaStream_t s, cudaError_t* err);
bool launch_step4_bf16(int R, int minb, const step_params& p, int n_rb, int nbx, cudaStream_t s, cudaError_t* err);
// Fifth form (stencil5.cuh): as the fourth, with the hops' operands staged in shared
// memory by per-lane asynchronous copies `depth` stages ahead (FP32: 3 or 4, BF16: 4
// or 6); one rhs per lane, R = 8 or 16, 128 registers.  Returns false when the flags
// or the operands' alignment need another form.
bool launch_step5_f32(int R, int depth, const step_params& p, int n_rb, int nbx, cudaStream_t s, cudaError_t* err);
bool launch_step5_bf16(int R, int depth, const step_params& p, int n_rb, int nbx, cudaStream_t s, cudaError_t* err);
// Staged form (rows by bulk asynchronous copies, stencil3.cuh) for FP32 (prec 1) and BF16
// (prec 2) storage, R = 8 or 16, rpt = 1 or 2 rhs per thread; nbx: rows of the bilinear
// partials (grid bound), ns: ring slots (0: as many as fit).  Returns false when the
// geometry or flags need another form.
bool launch_step3(int prec, int R, int rpt, int nbx, int ns, const step_params& p, int n_rb, cudaStream_t s,
                  cudaError_t* err);

// Z(4) noise (Sec. 1) into a field of precision prec and/or packed codes.
// ids[r] = (level, noise index) for rhs r (npad entries, device); entries with
// level == 0xffffffff give zero vectors (padding).
cudaError_t launch_noise(int prec, geom g, const uint2* ids, uint32_t tag, uint64_t seed, void* field,
                         uint32_t* codes, cudaStream_t s);

// Probe vectors (Sec. 6 probing): rhs r has unit entries at component comp[r] on every
// site of colour col[r] (colour table per site, n entries); value 0 elsewhere.
cudaError_t launch_probe(int prec, geom g, const int* site_colour, const int2* probe, void* field,
                         cudaStream_t s);

// Canonical complex128 [rhs][site][12] (device) <-> blocked field of precision prec.
cudaError_t launch_pack(int prec, geom g, int nrhs, const double2* canon, void* field, cudaStream_t s);
cudaError_t launch_unpack(int prec, geom g, int nrhs, const void* field, double2* canon, cudaStream_t s);

// BF16 dst = FP32 src rounded stochastically (stream key from *salt, device memory).
cudaError_t launch_convert_sr(void* dst, const void* src, geom g, const uint32_t* salt, cudaStream_t s);
// *salt advances one step of its sequence (a fresh stochastic-rounding stream per chain).
cudaError_t launch_salt_advance(uint32_t* salt, cudaStream_t s);

// dst (precision pd) = src (precision ps), same geometry.
cudaError_t launch_convert(int pd, void* dst, int ps, const void* src, geom g, cudaStream_t s);
// FP32 field dst = src moved into (to_paired = 1) or out of (0) the paired-component
// layout of SF_PAIRED; dst and src distinct.
cudaError_t launch_pair_layout(void* dst, const void* src, geom g, int to_paired, cudaStream_t s);

// Per-rhs partial dots for a set of basis fields: partial[bx][i][npad] =
// sum over the CTA's sites of conj(A_i) . w (optionally with Theta on w).
// prec 0 (F64, double2 fields) or 1 (F32, float2 fields); spc sites per CTA.
cudaError_t launch_multidot(int prec, geom g, const void* A, size_t a_stride, int nvec, const void* w,
                            int theta, int spc, double2* partial, cudaStream_t s);
// out[i][npad] = sum_bx partial[bx][i][npad] (+ out if accumulate).
cudaError_t launch_reduce(const double2* partial, int nbx, int nvec, int npad, double2* out, int accumulate,
                          cudaStream_t s);
// w -= sum_i A_i * h[i][r] (h device, double2 [nvec][npad]).
cudaError_t launch_basis_update(int prec, geom g, const void* A, size_t a_stride, int nvec, const double2* h,
                                void* w, cudaStream_t s);
// flag |= 1 when a FP64 link's third row is not the (phase-signed) conjugate cross
// product of its first two to 1e-10.
cudaError_t launch_su3_rows_check(const double2* links, int V, int slice, int Lt, int tap, int* flag,
                                  cudaStream_t s);
// FP32 fields: w <- w - sum_i h_i A_i (nvec <= 8), then per-CTA partials (rows of spc
// sites, as launch_multidot) of A_i^H w (norm false, nvec rows) or of w^H w (norm true).
cudaError_t launch_update_dot(geom g, const float2* A, size_t a_stride, int nvec, const double2* h, float2* w,
                              bool norm, int spc, double2* partial, cudaStream_t s);
// dst = scale(r) * src with scale = 1 / sqrt(nrm2[r].x), zero if nrm2 == 0.
cudaError_t launch_normalise(int prec, geom g, const void* src, const double2* nrm2, void* dst, cudaStream_t s);
// y = a[r] * x + b[r] * y (complex per-rhs coefficients on the device).
cudaError_t launch_axpby(int prec, geom g, const double2* a, const void* x, const double2* b, void* y,
                         cudaStream_t s);
// Apply gamma_5 (theta = 2) or gamma_4 (theta = 1) site-locally: dst = Theta src.
cudaError_t launch_gamma(int prec, geom g, int theta, const void* src, void* dst, cudaStream_t s);
// Bilinear partials of Z(4) codes against a field: partial[bx][npad] += sum conj(eta) Theta x.
cudaError_t launch_bilinear_codes(int prec, geom g, const uint32_t* codes, int theta, const void* x, int spc,
                                  double2* partial, cudaStream_t s);

// Deflation projections (Sec. 7) of noise codes against k single-vector fields (prec 0:
// FP64 double2, 1: FP32 float2): a[i][r] = sum conj(eta_r) (Theta z_i),
// b[i][r] = sum conj(u_i) eta_r  (partials per CTA).
cudaError_t launch_defl_proj(int prec, geom g, const uint32_t* codes, int theta, const void* Z, const void* U,
                             int k, int spc, double2* partial_a, double2* partial_b, cudaStream_t s);

// Projections of a batch field on k single-vector FP64 fields v_i and the matching
// update: partial[bx][i][npad] = sum conj(v_i) . f_r;  f_r += sum_i v_i coef[i][r].
cudaError_t launch_vec_proj(int prec, geom g, const double2* Vv, int k, const void* f, int spc, double2* partial,
                            cudaStream_t s);
cudaError_t launch_vec_update(int prec, geom g, const double2* Vv, int k, const double2* coef, void* f,
                              cudaStream_t s);

// FP32 forms of the two above (v_i FP32 copies, FP32 arithmetic, FP64 partials); the
// field keeps its own precision.  k * R * 8 bytes of coefficients must fit 48 KB.
cudaError_t launch_vec_proj32(int prec, geom g, const float2* Vv, int k, const void* f, int spc,
                              double2* partial, cudaStream_t s);
cudaError_t launch_vec_update32(int prec, geom g, const float2* Vv, int k, const double2* coef, void* f,
                                cudaStream_t s);

// Learned stencil network layers (net.cu).  Activations: blocked layout with 3*C
// components per site; links: the FP32 links of the context.
struct net_geom {
  int V, R, nrb, npad;
  int L[4];
  const void* links;
};
// out = layer(in) for (ci, co) in {(4,8), (8,8), (8,4), (4,4)}; W: 9 x co x ci complex, FP32
// (float2) or BF16 (two bfloat16); in and out FP32 or BF16 activations (FP32 weights only
// with FP32 activations); FP32 arithmetic.
cudaError_t launch_net_layer(const net_geom& g, int ci, int co, const void* in, bool in_bf16, const void* W,
                             bool w_bf16, void* out, bool out_bf16, cudaStream_t s);
// partial[b][9][co][ci] over b = rb * nbx + bx: sum delta conj(feature) (weight gradients);
// the layer input FP32 or BF16, delta FP32.
cudaError_t launch_net_wgrad(const net_geom& g, int ci, int co, const void* in, bool in_bf16, const float2* delta,
                             int spc, double2* partial, cudaStream_t s);

// Tensor-core deflation projections (tc_proj.cu): BF16 copy of [Theta z; u] (256 x Kp),
// the correction dots from that copy, and the projections P (FP64, rows 2 npad padded
// to 128, 256 columns) of a noise batch.
size_t tc_proj_smem_bytes();
cudaError_t launch_tc_pack_eig(int V, int k, long long Kp, int theta, const float2* Z, const float2* U, void* B,
                               cudaStream_t s);
cudaError_t launch_tc_pair_dots(long long Kp, int k, const void* B, double2* d, cudaStream_t s);
cudaError_t launch_tc_proj(const geom& g, const uint32_t* codes, const void* B, long long Kp, int nsplit,
                           float* partial, double* P, int* err, cudaStream_t s);

// Complex small-matrix kernels on the device for the Arnoldi bookkeeping.
// hcol[i] = h1[i] + h2[i] for i < n (per rhs), written into H column storage.
cudaError_t launch_add2(const double2* a, const double2* b, double2* out, int n, cudaStream_t s);

}  // namespace mmc
