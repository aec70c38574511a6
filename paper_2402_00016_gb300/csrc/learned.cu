// Host side of the learned gauge-covariant linear stencil network: creation,
// weights, application (inference), loss and weight gradients (training kernels
// of net.cu), the training loop (device forward/backward, host Adam) and the
// network's use as FGMRES preconditioner and as a Monte Carlo level operand.
// The method's paper has no learned part; the network approximates M^-1 of
// Sec. 1 and stays linear in its input, so a subtraction with it keeps the
// estimator of Eq. 2 unbiased.
#include <random>

#include "internal.h"

using namespace mmc::host;
using mmc::cd;
using mmc::geom;

namespace mmc {
namespace host {

bool is_net(const mmc_ctx* ctx, int h) {
  return h >= kNetBase && h - kNetBase < int(ctx->nets.size());
}

namespace {

int layer_offset(int l) {
  int off = 0;
  for (int k = 0; k < l; ++k) off += 9 * kNetCh[k] * kNetCh[k + 1];
  return off;
}

net_geom ngeom(const mmc_ctx* ctx, const geom& g) {
  net_geom n;
  n.V = g.V;
  n.R = g.R;
  n.nrb = g.nrb;
  n.npad = g.npad;
  for (int i = 0; i < 4; ++i) n.L[i] = ctx->dims[i];
  n.links = ctx->links32;
  return n;
}

// BF16 rounding of a weight (round to nearest even on the float value), on the host
float bf16_round(double v) {
  const __nv_bfloat16 b = __float2bfloat16_rn(float(v));
  return __bfloat162float(b);
}

int upload_net(mmc_ctx* ctx, Net& N) {
  std::vector<float2> h(kNetWeights);
  std::vector<__nv_bfloat162> hb(kNetWeights);
  for (int i = 0; i < kNetWeights; ++i) {
    h[i] = make_float2(float(N.w[i].real()), float(N.w[i].imag()));
    hb[i] = __floats2bfloat162_rn(float(N.w[i].real()), float(N.w[i].imag()));
  }
  if (!N.dw) CK(cudaMalloc(&N.dw, sizeof(float2) * kNetWeights));
  if (!N.dwb) CK(cudaMalloc(&N.dwb, sizeof(__nv_bfloat162) * kNetWeights));
  CK(cudaMemcpy(N.dw, h.data(), sizeof(float2) * kNetWeights, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(N.dwb, hb.data(), sizeof(__nv_bfloat162) * kNetWeights, cudaMemcpyHostToDevice));
  return MMC_OK;
}

// Adjoint weights of layer l (C_in x C_out blocks): W0^H, Wf[mu] <- Wb[mu]^H, Wb[mu] <- Wf[mu]^H
// (of the BF16-rounded weights for a BF16 network, the ones its forward pass uses).
std::vector<float2> adjoint_weights(const Net& N, int l) {
  const int ci = kNetCh[l], co = kNetCh[l + 1];
  const int off = layer_offset(l);
  std::vector<float2> a(size_t(9) * ci * co);
  for (int w = 0; w < 9; ++w) {
    const int src = (w == 0) ? 0 : (w <= 4 ? w + 4 : w - 4);
    for (int i = 0; i < ci; ++i)
      for (int o = 0; o < co; ++o) {
        cd v = std::conj(N.w[off + (size_t(src) * co + o) * ci + i]);
        if (N.bf16) v = cd(bf16_round(v.real()), bf16_round(v.imag()));
        a[(size_t(w) * ci + i) * co + o] = make_float2(float(v.real()), float(v.imag()));
      }
  }
  return a;
}

}  // namespace

// y = N x on FP32 fields (12 components per site) of nrhs vectors.  Activations
// a1, a2 (24 components) are context scratch; returned through *acts if given.
int net_apply(mmc_ctx* ctx, int h, const void* x, void* y, int nrhs, cudaStream_t s, void** acts) {
  Net& N = ctx->nets[h - kNetBase];
  const geom g = make_geom(ctx, nrhs);
  const net_geom ng = ngeom(ctx, g);
  const bool b = N.bf16;
  const size_t hid = size_t(g.npad) * g.V * 24 * (b ? sizeof(__nv_bfloat162) : sizeof(float2));
  void *a1, *a2;
  TRY(scratch(ctx, b ? "net_a1b" : "net_a1", hid, &a1));
  TRY(scratch(ctx, b ? "net_a2b" : "net_a2", hid, &a2));
  const void* W0 = b ? (const void*)(N.dwb + layer_offset(0)) : (const void*)(N.dw + layer_offset(0));
  const void* W1 = b ? (const void*)(N.dwb + layer_offset(1)) : (const void*)(N.dw + layer_offset(1));
  const void* W2 = b ? (const void*)(N.dwb + layer_offset(2)) : (const void*)(N.dw + layer_offset(2));
  CK(mmc::launch_net_layer(ng, 4, 8, x, false, W0, b, a1, b, s));
  CK(mmc::launch_net_layer(ng, 8, 8, a1, b, W1, b, a2, b, s));
  CK(mmc::launch_net_layer(ng, 8, 4, a2, b, W2, b, y, false, s));
  if (acts) {
    acts[0] = a1;
    acts[1] = a2;
  }
  return MMC_OK;
}

// Loss (1/B) sum_b ||N eta_b - x_b||^2 / ||x_b||^2 and gradients 2 dL/dconj(W) on one batch.
int net_loss_grad(mmc_ctx* ctx, int h, const void* eta, const void* xs, int nrhs, double* loss,
                  std::vector<cd>& grad, cudaStream_t s) {
  Net& N = ctx->nets[h - kNetBase];
  const geom g = make_geom(ctx, nrhs);
  const net_geom ng = ngeom(ctx, g);
  const size_t f32 = field_bytes(g, MMC_F32);
  const size_t hid = size_t(g.npad) * g.V * 24 * sizeof(float2);
  void *out, *d3, *d2, *d1, *aw, *part, *red;
  TRY(scratch(ctx, "net_out", f32, &out));
  TRY(scratch(ctx, "net_d3", f32, &d3));
  TRY(scratch(ctx, "net_d2", hid, &d2));
  TRY(scratch(ctx, "net_d1", hid, &d1));
  TRY(scratch(ctx, "net_aw", sizeof(float2) * 9 * 64, &aw));
  void* acts[2];
  TRY(net_apply(ctx, h, eta, out, nrhs, s, acts));
  // r = out - x ; norms
  std::vector<cd> one(g.npad, cd(1, 0)), mone(g.npad, cd(-1, 0));
  void *d1c, *dmc;
  TRY(scratch(ctx, "net_c1", g.npad * sizeof(double2), &d1c));
  TRY(scratch(ctx, "net_cm", g.npad * sizeof(double2), &dmc));
  {
    std::vector<double2> a(g.npad, make_double2(1, 0)), b(g.npad, make_double2(-1, 0));
    CK(cudaMemcpyAsync(d1c, a.data(), a.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dmc, b.data(), b.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  CK(mmc::launch_axpby(MMC_F32, g, (const double2*)dmc, xs, (const double2*)d1c, out, s));  // out <- out - x
  const int spc = 256, nbx = (g.V + spc - 1) / spc;
  TRY(scratch(ctx, "net_part", size_t(nbx) * g.npad * sizeof(double2), &part));
  TRY(scratch(ctx, "net_red", size_t(g.npad) * sizeof(double2) * 2, &red));
  std::vector<double2> rn(g.npad), xn(g.npad);
  CK(mmc::launch_multidot(MMC_F32, g, out, 0, 1, out, 0, spc, (double2*)part, s));
  CK(mmc::launch_reduce((double2*)part, nbx, 1, g.npad, (double2*)red, 0, s));
  CK(cudaMemcpyAsync(rn.data(), red, g.npad * sizeof(double2), cudaMemcpyDeviceToHost, s));
  CK(mmc::launch_multidot(MMC_F32, g, xs, 0, 1, xs, 0, spc, (double2*)part, s));
  CK(mmc::launch_reduce((double2*)part, nbx, 1, g.npad, (double2*)red + g.npad, 0, s));
  CK(cudaMemcpyAsync(xn.data(), (double2*)red + g.npad, g.npad * sizeof(double2), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double L = 0;
  std::vector<double2> sc(g.npad, make_double2(0, 0));
  for (int r = 0; r < nrhs; ++r) {
    if (!(xn[r].x > 0)) RET(MMC_ERR_ARG, "net loss: zero target vector");
    L += rn[r].x / xn[r].x;
    sc[r] = make_double2(2.0 / (double(nrhs) * xn[r].x), 0);
  }
  *loss = L / nrhs;
  void* dsc;
  TRY(scratch(ctx, "net_sc", g.npad * sizeof(double2), &dsc));
  CK(cudaMemcpyAsync(dsc, sc.data(), sc.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
  CK(mmc::launch_axpby(MMC_F32, g, (const double2*)dsc, out, nullptr, d3, s));  // delta3 = 2 r / (B ||x||^2)
  // weight gradients and backward data pass, last layer first
  grad.assign(kNetWeights, cd(0, 0));
  const int wspc = 256, wnbx = (g.V + wspc - 1) / wspc;
  const int nb_all = wnbx * g.nrb;
  TRY(scratch(ctx, "net_wpart", size_t(nb_all) * 9 * 64 * sizeof(double2), &part));
  const void* layer_in[3] = {eta, acts[0], acts[1]};
  const bool in_b[3] = {false, N.bf16, N.bf16};
  float2* deltas[3] = {(float2*)d1, (float2*)d2, (float2*)d3};
  for (int l = 2; l >= 0; --l) {
    const int ci = kNetCh[l], co = kNetCh[l + 1];
    const int nw = 9 * ci * co;
    CK(mmc::launch_net_wgrad(ng, ci, co, layer_in[l], in_b[l], deltas[l], wspc, (double2*)part, s));
    void* wred;
    TRY(scratch(ctx, "net_wred", size_t(nw) * sizeof(double2), &wred));
    // partials were written with stride 9*co*ci per block
    CK(mmc::launch_reduce((double2*)part, nb_all, nw, 1, (double2*)wred, 0, s));
    std::vector<double2> gw(nw);
    CK(cudaMemcpyAsync(gw.data(), wred, nw * sizeof(double2), cudaMemcpyDeviceToHost, s));
    if (l > 0) {
      std::vector<float2> aw_h = adjoint_weights(N, l);
      CK(cudaMemcpyAsync(aw, aw_h.data(), aw_h.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
      CK(mmc::launch_net_layer(ng, co, ci, deltas[l], false, aw, false, deltas[l - 1], false, s));
    }
    CK(cudaStreamSynchronize(s));
    const int off = layer_offset(l);
    for (int i = 0; i < nw; ++i) grad[off + i] = cd(gw[i].x, gw[i].y);
  }
  return MMC_OK;
}

}  // namespace host
}  // namespace mmc

extern "C" {

int mmc_net_create(mmc_ctx* ctx, const double* weights, uint64_t seed, int* handle) {
  TRY(check_ctx(ctx));
  if (!handle) return MMC_ERR_ARG;
  Net N;
  N.w.resize(kNetWeights);
  if (weights) {
    for (int i = 0; i < kNetWeights; ++i) N.w[i] = cd(weights[2 * i], weights[2 * i + 1]);
  } else {
    // near the channel-embedding identity, small seeded hop weights
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, 0.05);
    for (int l = 0; l < 3; ++l) {
      const int ci = kNetCh[l], co = kNetCh[l + 1], off = layer_offset(l);
      for (int w = 0; w < 9; ++w)
        for (int o = 0; o < co; ++o)
          for (int i = 0; i < ci; ++i) {
            cd v(nd(rng), nd(rng));
            if (w == 0 && o == i) v += 1.0;
            N.w[off + (size_t(w) * co + o) * ci + i] = v;
          }
    }
  }
  TRY(upload_net(ctx, N));
  ctx->nets.push_back(N);
  *handle = kNetBase + int(ctx->nets.size()) - 1;
  return MMC_OK;
}

int mmc_net_set_weights(mmc_ctx* ctx, int handle, const double* weights) {
  if (!ctx || !weights || !is_net(ctx, handle)) return MMC_ERR_ARG;
  Net& N = ctx->nets[handle - kNetBase];
  for (int i = 0; i < kNetWeights; ++i) N.w[i] = cd(weights[2 * i], weights[2 * i + 1]);
  return upload_net(ctx, N);
}

int mmc_net_get_weights(mmc_ctx* ctx, int handle, double* weights) {
  if (!ctx || !weights || !is_net(ctx, handle)) return MMC_ERR_ARG;
  const Net& N = ctx->nets[handle - kNetBase];
  for (int i = 0; i < kNetWeights; ++i) {
    weights[2 * i] = N.w[i].real();
    weights[2 * i + 1] = N.w[i].imag();
  }
  return MMC_OK;
}

int mmc_net_set_precision(mmc_ctx* ctx, int handle, int prec) {
  if (!ctx || !is_net(ctx, handle) || (prec != MMC_F32 && prec != MMC_BF16)) return MMC_ERR_ARG;
  ctx->nets[handle - kNetBase].bf16 = prec == MMC_BF16;
  return MMC_OK;
}

int mmc_net_apply(mmc_ctx* ctx, int handle, const void* x, void* y, int nrhs, void* stream) {
  TRY(check_ctx(ctx));
  if (!is_net(ctx, handle) || !x || !y || x == y || nrhs < 1) RET(MMC_ERR_ARG, "mmc_net_apply: bad argument");
  return net_apply(ctx, handle, x, y, nrhs, (cudaStream_t)stream, nullptr);
}

int mmc_net_loss_grad(mmc_ctx* ctx, int handle, const void* eta, const void* xs, int nrhs, double* loss,
                      double* grad) {
  TRY(check_ctx(ctx));
  if (!is_net(ctx, handle) || !eta || !xs || !loss || nrhs < 1) RET(MMC_ERR_ARG, "mmc_net_loss_grad: bad argument");
  std::vector<cd> g;
  TRY(net_loss_grad(ctx, handle, eta, xs, nrhs, loss, g, ctx->stream));
  if (grad)
    for (int i = 0; i < kNetWeights; ++i) {
      grad[2 * i] = g[i].real();
      grad[2 * i + 1] = g[i].imag();
    }
  return MMC_OK;
}

int mmc_net_train(mmc_ctx* ctx, int handle, const void* eta, const void* xs, int npairs, int batch, int iters,
                  double lr, double* loss_history) {
  TRY(check_ctx(ctx));
  if (!is_net(ctx, handle) || !eta || !xs || npairs < 1 || iters < 0 || !(lr > 0))
    RET(MMC_ERR_ARG, "mmc_net_train: bad argument");
  const geom gall = make_geom(ctx, npairs);
  if (batch < 1 || batch > npairs || (batch != npairs && (batch % gall.R || npairs % batch)))
    RET(MMC_ERR_ARG, "mmc_net_train: batch must divide npairs and be a multiple of the rhs block");
  Net& N = ctx->nets[handle - kNetBase];
  const size_t block_elems = size_t(gall.R) * ctx->V * 12;  // complex FP32 per rhs block
  const int nbatches = npairs / batch;
  std::vector<cd> m(kNetWeights, cd(0, 0));
  std::vector<double> v1(kNetWeights, 0.0), v2(kNetWeights, 0.0);
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  for (int it = 0; it < iters; ++it) {
    const int bi = it % nbatches;
    const size_t off = size_t(bi) * (batch / gall.R) * block_elems;
    const float2* e = reinterpret_cast<const float2*>(eta) + off;
    const float2* x = reinterpret_cast<const float2*>(xs) + off;
    double L;
    std::vector<cd> g;
    TRY(net_loss_grad(ctx, handle, e, x, batch, &L, g, ctx->stream));
    if (loss_history) loss_history[it] = L;
    if (!std::isfinite(L)) RET(MMC_ERR_NAN, "mmc_net_train: loss is not finite");
    const double c1 = 1 - std::pow(b1, it + 1), c2 = 1 - std::pow(b2, it + 1);
    for (int i = 0; i < kNetWeights; ++i) {
      m[i] = b1 * m[i] + (1 - b1) * g[i];
      v1[i] = b2 * v1[i] + (1 - b2) * g[i].real() * g[i].real();
      v2[i] = b2 * v2[i] + (1 - b2) * g[i].imag() * g[i].imag();
      const cd mh = m[i] / c1;
      N.w[i] -= lr * cd(mh.real() / (std::sqrt(v1[i] / c2) + eps), mh.imag() / (std::sqrt(v2[i] / c2) + eps));
    }
    TRY(upload_net(ctx, N));
  }
  return MMC_OK;
}

}  // extern "C"
