// Step kernel, staged form (stencil3.cuh): FP32 and BF16 storage, R = 8, 16.
#include <algorithm>

#include "stencil3.cuh"

namespace mmc {
bool launch_step3(int prec, int R, int rpt, int nbx, int ns, const step_params& p, int n_rb, cudaStream_t s,
                  cudaError_t* err) {
  if (prec == 1) {
    if (R == 16) return rpt == 2 ? sten3::launch3<float2, 16, 2>(p, n_rb, nbx, ns, s, err)
                                 : sten3::launch3<float2, 16, 1>(p, n_rb, nbx, ns, s, err);
    if (R == 8) return rpt == 2 ? sten3::launch3<float2, 8, 2>(p, n_rb, nbx, ns, s, err)
                                : sten3::launch3<float2, 8, 1>(p, n_rb, nbx, ns, s, err);
  } else if (prec == 2) {
    if (R == 16) return rpt == 2 ? sten3::launch3<__nv_bfloat162, 16, 2>(p, n_rb, nbx, ns, s, err)
                                 : sten3::launch3<__nv_bfloat162, 16, 1>(p, n_rb, nbx, ns, s, err);
    if (R == 8) return rpt == 2 ? sten3::launch3<__nv_bfloat162, 8, 2>(p, n_rb, nbx, ns, s, err)
                                : sten3::launch3<__nv_bfloat162, 8, 1>(p, n_rb, nbx, ns, s, err);
  }
  return false;
}
}  // namespace mmc
