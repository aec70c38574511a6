// Step kernel v2 instantiations for FP32 storage (R = 8, 16; one or two rhs per lane).
#include "stencil2.cuh"

namespace mmc {
bool launch_step2_f32(int R, int rpt, int minb, const step_params& p, int n_rb, cudaStream_t s, cudaError_t* err) {
  if (R == 16) {
    if (rpt == 2) return sten2::launch2<float2, 16, 2, 3>(p, n_rb, s, err);
    return minb >= 6 ? sten2::launch2<float2, 16, 1, 6>(p, n_rb, s, err) : sten2::launch2<float2, 16, 1, 4>(p, n_rb, s, err);
  }
  if (R == 8) {
    if (rpt == 2) return sten2::launch2<float2, 8, 2, 3>(p, n_rb, s, err);
    return minb >= 6 ? sten2::launch2<float2, 8, 1, 6>(p, n_rb, s, err) : sten2::launch2<float2, 8, 1, 4>(p, n_rb, s, err);
  }
  return false;
}
}  // namespace mmc
