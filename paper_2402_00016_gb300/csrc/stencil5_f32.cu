// Step kernel, fifth form (stencil5.cuh): FP32 storage, R = 8, 16, one rhs per lane,
// pipeline depth 3 or 4 stages.
#include "stencil5.cuh"

namespace mmc {
bool launch_step5_f32(int R, int depth, const step_params& p, int n_rb, int nbx, cudaStream_t s, cudaError_t* err) {
  if (R == 16) return depth == 3 ? sten5::launch5<float2, 16, 4, 3>(p, n_rb, nbx, s, err)
                                 : sten5::launch5<float2, 16, 4, 4>(p, n_rb, nbx, s, err);
  if (R == 8) return depth == 3 ? sten5::launch5<float2, 8, 4, 3>(p, n_rb, nbx, s, err)
                                : sten5::launch5<float2, 8, 4, 4>(p, n_rb, nbx, s, err);
  return false;
}
}  // namespace mmc
