// Step kernel, fifth form (stencil5.cuh): BF16 storage, R = 8, 16, one rhs per lane,
// pipeline depth 4 or 6 stages.
#include "stencil5.cuh"

namespace mmc {
bool launch_step5_bf16(int R, int depth, const step_params& p, int n_rb, int nbx, cudaStream_t s, cudaError_t* err) {
  if (R == 16) return depth == 6 ? sten5::launch5<__nv_bfloat162, 16, 4, 6>(p, n_rb, nbx, s, err)
                                 : sten5::launch5<__nv_bfloat162, 16, 4, 4>(p, n_rb, nbx, s, err);
  if (R == 8) return depth == 6 ? sten5::launch5<__nv_bfloat162, 8, 4, 6>(p, n_rb, nbx, s, err)
                                : sten5::launch5<__nv_bfloat162, 8, 4, 4>(p, n_rb, nbx, s, err);
  return false;
}
}  // namespace mmc
