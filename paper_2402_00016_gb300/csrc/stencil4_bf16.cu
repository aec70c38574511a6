// Step kernel, fourth form (stencil4.cuh): BF16 storage, R = 8, 16, one rhs per lane.
#include "stencil4.cuh"

namespace mmc {
bool launch_step4_bf16(int R, int minb, const step_params& p, int n_rb, int nbx, cudaStream_t s, cudaError_t* err) {
  if (R == 16) return minb == 3 ? sten4::launch4<__nv_bfloat162, 16, 3>(p, n_rb, nbx, s, err)
                                : sten4::launch4<__nv_bfloat162, 16, 4>(p, n_rb, nbx, s, err);
  if (R == 8) return minb == 3 ? sten4::launch4<__nv_bfloat162, 8, 3>(p, n_rb, nbx, s, err)
                               : sten4::launch4<__nv_bfloat162, 8, 4>(p, n_rb, nbx, s, err);
  return false;
}
}  // namespace mmc
