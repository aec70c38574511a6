// Step kernel, fourth form (stencil4.cuh): FP32 storage, R = 8, 16, one rhs per lane.
#include "stencil4.cuh"

namespace mmc {
bool launch_step4_f32(int R, int minb, const step_params& p, int n_rb, int nbx, cudaStream_t s, cudaError_t* err) {
  // minb 3: 168 registers; 4: 128; 5: 128 with the links staged in shared memory; 6 (special
  // unitary links): 168 with each link's third row rebuilt from the first two.  The paired-
  // component layout (SF_PAIRED) exists for 8-rhs blocks at 168 registers (minb 3 or 6).
  if (p.flags & SF_PAIRED) {
    if (R != 8 || (minb != 3 && minb != 6)) return false;
    return minb == 6 ? sten4::launch4<float2, 8, 3, false, true, true>(p, n_rb, nbx, s, err)
                     : sten4::launch4<float2, 8, 3, false, false, true>(p, n_rb, nbx, s, err);
  }
  if (R == 16) return minb == 3 ? sten4::launch4<float2, 16, 3, false, false>(p, n_rb, nbx, s, err)
                     : minb == 6 ? sten4::launch4<float2, 16, 3, false, true>(p, n_rb, nbx, s, err)
                     : minb == 5 ? sten4::launch4<float2, 16, 4, true, false>(p, n_rb, nbx, s, err)
                                 : sten4::launch4<float2, 16, 4, false, false>(p, n_rb, nbx, s, err);
  if (R == 8) return minb == 3 ? sten4::launch4<float2, 8, 3, false, false>(p, n_rb, nbx, s, err)
                    : minb == 6 ? sten4::launch4<float2, 8, 3, false, true>(p, n_rb, nbx, s, err)
                    : minb == 5 ? sten4::launch4<float2, 8, 4, true, false>(p, n_rb, nbx, s, err)
                                : sten4::launch4<float2, 8, 4, false, false>(p, n_rb, nbx, s, err);
  return false;
}
}  // namespace mmc
