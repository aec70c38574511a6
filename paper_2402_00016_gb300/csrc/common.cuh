// Device-side types and helpers shared by the library's kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mmc {

// Flags of the fused step kernel (see step_params).
enum StepFlags : int {
  SF_HOP = 1,        // compute the Wilson hop D of `in`
  SF_WRITE = 2,      // write `out`
  SF_AUX = 4,        // add g * aux
  SF_YACC = 8,       // y += w_in * in + w_out * out (accumulator field)
  SF_BIL_CODES = 16, // bilinear with Z(4) noise given by packed codes
  SF_BIL_LEFT = 32,  // bilinear with an explicit left field
  SF_BIL_OUT = 64,   // bilinear also of `out` (weight w_out)
  SF_DAGGER = 128,   // use M^+ (gamma_mu signs flipped)
  SF_PAIRED = 256    // fields in the paired-component layout (fourth form, FP32, 8-rhs blocks)
};

// Per-step parameters.  Fields use the blocked layout [rb][site][c][R]; with SF_PAIRED
// the components of a site pair up per rhs: [rb][site][c/2][R][c%2].
struct step_params {
  const void* in;
  void* out;
  const void* aux;
  void* y;                 // accumulator: double2 (F64) or float2 (F32, BF16)
  const uint32_t* codes;   // packed Z(4) codes [rb][site][R]
  const void* left;        // explicit left field (same storage as in)
  const double2* coef;     // [5][npad]: a, b, g, w_in, w_out (complex)
  double2* partial;        // [nbx][npad] bilinear partial sums (FP64)
  const void* links;       // F64: double2 [site][mu][9]; F32: float2 [site][mu][10]
  const int* rb_len;       // optional: steps per rhs block; blocks with step >= len exit
  const int* nbr;          // neighbour table [site][8]: x+mu (mu = 0..3), then x-mu
  const int* order;        // optional traversal order of the sites (4D blocks); null: lexicographic
  int step;
  int V, R, logL, npad, spc;  // sites, rhs block, log2(lanes per site), padded rhs, sites per CTA
  int Lx, Ly, Lz, Lt;
  int tap;                 // antiperiodic time
  int theta;               // 0: 1, 1: gamma_4, 2: gamma_5
  int flags;
  int* err;                // device flag: set by a kernel whose bounded wait gave up (staged form)
  long long wait_iters;    // bound of each mbarrier wait of the staged form (0: the default)
  int stall_test;          // fault injection: the staged form's producer issues no copies
  int hint;                // bit 0: store the result with an L2 evict-first policy (fourth form)
  const uint32_t* salt;    // non-null: BF16 results stochastically rounded, stream key from *salt and step
};

template <typename T>
struct cx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ cx<T> cmake(T r, T i) {
  cx<T> c;
  c.re = r;
  c.im = i;
  return c;
}

}  // namespace mmc
