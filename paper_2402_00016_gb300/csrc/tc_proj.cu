// Deflation projections of a Monte Carlo level (Sec. 7) on the 5th-generation
// tensor cores: for noise vectors eta_r and deflation vectors z_i, u_i
//     a[i][r] = eta_r^H Theta z_i,   b[i][r] = u_i^H eta_r.
// Written as one real BF16 GEMM with FP32 accumulation, P = A B^T:
//   A rows (M): per noise r two rows, eta~_r = (re, im) interleaved along K and
//               eta^_r = (im, -re); generated from the Z(4) codes in shared
//               memory (entries 0, +-1: exact in BF16);
//   B rows (N = 256): BF16 copies of Theta z_i (rows 0..127) and u_i (128..255),
//               K-major, K = 2 x 12 V real components (zero padded);
//   then a_re = P[2r][i], a_im = -P[2r+1][i], b_re = P[2r][128+i], b_im = P[2r+1][128+i].
// The exact correction sum_i c_i u_i^H Theta z_i is taken from the same BF16
// copies (tc_bf16_pair_dots), so the deflated estimator stays unbiased.
//
// One CTA (128 threads, 4 warps) owns an M tile of 128 rows (64 noises) and a
// K range (split K across SMs); its 128 x 256 FP32 accumulator lives in TMEM.
// Per K stage (64 BF16 = 128 B per row) the B tile arrives by TMA
// (cp.async.bulk.tensor, 128-byte swizzle, issued by thread 0 three stages ahead
// onto the stage's full barrier), the threads write the A tile from the codes
// (prefetched one stage ahead) in the same canonical K-major swizzled layout,
// fence the async proxy, and thread 0 issues four tcgen05.mma (K = 16 each) and
// a tcgen05.commit onto the stage's MMA barrier.  Three A and five B buffers
// rotate; every mbarrier wait is bounded and sets an error flag instead of hanging.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace mmc {
namespace {

constexpr int kTM = 128;      // M tile (rows of A = 2 x 64 noises)
constexpr int kTN = 256;      // N (rows of B: 128 Theta z, 128 u)
constexpr int kTK = 64;       // K per stage (128 bytes of BF16 per row)
constexpr int kAStages = 3;  // A tiles (built by the threads)
constexpr int kBStages = 5;  // B tiles (TMA), also the MMA barriers
constexpr int kATile = kTM * kTK * 2;   // 16 KB
constexpr int kBTile = kTN * kTK * 2;   // 32 KB
constexpr long long kWaitLimit = 1ll << 20;  // bounded spin (about a second)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFFu) >> 4);          // start address
  d |= uint64_t(1) << 16;                          // leading byte offset (unused for this layout)
  d |= uint64_t(1024 >> 4) << 32;                  // stride byte offset: 8 rows x 128 B
  d |= uint64_t(1) << 46;                          // descriptor version
  d |= uint64_t(2) << 61;                          // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M = 128, N = 256.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(kTN >> 3) << 17) |
                            (uint32_t(kTM >> 4) << 24);

// Byte offset of the 16-byte chunk j of row m in a K-major 128B-swizzled tile.
__device__ __forceinline__ uint32_t sw_off(int m, int j) {
  return uint32_t((m >> 3) * 1024 + (m & 7) * 128 + ((j ^ (m & 7)) << 4));
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (long long i = 0; i < kWaitLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ uint32_t bf16pair(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t addr, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}

// B stage: the 256 x 64 BF16 box at K offset kx of the [256][Kp] copy, by the tensor map
// (128-byte swizzle: the canonical K-major layout the MMA descriptors expect).
__device__ __forceinline__ void tma_load_b(uint32_t dst, const CUtensorMap* map, int kx, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(kx), "r"(0), "r"(mbar)
      : "memory");
}

// The codes of the (at most four) sites that the 32 complex components of K stage ks
// touch, for this thread's noise row; 0 outside the lattice or the batch.
__device__ __forceinline__ void stage_codes(const uint32_t* codes, const geom& g, long long ks, bool live_row, int rb,
                                            int rr, uint32_t (&cd)[4]) {
  const int comp0 = int(ks * (kTK / 2));
  const int site0 = comp0 / 12;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int st = site0 + t;
    cd[t] = (live_row && st < g.V) ? (__ldg(codes + ((size_t)rb * g.V + st) * g.R + rr) & 0xFFFFFFu) : 0u;
  }
}

__global__ void __launch_bounds__(128, 1)
    tc_proj_kernel(const __grid_constant__ CUtensorMap tmap_b, geom g, const uint32_t* __restrict__ codes,
                   long long Kp, int kstages_per_split, float* __restrict__ partial, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // carve 1024-aligned stage buffers
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  unsigned char* sbase = smem_raw + (base - smem_u32(smem_raw));
  unsigned char* A_s = sbase;                                 // kAStages x 16 KB
  unsigned char* B_s = sbase + kAStages * kATile;             // kBStages x 32 KB
  uint64_t* mbar = reinterpret_cast<uint64_t*>(B_s + kBStages * kBTile);  // MMAs of a stage done
  uint64_t* fullb = mbar + kBStages;                                     // B of a stage landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fullb + kBStages);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int mtile = blockIdx.x, split = blockIdx.y;
  const long long ks0 = (long long)split * kstages_per_split;
  const long long nks_total = Kp / kTK;
  const long long ks1 = min(ks0 + kstages_per_split, nks_total);
  const long long n_it = ks1 > ks0 ? ks1 - ks0 : 0;
  const int n12v = 12 * g.V;  // complex components of a noise vector (K / 2 without padding)

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kBStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fullb[s])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // this thread's A row: noise r, variant v (0: eta~, 1: eta^)
  const int m = tid;
  const int r = mtile * (kTM / 2) + (m >> 1);
  const int v = m & 1;
  const bool live_row = r < g.npad;
  const int rb = live_row ? r / g.R : 0, rr = live_row ? r % g.R : 0;

  // Schedule (thread 0): at stage j, wait for the MMAs of stage j - 2, then issue B(j + 3).
  // B(j + 3) goes to the buffer last read by the MMAs of stage j + 3 - kBStages = j - 2; the
  // A tile of stage j + 1 to the buffer last read by stage j + 1 - kAStages = j - 2, and the
  // threads write it after stage j's barrier, which follows that wait.  The MMAs of stage
  // j - 1 stay in flight while stage j's A tile is built.
  constexpr int kPre = 3;
  static_assert(kPre + 2 == kBStages && kAStages == 3, "the schedule above");
  long long issued = 0;       // B stages issued (thread 0)
  long long mma_waited = -1;  // last stage whose MMAs thread 0 has seen complete
  if (tid == 0) {
    for (; issued < n_it && issued < kPre; ++issued) {
      const int s = int(issued);
      mbar_expect_tx(smem_u32(&fullb[s]), uint32_t(kBTile));
      tma_load_b(smem_u32(B_s + s * kBTile), &tmap_b, int((ks0 + issued) * kTK), smem_u32(&fullb[s]));
    }
  }
  uint32_t cd[4];
  if (n_it > 0) stage_codes(codes, g, ks0, live_row, rb, rr, cd);
  bool failed = false;
  long long it = 0;
  for (; it < n_it; ++it) {
    const int sa = int(it % kAStages), sb = int(it % kBStages);
    int bad = 0;
    if (tid == 0) {
      if (it >= 2) {
        const long long prev = it - 2;
        bad = !mbar_wait(smem_u32(&mbar[prev % kBStages]), uint32_t((prev / kBStages) & 1));
        if (!bad) mma_waited = prev;
      }
      if (!bad && issued < n_it) {
        const int s2 = int(issued % kBStages);
        mbar_expect_tx(smem_u32(&fullb[s2]), uint32_t(kBTile));
        tma_load_b(smem_u32(B_s + s2 * kBTile), &tmap_b, int((ks0 + issued) * kTK), smem_u32(&fullb[s2]));
        ++issued;
      }
    }
    // ---- A tile row m: 64 K entries (32 complex components) from the Z(4) codes
    {
      const long long ks = ks0 + it;
      const int comp0 = int(ks * (kTK / 2));
      const int c0 = comp0 - 12 * (comp0 / 12);
      // the 2-bit codes of the four sites as one stream (site t at bit 24 t), then the 64
      // bits of this stage's 32 components from component c0 of the first site on
      const uint64_t lo = uint64_t(cd[0]) | (uint64_t(cd[1]) << 24) | (uint64_t(cd[2]) << 48);
      const uint64_t hi = uint64_t(cd[2] >> 16) | (uint64_t(cd[3]) << 8);
      const int sh = 2 * c0;
      const uint64_t wcodes = sh == 0 ? lo : ((lo >> sh) | (hi << (64 - sh)));
      const int nvalid = live_row ? min(32, n12v - comp0) : 0;  // components inside the field
      const uint32_t rot = v == 0 ? 0u : 3u;  // eta^ = (im, -re): the code turned by -1 quarter
      uint32_t w[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        // code k: i^k as a BF16 pair (re, im): k even -> (+-1, 0), k odd -> (0, +-1)
        const uint32_t k = (uint32_t(wcodes >> (2 * q)) + rot) & 3u;
        const uint32_t mag = 0x3F80u | ((k & 2u) << 14);  // BF16 1.0, sign bit for k >= 2
        const uint32_t val = mag << ((k & 1u) << 4);
        w[q] = q < nvalid ? val : 0u;
      }
      if (it + 1 < n_it) stage_codes(codes, g, ks + 1, live_row, rb, rr, cd);  // in flight during the MMAs
      unsigned char* At = A_s + sa * kATile;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t a = smem_u32(At) + sw_off(m, j);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(w[4 * j]), "r"(w[4 * j + 1]),
                     "r"(w[4 * j + 2]), "r"(w[4 * j + 3])
                     : "memory");
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0 && !bad) bad = !mbar_wait(smem_u32(&fullb[sb]), uint32_t((it / kBStages) & 1));  // B landed
    if (__syncthreads_or(bad)) {  // the same decision in every thread
      failed = true;
      break;
    }
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t ad = desc_sw128(smem_u32(A_s + sa * kATile));
      const uint64_t bd = desc_sw128(smem_u32(B_s + sb * kBTile));
#pragma unroll
      for (int kk = 0; kk < kTK / 16; ++kk) {
        const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
        // K step of 16 BF16 = 32 bytes inside the swizzled 128-byte row
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad + uint64_t(2 * kk)), "l"(bd + uint64_t(2 * kk)), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[sb]))
                   : "memory");
    }
  }
  // Drain, each wait bounded: the MMAs of the stages thread 0 has not yet seen complete, and
  // (after a failure) the B copies issued for stages that were never consumed.  A copy that
  // is still in flight when the CTA exits could land in the next CTA's shared memory: that
  // case reports 2 and the host retires the context.
  int drain = 0;
  if (tid == 0) {
    for (long long j = mma_waited + 1; j < it; ++j)
      if (!mbar_wait(smem_u32(&mbar[j % kBStages]), uint32_t((j / kBStages) & 1))) drain = 1;
    for (long long j = it; j < issued; ++j)
      if (!mbar_wait(smem_u32(&fullb[j % kBStages]), uint32_t((j / kBStages) & 1))) drain = 2;
  }
  if (__syncthreads_or(drain)) failed = true;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (failed) {
    if (tid == 0) atomicMax(err, drain == 2 ? 2 : 1);
  } else if (it > 0) {
    // epilogue: warp w reads TMEM lanes 32w..32w+31 (rows of the tile), 256 columns
    const int row = warp * 32 + (tid & 31);
    float* dst = partial + ((size_t)split * gridDim.x * kTM + (size_t)mtile * kTM + row) * kTN;
#pragma unroll 1
    for (int c0 = 0; c0 < kTN; c0 += 32) {
      uint32_t x[32];
      const uint32_t ta = tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), "=r"(x[6]), "=r"(x[7]),
            "=r"(x[8]), "=r"(x[9]), "=r"(x[10]), "=r"(x[11]), "=r"(x[12]), "=r"(x[13]), "=r"(x[14]), "=r"(x[15]),
            "=r"(x[16]), "=r"(x[17]), "=r"(x[18]), "=r"(x[19]), "=r"(x[20]), "=r"(x[21]), "=r"(x[22]),
            "=r"(x[23]), "=r"(x[24]), "=r"(x[25]), "=r"(x[26]), "=r"(x[27]), "=r"(x[28]), "=r"(x[29]),
            "=r"(x[30]), "=r"(x[31])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int q = 0; q < 32; q += 4)
        *reinterpret_cast<float4*>(dst + c0 + q) =
            make_float4(__uint_as_float(x[q]), __uint_as_float(x[q + 1]), __uint_as_float(x[q + 2]),
                        __uint_as_float(x[q + 3]));
    }
  } else {
    // empty K range: zero contribution
    const int row = warp * 32 + (tid & 31);
    float* dst = partial + ((size_t)split * gridDim.x * kTM + (size_t)mtile * kTM + row) * kTN;
    for (int c0 = 0; c0 < kTN; ++c0) dst[c0] = 0.f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTN) : "memory");
  }
}

// out[m][n] = sum over splits of partial[split][m][n] (FP64), m < Mtot.
__global__ void tc_reduce_kernel(const float* __restrict__ partial, int nsplit, long long Mtot, double* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Mtot * kTN) return;
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += partial[(size_t)k * Mtot * kTN + i];
  out[i] = s;
}

// BF16 copy of deflation vectors: rows 0..k-1 = Theta z_i, 128..128+k-1 = u_i, interleaved
// (re, im) along K = 24 V (zero padded to Kp); the other rows zero.
__global__ void tc_pack_eig_kernel(int V, int k, long long Kp, int theta, const float2* __restrict__ Z,
                                   const float2* __restrict__ U, __nv_bfloat16* __restrict__ B) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // over 256 x Kp/2 complex slots
  const long long half = Kp / 2;
  if (idx >= 256 * half) return;
  const int n = int(idx / half);
  const long long comp = idx % half;
  float re = 0.f, im = 0.f;
  const long long n12 = 12ll * V;
  if (comp < n12) {
    if (n < 128 && n < k) {
      const int site = int(comp / 12), c = int(comp % 12);
      const int src = (theta == 1) ? (c + 6) % 12 : c;
      const float sg = (theta == 2 && c >= 6) ? -1.f : 1.f;
      const float2 z = Z[(size_t)n * n12 + (size_t)site * 12 + src];
      re = sg * z.x;
      im = sg * z.y;
    } else if (n >= 128 && n - 128 < k) {
      const float2 u = U[(size_t)(n - 128) * n12 + comp];
      re = u.x;
      im = u.y;
    }
  }
  __nv_bfloat162 v = __floats2bfloat162_rn(re, im);
  *reinterpret_cast<__nv_bfloat162*>(B + (size_t)n * Kp + 2 * comp) = v;
}

// d[i] = sum conj(u_i) (Theta z_i) from the BF16 copy (rows i and 128 + i), FP64 sums.
__global__ void tc_pair_dot_kernel(long long Kp, int k, const __nv_bfloat16* __restrict__ B, double2* __restrict__ d) {
  __shared__ double2 sh[256];
  const int i = blockIdx.x;
  if (i >= k) return;
  const __nv_bfloat162* z = reinterpret_cast<const __nv_bfloat162*>(B + (size_t)i * Kp);
  const __nv_bfloat162* u = reinterpret_cast<const __nv_bfloat162*>(B + (size_t)(128 + i) * Kp);
  double re = 0, im = 0;
  for (long long q = threadIdx.x; q < Kp / 2; q += blockDim.x) {
    const float2 a = __bfloat1622float2(u[q]), b = __bfloat1622float2(z[q]);
    re += double(a.x) * b.x + double(a.y) * b.y;
    im += double(a.x) * b.y - double(a.y) * b.x;
  }
  sh[threadIdx.x] = make_double2(re, im);
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      sh[threadIdx.x].x += sh[threadIdx.x + off].x;
      sh[threadIdx.x].y += sh[threadIdx.x + off].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) d[i] = sh[0];
}

}  // namespace

size_t tc_proj_smem_bytes() { return size_t(kAStages) * kATile + size_t(kBStages) * kBTile + 1024 + 128; }

cudaError_t launch_tc_pack_eig(int V, int k, long long Kp, int theta, const float2* Z, const float2* U, void* B,
                               cudaStream_t s) {
  const long long n = 256 * (Kp / 2);
  tc_pack_eig_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(V, k, Kp, theta, Z, U, (__nv_bfloat16*)B);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_tc_pair_dots(long long Kp, int k, const void* B, double2* d, cudaStream_t s) {
  tc_pair_dot_kernel<<<k, 256, 0, s>>>(Kp, k, (const __nv_bfloat16*)B, d);
  count_launch();
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no link
// against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// P (2 npad_rows x 256, FP64) for the noise batch of geometry g; nsplit chosen by the caller.
cudaError_t launch_tc_proj(const geom& g, const uint32_t* codes, const void* B, long long Kp, int nsplit,
                           float* partial, double* P, int* err, cudaStream_t s) {
  const int mtiles = (2 * g.npad + kTM - 1) / kTM;
  const long long nks = Kp / kTK;
  const int per = int((nks + nsplit - 1) / nsplit);
  if (Kp % kTK != 0 || (reinterpret_cast<uintptr_t>(B) & 15) != 0 || (Kp + kTK) > (1ll << 31))
    return cudaErrorInvalidValue;
  // B: [256][Kp] BF16, K-major; boxes of 64 K x 256 rows, 128-byte swizzle.  Every box
  // starts at K = 64 ks: 128 bytes, so the x coordinate is 16-byte aligned.
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return cudaErrorNotSupported;
  CUtensorMap tmap;
  const cuuint64_t gdim[2] = {cuuint64_t(Kp), 256};
  const cuuint64_t gstride[1] = {cuuint64_t(Kp) * 2};
  const cuuint32_t box[2] = {kTK, kTN};
  const cuuint32_t estride[2] = {1, 1};
  if (encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(B), gdim, gstride, box, estride,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const size_t smem = tc_proj_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(tc_proj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  tc_proj_kernel<<<dim3(mtiles, nsplit), 128, smem, s>>>(tmap, g, codes, Kp, per, partial, err);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long Mtot = (long long)mtiles * kTM;
  tc_reduce_kernel<<<unsigned((Mtot * kTN + 255) / 256), 256, 0, s>>>(partial, nsplit, Mtot, P);
  count_launch();
  return cudaGetLastError();
}

}  // namespace mmc
