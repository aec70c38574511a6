// mmc_noise_noalloc: the Z(4) noise fill of mmc_noise without any device
// allocation.  mmc_noise keeps its per-vector (level, index) table in a buffer
// that the context allocates on first use; this variant keeps the table in a
// fixed static device array instead, for callers whose device memory is owned
// by someone else (a framework's caching allocator that holds the GPU's
// memory, a service with a fixed memory budget that forbids allocation once it
// is running).  The caller still passes the output field.
#include <mutex>
#include <vector>

#include "internal.h"

namespace {

// Largest padded batch the static table holds (32 KB per device, kept until exit).
constexpr int kNoallocMaxRhs = 4096;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint2 g_noise_ids[kNoallocMaxRhs];

// Device address of g_noise_ids per device, looked up once per device (under a
// std::call_once per device, so host threads making their first call on the same
// device at the same time do not race).  In host code the name g_noise_ids is only
// a host-side stand-in for the symbol, so the kernel must be given this address,
// never the name.
uint2* g_ids_addr[kMaxDevices] = {};
cudaError_t g_ids_err[kMaxDevices] = {};
std::once_flag g_ids_once[kMaxDevices];

}  // namespace

extern "C" int mmc_noise_noalloc(mmc_ctx* ctx, uint32_t level, uint32_t first, uint32_t tag, int nrhs, int prec,
                                 void* field, void* stream) {
  if (!ctx || !field || nrhs < 1 || prec < 0 || prec > 2) return MMC_ERR_ARG;
  const mmc::geom g = mmc::host::make_geom(ctx, nrhs);
  if (g.npad > kNoallocMaxRhs)
    RET(MMC_ERR_ARG, "mmc_noise_noalloc: at most " + std::to_string(kNoallocMaxRhs) +
                         " right-hand sides (padded to the rhs block); use mmc_noise for larger batches");
  if (ctx->device < 0 || ctx->device >= kMaxDevices) RET(MMC_ERR_ARG, "mmc_noise_noalloc: device index out of range");
  CK(cudaSetDevice(ctx->device));
  const int dev = ctx->device;
  std::call_once(g_ids_once[dev], [dev] {
    void* p = nullptr;
    g_ids_err[dev] = cudaGetSymbolAddress(&p, g_noise_ids);  // with device `dev` current
    if (g_ids_err[dev] == cudaSuccess) g_ids_addr[dev] = static_cast<uint2*>(p);
  });
  CK(g_ids_err[dev]);
  uint2* ids_dev = g_ids_addr[dev];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // every entry the kernel reads is rewritten here: nothing is left from an earlier call
  std::vector<uint2> ids(g.npad);
  for (int r = 0; r < g.npad; ++r) ids[r] = r < nrhs ? make_uint2(level, first + r) : make_uint2(0xffffffffu, 0u);
  CK(cudaMemcpyAsync(ids_dev, ids.data(), ids.size() * sizeof(uint2), cudaMemcpyHostToDevice, s));
  CK(mmc::launch_noise(prec, g, ids_dev, tag, ctx->seed, field, nullptr, s));
  CK(cudaStreamSynchronize(s));  // the table is shared by every call on this device
  return MMC_OK;
}
