// Grid product with library-owned scratch: an entry point that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they need a product: real-time or
// embedded loops whose device-memory footprint is fixed before they start (an allocation there
// can stall or fail unpredictably), hosts that forbid cudaMalloc after start-up, and code that
// runs inside another runtime's memory pool that does not let third-party libraries grow it.
// aim_grid_product may grow its workspace with cudaMalloc the first time it sees a larger batch.
// This variant uses instead a fixed scratch array that lives in the library's device image:
// every GPU that loads the library holds it until the process exits, and every call shares it.
#include <mutex>

#include "aim_internal.h"
#include "gridtypes.cuh"

namespace aim {

bool profiling_active();

// Scratch for the m x P intermediate grid of the product (tiled, one block per grid).
static __device__ __align__(256) unsigned char g_noalloc_scratch[AIM_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};   // per device: the device address of g_noalloc_scratch
}  // namespace

// Device address of the scratch array on `dev`, which must be the current device (looked up once
// per device; in host code the array's name is only a host-side stand-in, not a device address).
static aim_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(AIM_EINVAL, "device index out of range for the no-alloc scratch");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return fail(AIM_ECUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return AIM_OK;
}

}  // namespace aim

using namespace aim;

extern "C" aim_status aim_grid_product_noalloc(aim_ctx* ctx, int filtered, int nrhs, const void* u, void* v,
                                               int precision, void* stream) {
  if (!ctx || !u || !v || nrhs < 1) return fail(AIM_EINVAL, "bad argument");
  if (precision < AIM_FP64 || precision > AIM_FP64_NATIVE) return fail(AIM_EINVAL, "precision must be 0, 1 or 2");
  // the scratch address is per device, and the context's spectra and twiddles live on ctx->device
  AIM_TRY(check_device(ctx));
  if (profiling_active())
    return fail(AIM_ESTATE, "kernel timing (aim_profile_start) creates events; stop it before the no-alloc call");
  const size_t need = inter_bytes_needed(ctx, nrhs, precision);
  if (need > (size_t)AIM_NOALLOC_SCRATCH_BYTES)
    return fail(AIM_EINVAL, "grid intermediate of " + std::to_string(need) + " bytes exceeds the no-alloc scratch of " +
                                std::to_string((size_t)AIM_NOALLOC_SCRATCH_BYTES) + " bytes (reduce nrhs or m)");
  // u and v must be device memory: staging host data would need buffers
  cudaPointerAttributes au, av;
  if (cudaPointerGetAttributes(&au, u) != cudaSuccess || cudaPointerGetAttributes(&av, v) != cudaSuccess) {
    cudaGetLastError();
    return fail(AIM_EINVAL, "u and v must be device pointers");
  }
  if ((au.type != cudaMemoryTypeDevice && au.type != cudaMemoryTypeManaged) ||
      (av.type != cudaMemoryTypeDevice && av.type != cudaMemoryTypeManaged))
    return fail(AIM_EINVAL, "u and v must be device pointers");
  void* scratch = nullptr;
  AIM_TRY(scratch_address(ctx->device, &scratch));
  // the scratch goes to the product as its intermediate buffer; the context's own workspace is
  // neither used nor touched
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double2* uin = static_cast<const double2*>(u);
  double2* vout = static_cast<double2*>(v);
  const size_t sb = (size_t)AIM_NOALLOC_SCRATCH_BYTES;
  if (precision == AIM_MIXED) return grid_product_dense<float2>(ctx, filtered != 0, nrhs, uin, vout, scratch, sb, st);
  if (precision == AIM_FP64_NATIVE)
    return grid_product_dense<double2>(ctx, filtered != 0, nrhs, uin, vout, scratch, sb, st);
  return grid_product_dense<dfc>(ctx, filtered != 0, nrhs, uin, vout, scratch, sb, st);
}
