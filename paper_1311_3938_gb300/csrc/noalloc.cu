// aqc_norm2_noalloc: ||psi||^2 of a caller-owned device vector with no workspace and no device
// allocation.  Its reduction scratch (per-CTA partial sums, the last-CTA ticket and the result
// slot) lives in the file-scope array below, which every GPU that loads the library holds until
// the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/aqc.h"
#include "aqc_internal.h"

namespace aqc {
void set_global_error(const char* msg);  // message for aqc_last_error(NULL), defined in api.cu
}

namespace {

constexpr size_t kScratchBytes = AQC_NOALLOC_SCRATCH_BYTES;
constexpr size_t kOffCounter = 0;    // unsigned ticket, must be 0 when a reduction starts
constexpr size_t kOffSlots = 256;    // result slots (doubles)
constexpr size_t kOffPartials = 512; // one double per CTA

// Device scratch shared by every call on a device.  In host code this name is only a host-side
// stand-in: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" int aqc_norm2_noalloc(int precision, const void* psi, uint64_t n_amplitudes, void* cuda_stream,
                                 double* out) {
  using namespace aqc;
  if (precision != AQC_C128 && precision != AQC_C64) {
    set_global_error("aqc_norm2_noalloc: precision must be AQC_C128 or AQC_C64");
    return AQC_E_INVAL;
  }
  if (!psi || !out) {
    set_global_error("aqc_norm2_noalloc: psi and out must not be NULL");
    return AQC_E_INVAL;
  }
  if (((uintptr_t)psi) & (precision == AQC_C128 ? 15u : 7u)) {
    set_global_error("aqc_norm2_noalloc: psi must be aligned to its amplitude size (16 or 8 bytes)");
    return AQC_E_INVAL;
  }
  if (n_amplitudes == 0 || n_amplitudes > (1ull << kMaxN)) {
    set_global_error("aqc_norm2_noalloc: n_amplitudes must be in [1, 2^31]");
    return AQC_E_INVAL;
  }
  const int grid = reduce_grid(n_amplitudes);
  const size_t need = kOffPartials + (size_t)grid * sizeof(double);
  if (need > kScratchBytes) {
    set_global_error("aqc_norm2_noalloc: reduction needs more than the static scratch holds");
    return AQC_E_UNSUPPORTED;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_global_error("aqc_norm2_noalloc: no usable current CUDA device");
    return AQC_E_CUDA;
  }
  // once per device, with that device current: the scratch array's device address
  char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        set_global_error("aqc_norm2_noalloc: cudaGetSymbolAddress failed");
        return AQC_E_CUDA;
      }
      g_scratch_addr[dev] = p;
    }
    base = (char*)g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned* counter = (unsigned*)(base + kOffCounter);
  double* slots = (double*)(base + kOffSlots);
  double* partials = (double*)(base + kOffPartials);
  // the array keeps the previous call's contents: the ticket must start at zero
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = launch_reduce(precision, 0, psi, n_amplitudes, partials, counter, slots, grid, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, slots + kSlotNorm2, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return AQC_E_CUDA;
  }
  return AQC_OK;
}
