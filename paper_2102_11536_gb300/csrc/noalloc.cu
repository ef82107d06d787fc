// Preconditioner application that performs no device allocation: its two
// intermediate buffers live in a fixed array compiled into this library
// (see iga_apply_Pinv_noalloc in include/iga_galpha.h).
#include <mutex>

#include "iga_internal.h"

namespace {

// Two scratch buffers of kNoAllocMaxElems doubles each (16 MiB in total). The array
// is part of the library's device image, so every GPU that loads the library
// holds it until the process exits.
__device__ __align__(256) double g_pinv_scratch[2 * iga::kNoAllocMaxElems];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Device address of g_pinv_scratch on `device` (which must be current). The host
// name g_pinv_scratch is only a stand-in for the symbol; the address a kernel can
// use comes from cudaGetSymbolAddress, once per device.
cudaError_t scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_pinv_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" int iga_apply_Pinv_noalloc(iga_handle* h, int nvec, const double* x, double* y) {
  if (!h) return IGA_EINVAL;
  int device = 0;
  int rc = iga::handle_device(h, &device);
  if (rc != IGA_OK) return rc;
  if (nvec < 1 || nvec > iga::kMaxVec || !x || !y)
    return iga::handle_fail(h, IGA_EINVAL, "iga_apply_Pinv_noalloc: bad arguments");
  long long ndof = 0;
  iga_ndof(h, &ndof);
  if ((long long)nvec * ndof > iga::kNoAllocMaxElems)
    return iga::handle_fail(h, IGA_EINVAL,
                            "iga_apply_Pinv_noalloc: nvec * N exceeds the fixed scratch of 1048576 values");
  double* base = nullptr;
  cudaError_t e = scratch_address(device, &base);
  if (e != cudaSuccess)
    return iga::handle_fail(h, IGA_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  // Nothing here needs to start at zero: every mode product writes all of its
  // outputs before the next one reads them.
  return iga::pinv_with_scratch(h, nvec, x, y, base, base + iga::kNoAllocMaxElems);
}
