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
struct ScratchAddr {
  unsigned long long ctx_id = 0;  // driver context the address belongs to (0: none yet)
  double* addr = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

// Process-unique id of the current driver context (cuCtxGetId ids are never reused
// within a process), looked up through the runtime's driver entry points.
cudaError_t current_context_id(unsigned long long* id) {
  static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || !f1 ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess || !f2)
      return cudaErrorNotSupported;
    get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f1);
    get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  unsigned long long v = 0;
  if (get_id(ctx, &v) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  *id = v;
  return cudaSuccess;
}

// Device address of g_pinv_scratch on `device` (which must be current). The host
// name g_pinv_scratch is only a stand-in for the symbol; the address a kernel can
// use comes from cudaGetSymbolAddress, once per device and context: a device reset
// ends the context (and the module holding the array), so the next call looks the
// address up again in the new one.
cudaError_t scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  ScratchAddr& c = g_scratch_addr[device];
  unsigned long long id = 0;
  if (c.addr) {
    cudaError_t e = current_context_id(&id);
    if (e != cudaSuccess) return e;
  }
  if (!c.addr || c.ctx_id != id) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_pinv_scratch);
    if (e != cudaSuccess) return e;
    e = current_context_id(&id);  // the context exists now
    if (e != cudaSuccess) return e;
    c.addr = static_cast<double*>(p);
    c.ctx_id = id;
  }
  *out = c.addr;
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
