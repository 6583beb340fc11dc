// Allocation-free variant of the operator apply.
//
// vsie_apply may grow a device buffer on its first call for a given size: when the
// targets alone cannot fill the GPU, the far-field sums split the sources across blocks
// and keep per-split partial sums in that buffer.  Some callers cannot let a library call
// cudaMalloc once set-up is over: a host application that reserves all device memory for
// its own pool at start-up and accounts for every byte afterwards, or a latency-critical
// loop that must not hit cudaMalloc's implicit device synchronisation.  vsie_apply_noalloc
// computes the same y = A x with the partial sums in a fixed, file-scope device array.
// The paper has no counterpart to this; it is an interface concern of this library.

#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "vsie_internal.h"

namespace vsie {

// Capacity of the split-partial scratch, in double2 elements: 2^21 = 2,097,152 elements
// (32 MiB).  Every device that loads the library holds this array until process exit.
constexpr size_t kNoAllocScratchElems = (size_t)1 << 21;

static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocScratchElems];

// Device address of g_noalloc_scratch, looked up once per device (host code may not use
// the symbol itself as a device pointer: on the host it names a shadow variable).  The
// address belongs to the device's context as it was at the lookup: after a device reset
// (cudaDeviceReset) the module is loaded again, possibly elsewhere, and the cached address
// is stale, so the entry point must not be used across a reset.
constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static double2* g_noalloc_ptr[kMaxDevices] = {};

static vsie_status noalloc_scratch(int device, double2** out) {
  if (device < 0 || device >= kMaxDevices) {
    set_error("vsie_apply_noalloc: device ordinal out of range");
    return VSIE_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    int prev = -1;
    VSIE_CUDA(cudaGetDevice(&prev));
    if (prev != device) VSIE_CUDA(cudaSetDevice(device));
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
    g_noalloc_ptr[device] = static_cast<double2*>(p);
  }
  *out = g_noalloc_ptr[device];
  return VSIE_OK;
}

// Set-up at operator creation: loads the array on the device (with lazy module loading
// the library's device image, and this array with it, is materialised on first use) and
// caches its address, so that later vsie_apply_noalloc calls allocate nothing.  A failure
// here is not an error of the creation: the first vsie_apply_noalloc call retries and
// reports it.
void noalloc_prepare(int device) {
  double2* p = nullptr;
  if (noalloc_scratch(device, &p) != VSIE_OK) clear_error();
}

}  // namespace vsie

using namespace vsie;

extern "C" vsie_status vsie_apply_noalloc(vsie_handle* h, const void* d_x, void* d_y,
                                          int32_t nrhs, int32_t precision, void* stream) {
  clear_error();
  TraceRange trace("vsie_apply_noalloc");
  if (!h || !d_x || !d_y) {
    set_error("vsie_apply_noalloc: null handle or vector");
    return VSIE_ERR_ARG;
  }
  if (nrhs < 1 || (precision != 32 && precision != 48 && precision != 64) || d_x == d_y) {
    set_error("vsie_apply_noalloc: nrhs must be >= 1, precision 32, 48 or 64, x and y distinct");
    return VSIE_ERR_ARG;
  }
  const size_t need = far_split_elems(h, precision);
  if (need > kNoAllocScratchElems) {
    set_error("vsie_apply_noalloc: this operator's launch shape needs " + std::to_string(need) +
              " scratch elements; the fixed scratch holds " + std::to_string(kNoAllocScratchElems) +
              " (use vsie_apply)");
    return VSIE_ERR_ARG;
  }
  double2* scratch = nullptr;
  VSIE_TRY(noalloc_scratch(h->device, &scratch));
  cudaStream_t st = (cudaStream_t)stream;
  const double2* x = (const double2*)d_x;
  double2* y = (double2*)d_y;
  for (int r = 0; r < nrhs; ++r) {
    const double2* xr = x + (size_t)r * h->n;
    double2* yr = y + (size_t)r * h->n;
    VSIE_TRY(far_prescale(h, xr, precision, st, nullptr));
    VSIE_TRY(far_sums_into(h, yr, precision, scratch, st));
    VSIE_TRY(correction_apply(h, xr, yr, precision, st));
  }
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}
