// static_scratch.cu -- bdis_match_static: the method with no device allocation.
//
// For callers that cannot allocate GPU memory (a real-time loop with a frozen
// memory map, a plug-in inside a process that owns the allocator, a path
// where cudaMalloc may synchronise or fail). The scratch memory bdis_match
// takes from its handle's workspace comes here from one fixed array compiled
// into the library; the kernels are the same. The paper has no counterpart.
#include <stdio.h>

#include "bdis_internal.cuh"

namespace {

constexpr size_t kScratchBytes = BDIS_STATIC_SCRATCH_BYTES;

// The scratch itself. In host code this name is only a host-side stand-in for
// the device array, never a device address: kernels get the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch on the current device. Looked up on every call
// (cheap once the module is loaded), so that a context recreated after
// cudaDeviceReset never sees a stale address. The first lookup on a device
// loads the module there (lazy loading), which is when the array is reserved.
bdis_status scratch_address(void **out) {
  void *ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
  if (e != cudaSuccess) return bdis::record_cuda(e);
  *out = ptr;
  return BDIS_OK;
}

}  // namespace

extern "C" bdis_status bdis_match_static(const bdis_image *left, const bdis_image *right,
                                         const bdis_params *p, float *disparity_out,
                                         void *stream) {
  bdis_status s = bdis::check_match_args(left, right, p, disparity_out);
  if (s != BDIS_OK) return s;
  const size_t need = bdis::match_scratch_bytes(left->width, left->height, left->count, *p);
  if (need > kScratchBytes) {
    char msg[200];
    snprintf(msg, sizeof msg,
             "bdis_match_static: %d pair(s) of %dx%d need %zu bytes of scratch; the static "
             "array holds %zu",
             left->count, left->width, left->height, need, kScratchBytes);
    bdis::set_last_error(msg);
    return BDIS_E_UNSUPPORTED;
  }
  s = bdis::check_match_pointers(left, right, disparity_out);
  if (s != BDIS_OK) return s;
  void *scratch = nullptr;
  s = scratch_address(&scratch);
  if (s != BDIS_OK) return s;
  return bdis::run_match_in(scratch, kScratchBytes, static_cast<cudaStream_t>(stream), *left,
                            *right, *p, disparity_out);
}
