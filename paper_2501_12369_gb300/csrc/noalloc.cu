// darb_bin_sort_noalloc: darb_bin_sort with library-owned scratch, for callers that cannot
// allocate device memory.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes.  Every GPU that loads
// this library holds it until the process exits.  In host code the array's name is only a
// host-side stand-in, never a device address, so the first call on each device (with that
// device current) resolves the real address with cudaGetSymbolAddress and caches it; later
// calls on that device reuse it.  That first call may load this file's module, so it should
// come before any stream capture.  The cached address belongs to the device's context of that
// first call: a caller must not reset the device (cudaDeviceReset) while it uses this entry
// point, because the module is reloaded with the new context and may live at another address.
// All calls share the one array: the sort clears the parts that must start at zero on every
// call, and calls whose work overlaps on the GPU race.
#include <mutex>

#include "trace.h"
#include "validate.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;  // 64 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device; resolved once per device.
darb_status scratch_address(void **ptr) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DARB_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return DARB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return DARB_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *ptr = g_scratch_ptr[dev];
    return DARB_OK;
}

}  // namespace

extern "C" darb_status darb_bin_sort_noalloc(const darb_projected *proj, int32_t n, int32_t tile,
                                             const darb_camera *cam, const darb_kernel_params *kparams,
                                             uint64_t capacity, const darb_binning *out,
                                             uint64_t *num_instances_host, darb_stream stream) {
    DARB_TRACE(__func__);
    size_t need = 0;
    const darb_status qs = darb_bin_sort_workspace_size(n, tile, cam, capacity, DARB_SORT_DEPTH_THEN_TILE, &need);
    if (qs != DARB_OK) return qs;
    if (need > kNoAllocScratchBytes) return DARB_ERR_WORKSPACE;  // beyond the static scratch
    void *scratch = nullptr;
    const darb_status as = scratch_address(&scratch);
    if (as != DARB_OK) return as;
    // on the caller's stream only: no library side stream is created for this entry point
    return darb::bin_sort_entry(proj, n, tile, cam, kparams, scratch, kNoAllocScratchBytes, capacity,
                                DARB_SORT_DEPTH_THEN_TILE, out, num_instances_host, stream, false);
}
