// Scratch memory of the allocation-free diagnostics entry point
// (tled_get_stats_noalloc in include/tled.h).
//
// Some callers cannot allocate device memory at the moment they want the
// diagnostics: real-time loops in which an allocation would synchronise the
// device or take an unbounded time, and processes whose device memory is fully
// reserved by another framework's caching allocator.  For them the reduction's block
// partial sums live in this file-scope array instead of the caller's
// workspace.  It is kNoAllocMaxBlocks x 8 doubles (18,944 bytes) and stays
// resident on every GPU that loads the library until the process exits.
#include <mutex>

#include "tled_internal.h"

namespace tled {

static __device__ __align__(256) double g_noalloc_stats_scratch[kNoAllocMaxBlocks * 8];

namespace {
std::mutex g_mu;
constexpr int kMaxDevices = 256;
double *g_dev_ptr[kMaxDevices] = {nullptr};
}  // namespace

// Device address of the scratch array on `device`.  The host-side name of the
// array is only a stand-in, so the address is looked up once per device (with
// that device current) and cached for the process.  A cudaDeviceReset of the
// device ends the context that address belongs to, so the cached address is
// stale afterwards (the header says so).  The caller must have made `device`
// current.  Returns cudaSuccess or the lookup's error.
cudaError_t noalloc_scratch(int device, double **ptr) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_stats_scratch);
        if (e != cudaSuccess) return e;
        g_dev_ptr[device] = static_cast<double *>(p);
    }
    *ptr = g_dev_ptr[device];
    return cudaSuccess;
}

}  // namespace tled
