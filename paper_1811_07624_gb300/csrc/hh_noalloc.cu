// hh_backward_noalloc: the adjoint of hh_backward for callers that must not
// allocate device memory (see include/hh.h).  Its scratch is one file-scope
// device array of kNoAllocScratchBytes, part of this library's device image,
// so it exists on every device that loads the library until the process ends.
#include <mutex>

#include "hh_internal.cuh"

namespace hh {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB

// Shared by every call on a device: calls that overlap on the GPU race on it.
// The backward kernel initialises every byte it later reads (each CTA zeroes
// its own partial sums), so nothing left from an earlier call is used.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device with cudaGetSymbolAddress (which resolves it on the current
// device) and cached under that same device's ordinal.
hh_status scratch_address(void **out) {
    int dev = -1;
    cudaError_t ed = cudaGetDevice(&dev);
    if (ed != cudaSuccess) return cuda_fail(ed, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(HH_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress (no-alloc scratch)");
        if (!ptr) return fail(HH_ERR_CUDA, "cudaGetSymbolAddress returned a null address");
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return HH_OK;
}

}  // namespace
}  // namespace hh

using namespace hh;

extern "C" hh_status hh_backward_noalloc(hh_plan_t plan, hh_mode mode, const void *saved,
                                         int64_t lds, const void *gY, int64_t ldgy, void *gX,
                                         int64_t ldgx, void *gU, void *gd, int64_t batch,
                                         void *stream) {
    TraceRange trace("hh_backward_noalloc");
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    hh_status st = check_backward_args(p, mode, saved, lds, gY, ldgy, gX, ldgx, gU, gd, batch);
    if (st) return st;
    if (batch == 0 && !gU && !gd) return HH_OK;
    void *scratch = nullptr;
    // check_backward_args has made sure the current device is the plan's
    if ((st = scratch_address(&scratch))) return st;
    // backward() with a caller buffer never allocates: it lowers the number of
    // CTAs until their partial sums fit, and rejects the call if one CTA's do not.
    return backward(p, mode, saved, lds, gY, ldgy, gX, ldgx, gU, gd, batch, scratch,
                    kNoAllocScratchBytes, reinterpret_cast<cudaStream_t>(stream));
}
