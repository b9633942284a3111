// Test hooks for failure handling (no paper counterpart): an injected device
// allocation failure, and a self-test of the bounded mbarrier wait that every
// pipeline kernel uses.  Neither faults, traps or hangs the GPU.
#include <atomic>

#include "hh_tc.cuh"

namespace hh {

// k > 0: the k-th device allocation from now on fails.
static std::atomic<int> g_fail_alloc{0};

static bool injected_failure() {
    int k = g_fail_alloc.load();
    while (k > 0) {
        if (g_fail_alloc.compare_exchange_weak(k, k - 1)) return k == 1;
    }
    return false;
}

cudaError_t dev_malloc(void **p, size_t bytes) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, st);
}

namespace {

// One thread waits, with the library's bounded wait, on an mbarrier that
// nothing arrives on; it records HH_ERR_TIMEOUT when the wait gives up.
__global__ void wait_probe_kernel(long long cycles, int *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
    *status = tc::mbar_wait(&bar, 0, cycles) ? (int)HH_OK : (int)HH_ERR_TIMEOUT;
}

}  // namespace
}  // namespace hh

using namespace hh;

extern "C" {

hh_status hh_debug_fail_alloc(int k) {
    if (k < 0) return fail(HH_ERR_INVALID_ARG, "k = %d < 0", k);
    g_fail_alloc.store(k);
    return HH_OK;
}

hh_status hh_debug_wait_timeout(int64_t cycles, void *stream) {
    if (cycles < 1 || cycles > 4000000000LL)
        return fail(HH_ERR_INVALID_ARG, "cycles = %lld outside [1, 4e9]", (long long)cycles);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int *d = nullptr;
    int word = -1;
    cudaError_t e;
    if ((e = cudaMallocAsync(reinterpret_cast<void **>(&d), sizeof(int), s))) return cuda_fail(e, "probe status");
    wait_probe_kernel<<<1, 32, 0, s>>>(cycles, d);
    if ((e = cudaGetLastError()) == cudaSuccess)
        e = cudaMemcpyAsync(&word, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    // the status word is freed on every path once it was allocated
    const cudaError_t ef = cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = ef;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "wait probe");
    if (word == HH_ERR_TIMEOUT)
        return fail(HH_ERR_TIMEOUT, "the bounded wait gave up after %lld cycles (expected)",
                    (long long)cycles);
    return word == HH_OK ? HH_OK : fail(HH_ERR_CUDA, "wait probe status %d", word);
}

}  // extern "C"
