// Internal declarations shared by the libhh translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <mutex>
#include <string>

#include "hh.h"

namespace hh {

// NVTX range named after one C-ABI call, visible in Nsight timelines (a
// pointer test and nothing more when no tool is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Device ordinals the library keeps per-device state for (kernel attributes,
// occupancy, the no-allocation scratch address).
constexpr int kMaxDevices = 64;

// Once-per-device set-up of a kernel.  Attributes such as the dynamic
// shared-memory opt-in are per-device settings, so the set-up runs the first
// time each device ordinal launches the kernel (under a lock: launches may
// come from several host threads) and its result, e.g. the resident CTAs per
// SM measured with that opt-in, is cached under the same ordinal.
struct PerDevice {
    std::mutex mu;
    int value[kMaxDevices] = {};
    bool done[kMaxDevices] = {};
};
// Runs setup(int &value) -> cudaError_t on the current device's first call;
// returns the cached value in `out`.
template <typename F>
cudaError_t per_device(PerDevice &pd, int &out, F &&setup) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(pd.mu);
    if (!pd.done[dev]) {
        int v = 0;
        e = setup(v);
        if (e != cudaSuccess) return e;
        pd.value[dev] = v;
        pd.done[dev] = true;
    }
    out = pd.value[dev];
    return cudaSuccess;
}

// Row stride (elements) of every per-plan vector stored on the device: the
// next power of two >= max(n, 1024) up to 16384, else n rounded up to 1024.
// Every fused-kernel column tiling covers at most this many columns, so the
// kernels read zero padding, never past the allocation.
inline int64_t padded_ld(int64_t n) {
    if (n <= 16384) {
        int64_t c = 1024;
        while (c < n) c *= 2;
        return c;
    }
    return round_up(n, 1024);
}

struct Plan {
    int64_t n = 0, h = 0;
    hh_dtype dtype = HH_F32;
    hh_path path = HH_PATH_FUSED;
    int device = 0;
    int64_t ldv = 0;        // padded row stride of every stored vector, elements
    // FUSED path, compute dtype (float or double):
    void *u = nullptr;      // h x ldv, v_k as given (zero padded), compute dtype
    void *tau_t = nullptr;  // h, tau_k rounded to the compute dtype: H_k z = z - tau_k v_k (v_k . z)
    void *gram = nullptr;   // h x 16, gram[k*16 + j] = v_k . v_{k+j} (j = 1..15, FP64 sums), compute dtype
    void *d = nullptr;      // ldv, spectrum (zero padded), or null
    void *sign = nullptr;   // ldv, +-1 (one padded), or null
    double *tau = nullptr;  // h, tau_k = 2 / v_k^T v_k (0 for v_k = 0)
    double *vnorm = nullptr;// h, |v_k|
    int *start = nullptr;   // h, first non-zero column of v_k (n for v_k = 0)
    bool skip_prefix = false;  // F32 kernels skip zero prefixes (hh_plan_skip_prefix)
    bool skip_auto = false;    // at create, the zero prefixes held >= 1/16 of U
    int *err = nullptr;     // device status word: a kernel's bounded wait expired (HH_ERR_TIMEOUT)
    int *upd = nullptr;     // device flag of the last hh_update's prepare kernels (bit 1: U, 2: d)
    int num_sms = 0;
    // WY path (BF16 storage): filled by wy_prepare
    void *wy = nullptr;
};

// Thread-local error message, set by fail().
hh_status fail(hh_status st, const char *fmt, ...);
hh_status cuda_fail(cudaError_t e, const char *what);

// Device allocations of the library go through these; the test hook
// hh_debug_fail_alloc can make the k-th one fail (cudaErrorMemoryAllocation).
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st);
template <typename T>
inline cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc(reinterpret_cast<void **>(p), bytes);
}

// A pointer the kernels of device `dev` may dereference (device or managed memory).
bool device_ptr(const void *p, int dev);
// The plan is non-null and belongs to the current device.
hh_status check_plan(const Plan *p);

inline size_t dtype_size(hh_dtype t) {
    return t == HH_F64 ? 8 : (t == HH_BF16 ? 2 : 4);
}

// ---- prepare (hh_prepare.cu) ----
// Normalise the reflectors in FP64 and write the plan's device vectors.
// Sets *nonfinite (device int) if U or d holds a NaN/Inf.
hh_status prepare_fused(Plan *p, const void *U, int64_t ldu, const void *d, const int8_t *sign,
                        int *bad_flag, cudaStream_t st);
// New reflector values (and spectrum) for an existing F32/F64 plan, stream-ordered,
// no allocation: a NaN or Inf becomes HH_ERR_NONFINITE in the status word.
hh_status update_fused(Plan *p, const void *U, int64_t ldu, const void *d, cudaStream_t st);

// ---- compact-WY path on the tensor cores (hh_wy.cu), BF16 plans ----
hh_status wy_prepare(Plan *p, const void *U, int64_t ldu, const int8_t *sign, int *flag,
                     cudaStream_t st);
hh_status wy_prepare_sign(Plan *p, const int8_t *sign, int *flag, cudaStream_t st);
void wy_release_workspace(Plan *p);
void wy_free(Plan *p);
hh_status wy_apply(const Plan *p, hh_mode mode, const void *X, int64_t ldx, void *Y, int64_t ldy,
                   int64_t batch, cudaStream_t st);

// ---- fused apply (hh_fused.cu) ----
hh_status fused_apply(const Plan *p, hh_mode mode, const void *X, int64_t ldx, void *Y,
                      int64_t ldy, int64_t batch, cudaStream_t st);
// The same; mode SYM with P (may be null) also writes p = W^T (sigma .* x)
// (rows of P, leading dimension ldp).
hh_status fused_apply_p(const Plan *p, hh_mode mode, const void *X, int64_t ldx, void *Y,
                        int64_t ldy, void *P, int64_t ldp, int64_t batch, cudaStream_t st);

// ---- adjoint (hh_backward.cu) ----
// Argument checks shared by the adjoint entry points (hh_api.cu).
hh_status check_backward_args(const Plan *p, hh_mode mode, const void *saved, int64_t lds,
                              const void *gY, int64_t ldgy, const void *gX, int64_t ldgx,
                              const void *gU, const void *gd, int64_t batch);
// scratch: caller-provided device buffer of scratch_bytes, or null to allocate
// (stream-ordered) per call.
hh_status backward(const Plan *p, hh_mode mode, const void *S, int64_t lds, const void *gY,
                   int64_t ldg, void *gX, int64_t ldgx, void *gU, void *gd, int64_t batch,
                   void *scratch, size_t scratch_bytes, cudaStream_t st);
// Mode SYM from p = W^T (sigma .* x) and y = S_bar x (the input is not needed).
hh_status backward_sym_py(const Plan *p, const void *P, int64_t ldp, const void *Y, int64_t ldy,
                          const void *gY, int64_t ldg, void *gX, int64_t ldgx, void *gU, void *gd,
                          int64_t batch, cudaStream_t st);
// Mode SYM with the forward output y = S_bar x (q = sigma .* y is read).
hh_status backward_sym_y(const Plan *p, const void *X, int64_t ldx, const void *Y, int64_t ldy,
                         const void *gY, int64_t ldg, void *gX, int64_t ldgx, void *gU, void *gd,
                         int64_t batch, cudaStream_t st);

// ---- fast Mahalanobis distance (hh_mahalanobis.cu, hh_backward.cu) ----
hh_status mahalanobis(const Plan *p, const void *X, int64_t ldx, int64_t nrows, const int64_t *ia,
                      const int64_t *ib, int64_t npairs, void *out, cudaStream_t st);
hh_status mahalanobis_backward(const Plan *p, const void *X, int64_t ldx, int64_t nrows,
                               const int64_t *ia, const int64_t *ib, int64_t npairs,
                               const void *gout, void *gU, void *gd, cudaStream_t st);

}  // namespace hh
