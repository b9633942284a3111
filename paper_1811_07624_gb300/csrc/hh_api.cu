// C ABI of libhh: argument checks, plan lifetime, dispatch to the kernels.
#include <stdarg.h>
#include <stdio.h>

#include <new>
#include <vector>

#include "hh_internal.cuh"

namespace hh {

static thread_local std::string g_last_error;

hh_status fail(hh_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

hh_status cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(HH_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(HH_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// A pointer the current device's kernels may dereference: device memory of the
// current device, or managed memory.  Host and unregistered pointers are not.
bool device_ptr(const void *p, int dev) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

static void free_plan(Plan *p) {
    if (!p) return;
    wy_free(p);
    cudaFree(p->u);
    cudaFree(p->d);
    cudaFree(p->sign);
    cudaFree(p->tau);
    cudaFree(p->tau_t);
    cudaFree(p->gram);
    cudaFree(p->vnorm);
    cudaFree(p->err);
    cudaFree(p->upd);
    cudaFree(p->start);
    delete p;
}

hh_status check_plan(const Plan *p) {
    if (!p) return fail(HH_ERR_INVALID_ARG, "plan is NULL");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device)
        return fail(HH_ERR_INVALID_ARG, "plan was created on device %d, current device is %d",
                    p->device, dev);
    return HH_OK;
}

static hh_status check_rows(const Plan *p, const void *A, int64_t lda, int64_t batch,
                            const char *name) {
    if (lda < p->n) return fail(HH_ERR_INVALID_ARG, "%s: leading dimension %lld < n = %lld", name,
                                (long long)lda, (long long)p->n);
    if (batch > 0 && !device_ptr(A, p->device))
        return fail(HH_ERR_INVALID_ARG, "%s: not a device pointer of device %d", name, p->device);
    return HH_OK;
}

static hh_status apply_common(hh_plan_t plan, hh_mode mode, const void *X, int64_t ldx, void *Y,
                              int64_t ldy, int64_t batch, void *stream) {
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    hh_status st = check_plan(p);
    if (st) return st;
    if (batch < 0) return fail(HH_ERR_INVALID_ARG, "batch %lld < 0", (long long)batch);
    if ((st = check_rows(p, X, ldx, batch, "X"))) return st;
    if ((st = check_rows(p, Y, ldy, batch, "Y"))) return st;
    if (mode == HH_MODE_SYM && !p->d)
        return fail(HH_ERR_INVALID_ARG, "apply_sym: the plan has no spectrum d");
    if (X == Y && ldx != ldy)
        return fail(HH_ERR_INVALID_ARG, "in-place apply needs ldx == ldy");
    if (batch == 0) return HH_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (p->path == HH_PATH_FUSED) return fused_apply(p, mode, X, ldx, Y, ldy, batch, s);
    if (p->path == HH_PATH_WY) return wy_apply(p, mode, X, ldx, Y, ldy, batch, s);
    return fail(HH_ERR_UNSUPPORTED, "no kernel for this plan's path");
}

hh_status check_backward_args(const Plan *p, hh_mode mode, const void *saved, int64_t lds,
                              const void *gY, int64_t ldgy, const void *gX, int64_t ldgx,
                              const void *gU, const void *gd, int64_t batch) {
    hh_status st = check_plan(p);
    if (st) return st;
    if (mode != HH_MODE_W && mode != HH_MODE_WT && mode != HH_MODE_SYM)
        return fail(HH_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
    if (p->path != HH_PATH_FUSED)
        return fail(HH_ERR_UNSUPPORTED, "backward: F32 and F64 plans only");
    if (batch < 0) return fail(HH_ERR_INVALID_ARG, "batch %lld < 0", (long long)batch);
    if (mode == HH_MODE_SYM && !p->d)
        return fail(HH_ERR_INVALID_ARG, "backward SYM: the plan has no spectrum d");
    if (gd && mode != HH_MODE_SYM)
        return fail(HH_ERR_INVALID_ARG, "backward: gd is only defined for mode SYM");
    if ((st = check_rows(p, saved, lds, batch, "saved"))) return st;
    if ((st = check_rows(p, gY, ldgy, batch, "gY"))) return st;
    if (gX && (st = check_rows(p, gX, ldgx, batch, "gX"))) return st;
    if (gX && (gX == saved || gX == gY))
        return fail(HH_ERR_INVALID_ARG, "backward: gX may not alias saved or gY");
    if (gU && p->h > 0 && !device_ptr(gU, p->device))
        return fail(HH_ERR_INVALID_ARG, "gU: not a device pointer of device %d", p->device);
    if (gd && !device_ptr(gd, p->device))
        return fail(HH_ERR_INVALID_ARG, "gd: not a device pointer of device %d", p->device);
    return HH_OK;
}

}  // namespace hh

using namespace hh;

extern "C" {

const char *hh_last_error(void) { return g_last_error.c_str(); }

const char *hh_version(void) { return "libhh 0.1 (sm_103a)"; }

hh_status hh_create(hh_plan_t *out, int64_t n, int64_t h, const void *U, int64_t ldu,
                    const void *d, hh_dtype dtype) {
    return hh_create_ex(out, n, h, U, ldu, d, nullptr, dtype, HH_PATH_AUTO, nullptr);
}

hh_status hh_create_ex(hh_plan_t *out, int64_t n, int64_t h, const void *U, int64_t ldu,
                       const void *d, const int8_t *sign, hh_dtype dtype, hh_path path,
                       void *stream) {
    TraceRange trace("hh_create_ex");
    if (!out) return fail(HH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1) return fail(HH_ERR_INVALID_ARG, "n = %lld < 1", (long long)n);
    if (h < 0) return fail(HH_ERR_INVALID_ARG, "h = %lld < 0", (long long)h);
    if (n > (int64_t(1) << 24) || h > (int64_t(1) << 20))
        return fail(HH_ERR_INVALID_ARG, "n = %lld or h = %lld too large", (long long)n,
                    (long long)h);
    if (dtype != HH_F32 && dtype != HH_F64 && dtype != HH_BF16)
        return fail(HH_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    if (path != HH_PATH_AUTO && path != HH_PATH_FUSED && path != HH_PATH_WY)
        return fail(HH_ERR_INVALID_ARG, "unknown path %d", (int)path);
    if (path == HH_PATH_AUTO) path = dtype == HH_BF16 ? HH_PATH_WY : HH_PATH_FUSED;
    if (path == HH_PATH_FUSED && dtype == HH_BF16)
        return fail(HH_ERR_UNSUPPORTED, "the fused path computes in F32 or F64");
    if (path == HH_PATH_WY && dtype != HH_BF16)
        return fail(HH_ERR_UNSUPPORTED, "the compact-WY path computes in BF16");
    if (h > 0 && ldu < n)
        return fail(HH_ERR_INVALID_ARG, "ldu = %lld < n = %lld", (long long)ldu, (long long)n);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (h > 0 && !device_ptr(U, dev))
        return fail(HH_ERR_INVALID_ARG, "U: not a device pointer of device %d", dev);
    if (d && !device_ptr(d, dev))
        return fail(HH_ERR_INVALID_ARG, "d: not a device pointer of device %d", dev);
    if (sign && !device_ptr(sign, dev))
        return fail(HH_ERR_INVALID_ARG, "sign: not a device pointer of device %d", dev);

    Plan *p = new (std::nothrow) Plan();
    if (!p) return fail(HH_ERR_OOM, "host allocation failed");
    p->n = n;
    p->h = h;
    p->dtype = dtype;
    p->path = path;
    p->device = dev;
    p->ldv = padded_ld(n);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int *flag = nullptr;
    hh_status st = HH_OK;
    size_t es = dtype_size(dtype);
    if ((e = dev_malloc(&p->u, es * (size_t)p->ldv * (size_t)(h > 0 ? h : 1))) ||
        (e = dev_malloc(&p->tau, sizeof(double) * (size_t)(h > 0 ? h : 1))) ||
        (e = dev_malloc(&p->tau_t, es * (size_t)(h > 0 ? h : 1))) ||
        (e = dev_malloc(&p->gram, es * 16 * (size_t)(h > 0 ? h : 1))) ||
        (e = dev_malloc(&p->vnorm, sizeof(double) * (size_t)(h > 0 ? h : 1))) ||
        (e = dev_malloc(&p->start, sizeof(int) * (size_t)(h > 0 ? h : 1))) ||
        (d && (e = dev_malloc(&p->d, es * (size_t)p->ldv))) ||
        (sign && (e = dev_malloc(&p->sign, es * (size_t)p->ldv))) ||
        (e = dev_malloc(&p->err, sizeof(int))) || (e = dev_malloc(&p->upd, sizeof(int))) ||
        (e = dev_malloc(&flag, sizeof(int)))) {
        st = cuda_fail(e, "cudaMalloc (plan)");
        goto done;
    }
    if ((e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev))) {
        st = cuda_fail(e, "cudaDeviceGetAttribute");
        goto done;
    }
    if ((e = cudaMemsetAsync(flag, 0, sizeof(int), s)) ||
        (e = cudaMemsetAsync(p->err, 0, sizeof(int), s)) ||
        (e = cudaMemsetAsync(p->upd, 0, sizeof(int), s))) {
        st = cuda_fail(e, "cudaMemsetAsync");
        goto done;
    }
    if (path == HH_PATH_WY) {
        st = wy_prepare(p, U, ldu, sign, flag, s);
        if (!st) st = wy_prepare_sign(p, sign, flag, s);
    } else {
        st = prepare_fused(p, U, ldu, d, sign, flag, s);
    }
    if (st) goto done;
    {
        int hflag = 0;
        if ((e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
            (e = cudaStreamSynchronize(s))) {
            st = cuda_fail(e, "plan preparation");
            goto done;
        }
        if (path == HH_PATH_WY) wy_release_workspace(p);
        if (path == HH_PATH_FUSED && h > 0 && !(hflag & 1)) {
            // zero prefixes (e.g. the reflectors of a partial QR factorization):
            // worth skipping when they hold at least 1/16 of U's entries
            std::vector<int> hs((size_t)h);
            if ((e = cudaMemcpy(hs.data(), p->start, sizeof(int) * (size_t)h,
                                cudaMemcpyDeviceToHost))) {
                st = cuda_fail(e, "plan preparation");
                goto done;
            }
            double zeros = 0;
            for (int v : hs) zeros += v;
            p->skip_auto = zeros * 16.0 >= (double)n * (double)h;
            p->skip_prefix = p->skip_auto;
        }
        if (hflag & 1) st = fail(HH_ERR_NONFINITE, "U holds a NaN or Inf");
        else if (hflag & 2) st = fail(HH_ERR_NONFINITE, "d holds a NaN or Inf");
        else if (hflag & 4) st = fail(HH_ERR_INVALID_ARG, "sign holds a value other than +1/-1");
    }
done:
    cudaFree(flag);
    if (st) {
        free_plan(p);
        return st;
    }
    *out = reinterpret_cast<hh_plan_t>(p);
    return HH_OK;
}

hh_status hh_destroy(hh_plan_t plan) {
    if (!plan) return HH_OK;
    Plan *p = reinterpret_cast<Plan *>(plan);
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    cudaError_t e = cudaDeviceSynchronize();
    free_plan(p);
    if (cur != p->device) cudaSetDevice(cur);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize (destroy)");
    return HH_OK;
}

hh_status hh_sync(hh_plan_t plan, void *stream) {
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    hh_status st = check_plan(p);
    if (st) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int word = 0;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(&word, p->err, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemsetAsync(p->err, 0, sizeof(int), s)) || (e = cudaStreamSynchronize(s)))
        return cuda_fail(e, "hh_sync");
    if (word == HH_ERR_TIMEOUT)
        return fail(HH_ERR_TIMEOUT, "a kernel's bounded wait on its bulk copy expired");
    if (word == HH_ERR_INVALID_ARG)
        return fail(HH_ERR_INVALID_ARG, "a pair index was outside [0, nrows)");
    if (word == HH_ERR_NONFINITE)
        return fail(HH_ERR_NONFINITE, "an update's U or d held a NaN or Inf");
    if (word != 0) return fail(HH_ERR_CUDA, "device status word %d", word);
    return HH_OK;
}

hh_status hh_update(hh_plan_t plan, const void *U, int64_t ldu, const void *d, void *stream) {
    TraceRange trace("hh_update");
    Plan *p = reinterpret_cast<Plan *>(plan);
    hh_status st = check_plan(p);
    if (st) return st;
    if (p->path != HH_PATH_FUSED)
        return fail(HH_ERR_UNSUPPORTED, "update: F32 and F64 plans only (compact-WY: create anew)");
    if (p->h > 0 && ldu < p->n)
        return fail(HH_ERR_INVALID_ARG, "ldu = %lld < n = %lld", (long long)ldu, (long long)p->n);
    if (p->h > 0 && !device_ptr(U, p->device))
        return fail(HH_ERR_INVALID_ARG, "U: not a device pointer of device %d", p->device);
    if ((d != nullptr) != (p->d != nullptr))
        return fail(HH_ERR_INVALID_ARG, p->d ? "update: the plan has a spectrum, d is required"
                                             : "update: the plan has no spectrum, d must be NULL");
    if (d && !device_ptr(d, p->device))
        return fail(HH_ERR_INVALID_ARG, "d: not a device pointer of device %d", p->device);
    return update_fused(p, U, ldu, d, reinterpret_cast<cudaStream_t>(stream));
}

hh_status hh_plan_info(hh_plan_t plan, int64_t *n, int64_t *h, hh_dtype *dtype, hh_path *path) {
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p) return fail(HH_ERR_INVALID_ARG, "plan is NULL");
    if (n) *n = p->n;
    if (h) *h = p->h;
    if (dtype) *dtype = p->dtype;
    if (path) *path = p->path;
    return HH_OK;
}

hh_status hh_plan_skip_prefix(hh_plan_t plan, int mode, int *enabled) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p) return fail(HH_ERR_INVALID_ARG, "plan is NULL");
    if (mode < -2 || mode > 1)
        return fail(HH_ERR_INVALID_ARG, "mode %d (expected -2, -1, 0 or 1)", mode);
    if (mode != -2 && p->path == HH_PATH_FUSED && p->dtype == HH_F32 && p->h > 0)
        p->skip_prefix = mode == -1 ? p->skip_auto : mode == 1;
    if (enabled) *enabled = p->skip_prefix ? 1 : 0;
    return HH_OK;
}

hh_status hh_apply(hh_plan_t plan, const void *X, int64_t ldx, void *Y, int64_t ldy,
                   int64_t batch, void *stream) {
    TraceRange trace("hh_apply");
    return apply_common(plan, HH_MODE_W, X, ldx, Y, ldy, batch, stream);
}

hh_status hh_apply_T(hh_plan_t plan, const void *X, int64_t ldx, void *Y, int64_t ldy,
                     int64_t batch, void *stream) {
    TraceRange trace("hh_apply_T");
    return apply_common(plan, HH_MODE_WT, X, ldx, Y, ldy, batch, stream);
}

hh_status hh_apply_sym(hh_plan_t plan, const void *X, int64_t ldx, void *Y, int64_t ldy,
                       int64_t batch, void *stream) {
    TraceRange trace("hh_apply_sym");
    return apply_common(plan, HH_MODE_SYM, X, ldx, Y, ldy, batch, stream);
}

hh_status hh_backward(hh_plan_t plan, hh_mode mode, const void *saved, int64_t lds,
                      const void *gY, int64_t ldgy, void *gX, int64_t ldgx, void *gU, void *gd,
                      int64_t batch, void *stream) {
    TraceRange trace("hh_backward");
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    hh_status st = check_backward_args(p, mode, saved, lds, gY, ldgy, gX, ldgx, gU, gd, batch);
    if (st) return st;
    if (batch == 0 && !gU && !gd) return HH_OK;
    return backward(p, mode, saved, lds, gY, ldgy, gX, ldgx, gU, gd, batch, nullptr, 0,
                    reinterpret_cast<cudaStream_t>(stream));
}

hh_status hh_apply_sym_p(hh_plan_t plan, const void *X, int64_t ldx, void *Y, int64_t ldy,
                         void *P, int64_t ldp, int64_t batch, void *stream) {
    TraceRange trace("hh_apply_sym_p");
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    hh_status st = check_plan(p);
    if (st) return st;
    if (p->path != HH_PATH_FUSED)
        return fail(HH_ERR_UNSUPPORTED, "apply_sym_p: F32 and F64 plans only");
    if (batch < 0) return fail(HH_ERR_INVALID_ARG, "batch %lld < 0", (long long)batch);
    if ((st = check_rows(p, X, ldx, batch, "X"))) return st;
    if ((st = check_rows(p, Y, ldy, batch, "Y"))) return st;
    if ((st = check_rows(p, P, ldp, batch, "P"))) return st;
    if (!p->d) return fail(HH_ERR_INVALID_ARG, "apply_sym: the plan has no spectrum d");
    if (X == Y && ldx != ldy) return fail(HH_ERR_INVALID_ARG, "in-place apply needs ldx == ldy");
    if (batch > 0 && (P == X || P == Y))
        return fail(HH_ERR_INVALID_ARG, "apply_sym_p: P may alias neither X nor Y");
    if (batch == 0) return HH_OK;
    return fused_apply_p(p, HH_MODE_SYM, X, ldx, Y, ldy, P, ldp, batch,
                         reinterpret_cast<cudaStream_t>(stream));
}

hh_status hh_backward_sym_py(hh_plan_t plan, const void *P, int64_t ldp, const void *y,
                             int64_t ldy, const void *gY, int64_t ldgy, void *gX, int64_t ldgx,
                             void *gU, void *gd, int64_t batch, void *stream) {
    TraceRange trace("hh_backward_sym_py");
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    hh_status st =
        check_backward_args(p, HH_MODE_SYM, P, ldp, gY, ldgy, gX, ldgx, gU, gd, batch);
    if (st) return st;
    if ((st = check_rows(p, y, ldy, batch, "y"))) return st;
    if (gX && gX == y) return fail(HH_ERR_INVALID_ARG, "backward: gX may not alias y");
    if (batch == 0 && !gU && !gd) return HH_OK;
    return backward_sym_py(p, P, ldp, y, ldy, gY, ldgy, gX, ldgx, gU, gd, batch,
                           reinterpret_cast<cudaStream_t>(stream));
}

hh_status hh_backward_sym_y(hh_plan_t plan, const void *x, int64_t ldx, const void *y,
                            int64_t ldy, const void *gY, int64_t ldgy, void *gX, int64_t ldgx,
                            void *gU, void *gd, int64_t batch, void *stream) {
    TraceRange trace("hh_backward_sym_y");
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    hh_status st =
        check_backward_args(p, HH_MODE_SYM, x, ldx, gY, ldgy, gX, ldgx, gU, gd, batch);
    if (st) return st;
    if ((st = check_rows(p, y, ldy, batch, "y"))) return st;
    if (gX && gX == y) return fail(HH_ERR_INVALID_ARG, "backward: gX may not alias y");
    if (batch == 0 && !gU && !gd) return HH_OK;
    return backward_sym_y(p, x, ldx, y, ldy, gY, ldgy, gX, ldgx, gU, gd, batch,
                          reinterpret_cast<cudaStream_t>(stream));
}

static hh_status check_pairs(const Plan *p, const void *X, int64_t ldx, int64_t nrows,
                             const int64_t *ia, const int64_t *ib, int64_t npairs) {
    hh_status st = check_plan(p);
    if (st) return st;
    if (p->path != HH_PATH_FUSED)
        return fail(HH_ERR_UNSUPPORTED, "mahalanobis: F32 and F64 plans only");
    if (!p->d) return fail(HH_ERR_INVALID_ARG, "mahalanobis: the plan has no spectrum d");
    if (nrows < 0 || npairs < 0)
        return fail(HH_ERR_INVALID_ARG, "nrows = %lld, npairs = %lld", (long long)nrows,
                    (long long)npairs);
    if (npairs > 0 && nrows == 0) return fail(HH_ERR_INVALID_ARG, "pairs given but X has no rows");
    if ((st = check_rows(p, X, ldx, npairs > 0 ? nrows : 0, "X"))) return st;
    if (npairs > 0 && (!device_ptr(ia, p->device) || !device_ptr(ib, p->device)))
        return fail(HH_ERR_INVALID_ARG, "ia, ib: not device pointers of device %d", p->device);
    return HH_OK;
}

hh_status hh_mahalanobis(hh_plan_t plan, const void *X, int64_t ldx, int64_t nrows,
                         const int64_t *ia, const int64_t *ib, int64_t npairs, void *out,
                         void *stream) {
    TraceRange trace("hh_mahalanobis");
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    hh_status st = check_pairs(p, X, ldx, nrows, ia, ib, npairs);
    if (st) return st;
    if (npairs == 0) return HH_OK;
    if (!device_ptr(out, p->device))
        return fail(HH_ERR_INVALID_ARG, "out: not a device pointer of device %d", p->device);
    return mahalanobis(p, X, ldx, nrows, ia, ib, npairs, out,
                       reinterpret_cast<cudaStream_t>(stream));
}

hh_status hh_mahalanobis_backward(hh_plan_t plan, const void *X, int64_t ldx, int64_t nrows,
                                  const int64_t *ia, const int64_t *ib, int64_t npairs,
                                  const void *gout, void *gU, void *gd, void *stream) {
    TraceRange trace("hh_mahalanobis_backward");
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    hh_status st = check_pairs(p, X, ldx, nrows, ia, ib, npairs);
    if (st) return st;
    if (npairs > 0 && !device_ptr(gout, p->device))
        return fail(HH_ERR_INVALID_ARG, "gout: not a device pointer of device %d", p->device);
    if (gU && p->h > 0 && !device_ptr(gU, p->device))
        return fail(HH_ERR_INVALID_ARG, "gU: not a device pointer of device %d", p->device);
    if (gd && !device_ptr(gd, p->device))
        return fail(HH_ERR_INVALID_ARG, "gd: not a device pointer of device %d", p->device);
    if (!gU && !gd) return HH_OK;
    return mahalanobis_backward(p, X, ldx, nrows, ia, ib, npairs, gout, gU, gd,
                                reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
