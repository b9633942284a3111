// Plan preparation (create time, not on the hot path): reflector normalisation
// in FP64 and the padded device copies of the reflectors, spectrum and sign.
//
// Reflector k is H_k = I - tau_k v_k v_k^T with tau_k = 2 / (v_k^T v_k)
// (§II-A, Eq. (2) with u_k = v_k / |v_k|); tau_k = 0 when v_k = 0, so
// H_k = I (§II-B).  The kernels read v_k as given (zero padded to the plan's
// row stride) and apply H_k z = z - tau_k v_k (v_k . z); tau_k is stored
// separately, in FP64 and rounded to the compute type.
#include "hh_internal.cuh"

namespace hh {
namespace {

constexpr int kPrepThreads = 256;

template <typename T>
__device__ inline double to_f64(T v) { return (double)v; }

// One CTA per reflector: FP64 sum of squares (fixed-order tree), tau, |v|,
// the first non-zero column (n for v = 0), then the zero-padded copy in the
// compute type.
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kPrepThreads)
prepare_reflectors_kernel(const Tin *__restrict__ U, int64_t ldu, int64_t n, int64_t ldv,
                          Tout *__restrict__ u_out, double *__restrict__ tau,
                          Tout *__restrict__ tau_t, double *__restrict__ vnorm,
                          int *__restrict__ start, int *__restrict__ flag) {
    __shared__ double red[kPrepThreads];
    __shared__ int first;
    const int64_t k = blockIdx.x;
    const Tin *v = U + k * ldu;
    if (threadIdx.x == 0) first = (int)n;
    __syncthreads();
    double s = 0.0;
    bool finite = true;
    int f = (int)n;
    for (int64_t j = threadIdx.x; j < n; j += kPrepThreads) {
        double x = to_f64(v[j]);
        finite &= isfinite(x);
        s += x * x;
        if (x != 0.0 && j < f) f = (int)j;
    }
    if (!finite) atomicOr(flag, 1);
    if (f < (int)n) atomicMin(&first, f);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kPrepThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double nn = red[0];
    const double t = nn > 0.0 ? 2.0 / nn : 0.0;
    if (threadIdx.x == 0) {
        tau[k] = t;
        tau_t[k] = (Tout)t;
        vnorm[k] = sqrt(nn);
        start[k] = first;
        if (!isfinite(nn)) atomicOr(flag, 1);
    }
    Tout *o = u_out + k * ldv;
    for (int64_t j = threadIdx.x; j < ldv; j += kPrepThreads)
        o[j] = j < n ? (Tout)v[j] : (Tout)0;
}

// Band of the reflector Gram matrix used by the blocked chain kernels:
// gram[k*16 + j] = v_k . v_{k+j} for j = 1..15 (FP64 sum, fixed-order tree),
// 0 where k + j >= h; gram[k*16] is unused (0).  One CTA per (k, j).
template <typename T>
__global__ void __launch_bounds__(kPrepThreads)
prepare_gram_kernel(const T *__restrict__ u, int64_t ldv, int64_t n, int64_t h,
                    T *__restrict__ gram) {
    __shared__ double red[kPrepThreads];
    const int64_t k = blockIdx.x;
    const int j = blockIdx.y;  // 0..15
    double s = 0.0;
    if (j > 0 && k + j < h) {
        const T *a = u + k * ldv, *b = u + (k + j) * ldv;
        for (int64_t i = threadIdx.x; i < n; i += kPrepThreads) s += (double)a[i] * (double)b[i];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kPrepThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) gram[k * 16 + j] = (T)red[0];
}

template <typename Tin, typename Tout>
__global__ void prepare_vectors_kernel(const Tin *__restrict__ d, const int8_t *__restrict__ sign,
                                       int64_t n, int64_t ldv, Tout *__restrict__ d_out,
                                       Tout *__restrict__ s_out, int *__restrict__ flag) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ldv;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (d_out) {
            double x = j < n ? to_f64(d[j]) : 0.0;
            if (!isfinite(x)) atomicOr(flag, 2);
            d_out[j] = (Tout)x;
        }
        if (s_out) {
            int s = j < n ? (int)sign[j] : 1;
            if (s != 1 && s != -1) atomicOr(flag, 4);
            s_out[j] = (Tout)(s < 0 ? -1.0 : 1.0);
        }
    }
}

template <typename T>
hh_status prepare_typed(Plan *p, const void *U, int64_t ldu, const void *d, const int8_t *sign,
                        int *flag, cudaStream_t st) {
    if (p->h > 0) {
        prepare_reflectors_kernel<T, T><<<(unsigned)p->h, kPrepThreads, 0, st>>>(
            (const T *)U, ldu, p->n, p->ldv, (T *)p->u, p->tau, (T *)p->tau_t, p->vnorm, p->start,
            flag);
        prepare_gram_kernel<T><<<dim3((unsigned)p->h, 16), kPrepThreads, 0, st>>>(
            (const T *)p->u, p->ldv, p->n, p->h, (T *)p->gram);
    }
    if (d || sign) {
        int blocks = (int)((p->ldv + 255) / 256);
        prepare_vectors_kernel<T, T><<<blocks, 256, 0, st>>>(
            (const T *)d, sign, p->n, p->ldv, (T *)p->d, (T *)p->sign, flag);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "prepare kernels");
    return HH_OK;
}

// After an update: a NaN or Inf seen by the prepare kernels (bits 1, 2 of
// *upd) becomes HH_ERR_NONFINITE in the status word, unless an earlier error
// is there; the flag is cleared for the next update.
__global__ void update_status_kernel(int *upd, int *err) {
    if (*upd & 3) atomicCAS(err, 0, (int)HH_ERR_NONFINITE);
    *upd = 0;
}

template <typename T>
hh_status update_typed(Plan *p, const void *U, int64_t ldu, const void *d, cudaStream_t st) {
    if (p->h > 0) {
        prepare_reflectors_kernel<T, T><<<(unsigned)p->h, kPrepThreads, 0, st>>>(
            (const T *)U, ldu, p->n, p->ldv, (T *)p->u, p->tau, (T *)p->tau_t, p->vnorm, p->start,
            p->upd);
        prepare_gram_kernel<T><<<dim3((unsigned)p->h, 16), kPrepThreads, 0, st>>>(
            (const T *)p->u, p->ldv, p->n, p->h, (T *)p->gram);
    }
    if (d) {  // the sign is kept: no sign input, no sign output
        int blocks = (int)((p->ldv + 255) / 256);
        prepare_vectors_kernel<T, T><<<blocks, 256, 0, st>>>((const T *)d, nullptr, p->n, p->ldv,
                                                             (T *)p->d, nullptr, p->upd);
    }
    update_status_kernel<<<1, 1, 0, st>>>(p->upd, p->err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "update kernels");
    return HH_OK;
}

}  // namespace

hh_status update_fused(Plan *p, const void *U, int64_t ldu, const void *d, cudaStream_t st) {
    if (p->dtype == HH_F32) return update_typed<float>(p, U, ldu, d, st);
    if (p->dtype == HH_F64) return update_typed<double>(p, U, ldu, d, st);
    return fail(HH_ERR_UNSUPPORTED, "update: F32 and F64 plans only");
}

hh_status prepare_fused(Plan *p, const void *U, int64_t ldu, const void *d, const int8_t *sign,
                        int *flag, cudaStream_t st) {
    if (p->dtype == HH_F32) return prepare_typed<float>(p, U, ldu, d, sign, flag, st);
    if (p->dtype == HH_F64) return prepare_typed<double>(p, U, ldu, d, sign, flag, st);
    return fail(HH_ERR_UNSUPPORTED, "fused path: dtype must be F32 or F64");
}

}  // namespace hh
