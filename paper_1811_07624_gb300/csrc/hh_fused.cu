// Dispatch of the fused apply to the F32 / F64 kernel instantiations.
#include "hh_internal.cuh"

namespace hh {

cudaError_t fused_dispatch_f32(hh_mode mode, const float *X, int64_t ldx, float *Y, int64_t ldy,
                               int64_t batch, int64_t n, const float *U, const float *tau, int64_t ldv, int h,
                               const float *gram, const float *sign, const float *d, int vec_ok,
                               int *err, int num_sms, cudaStream_t st, const int *start, float *P,
                               int64_t ldp);
cudaError_t fused_dispatch_f64(hh_mode mode, const double *X, int64_t ldx, double *Y,
                               int64_t ldy, int64_t batch, int64_t n, const double *U,
                               const double *tau, int64_t ldv, int h, const double *sign, const double *d,
                               int vec_ok, cudaStream_t st);

hh_status fused_apply(const Plan *p, hh_mode mode, const void *X, int64_t ldx, void *Y,
                      int64_t ldy, int64_t batch, cudaStream_t st) {
    return fused_apply_p(p, mode, X, ldx, Y, ldy, nullptr, 0, batch, st);
}

hh_status fused_apply_p(const Plan *p, hh_mode mode, const void *X, int64_t ldx, void *Y,
                        int64_t ldy, void *P, int64_t ldp, int64_t batch, cudaStream_t st) {
    const size_t es = dtype_size(p->dtype);
    const int vec = (int)(16 / es);
    const int vec_ok = ((uintptr_t)X % 16 == 0) && ((uintptr_t)Y % 16 == 0) && (ldx % vec == 0) &&
                       (ldy % vec == 0);
    cudaError_t e;
    if (p->dtype == HH_F32)
        e = fused_dispatch_f32(mode, (const float *)X, ldx, (float *)Y, ldy, batch, p->n,
                               (const float *)p->u, (const float *)p->tau_t, p->ldv, (int)p->h,
                               (const float *)p->gram, (const float *)p->sign,
                               (const float *)p->d,
                               vec_ok && (!P || ((uintptr_t)P % 16 == 0 && ldp % 4 == 0)),
                               p->err, p->num_sms, st, p->skip_prefix ? p->start : nullptr,
                               (float *)P, ldp);
    else if (p->dtype == HH_F64) {
        // p first (a W^T pass), so that Y may alias X
        e = cudaSuccess;
        if (P && mode == HH_MODE_SYM)
            e = fused_dispatch_f64(HH_MODE_WT, (const double *)X, ldx, (double *)P, ldp, batch,
                                   p->n, (const double *)p->u, (const double *)p->tau_t, p->ldv,
                                   (int)p->h, (const double *)p->sign, (const double *)p->d,
                                   vec_ok && (uintptr_t)P % 16 == 0 && ldp % 2 == 0, st);
        if (e == cudaSuccess)
            e = fused_dispatch_f64(mode, (const double *)X, ldx, (double *)Y, ldy, batch, p->n,
                                   (const double *)p->u, (const double *)p->tau_t, p->ldv,
                                   (int)p->h, (const double *)p->sign, (const double *)p->d,
                                   vec_ok, st);
    } else
        return fail(HH_ERR_UNSUPPORTED, "fused path: dtype must be F32 or F64");
    if (e != cudaSuccess) return cuda_fail(e, "fused apply launch");
    return HH_OK;
}

}  // namespace hh
