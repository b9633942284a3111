// Fast Mahalanobis distances (§IV-C): for a pair of rows (x_a, x_b),
//     d_S(x_a, x_b) = (x_a - x_b)^T S (x_a - x_b),  S = D W diag(d) W^T D,
// computed as sum_m d_m [W^T (sigma .* (x_a - x_b))]_m^2: one W^T chain
// (4nh operations, §II-A) per pair instead of a dense n x n product.
//
// Layout as the register chain of hh_fused.cuh: a CTA holds RG groups of G
// threads, each group RT pairs; the difference of the two gathered rows is
// formed in registers, the chain runs there, and the weighted sum of squares is
// reduced like a dot product.  Pair indices are bounds-checked in the kernel:
// an index outside [0, nrows) sets the plan's status word to
// HH_ERR_INVALID_ARG and that pair's output to NaN.
#include "hh_fused.cuh"

// (G, NG, RT, RG) of the F32 n <= 4096 configuration.
#ifndef HH_M4096_G
#define HH_M4096_G 256
#define HH_M4096_NG 4
#define HH_M4096_RT 4
#define HH_M4096_RG 2
#endif

namespace hh {
namespace {

template <typename T, int G, int NG, int RT, int RG>
__global__ void __launch_bounds__(G *RG)
mahalanobis_kernel(const T *X, int64_t ldx, int64_t nrows, const int64_t *__restrict__ ia,
                   const int64_t *__restrict__ ib, int64_t npairs, T *__restrict__ out, int n,
                   const T *__restrict__ U, const T *__restrict__ tau, int64_t ldv, int h,
                   const T *__restrict__ sign, const T *__restrict__ d, int vec_ok,
                   int *__restrict__ err) {
    using C = fused::Cfg<T, G, NG, RT, RG>;
    constexpr int VEC = C::VEC, E = C::E, NW = C::NW;
    __shared__ T red[2 * RG * RT * NW];
    const int tid = threadIdx.x;
    const int rg = tid / G;
    const int t = tid - rg * G;
    const int warp = t >> 5, lane = t & 31;
    const int64_t p0 = ((int64_t)blockIdx.x * RG + rg) * RT;
    int buf = 0;

    T x[RT][E];
    bool bad[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        const int64_t pr = p0 + r;
        int64_t a = 0, b = 0;
        bad[r] = false;
        if (pr < npairs) {
            a = ia[pr];
            b = ib[pr];
            if (a < 0 || a >= nrows || b < 0 || b >= nrows) {
                bad[r] = true;
                a = b = 0;
                if (t == 0) atomicExch(err, (int)HH_ERR_INVALID_ARG);
            }
        }
        const bool live = pr < npairs && !bad[r];
        const T *xa = X + a * ldx, *xb = X + b * ldx;
#pragma unroll
        for (int i = 0; i < NG; ++i) {
            const int col = (t + G * i) * VEC;
            T ga[VEC], gb[VEC];
            if (live && vec_ok && col + VEC <= n) {
                fused::ldg_granule<T>(xa + col, ga);
                fused::ldg_granule<T>(xb + col, gb);
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    const bool in = live && col + e < n;
                    ga[e] = in ? xa[col + e] : T(0);
                    gb[e] = in ? xb[col + e] : T(0);
                }
            }
#pragma unroll
            for (int e = 0; e < VEC; ++e) x[r][i * VEC + e] = ga[e] - gb[e];
        }
    }
    if (sign) fused::scale_cols<T, G, NG, RT, RG>(x, sign, t);
    for (int k = 0; k < h; ++k)
        fused::reflect<T, G, NG, RT, RG>(x, U + (size_t)k * ldv, __ldg(tau + k), t, lane, warp,
                                         rg, red, buf);
    // weighted sum of squares, reduced across the row group
    T dv[E];
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        T g[VEC];
        fused::ldg_granule<T>(d + (size_t)(t + G * i) * VEC, g);
#pragma unroll
        for (int e = 0; e < VEC; ++e) dv[i * VEC + e] = g[e];
    }
    T p[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        T s = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) s = fma(dv[e] * x[r][e], x[r][e], s);
        p[r] = s;
    }
    T v = fused::warp_reduce_rows<T, RT>(p, lane);
    constexpr int SH = 5 - fused::ilog2(RT);
    T tot[RT];
    if constexpr (NW == 1) {
#pragma unroll
        for (int r = 0; r < RT; ++r) tot[r] = __shfl_sync(0xffffffffu, v, r << SH);
    } else {
        if ((lane & ((1 << SH) - 1)) == 0)
            red[fused::red_index<RG, RT, NW>(buf, rg, lane >> SH, warp)] = v;
        __syncthreads();
        T q = lane < RT * NW ? red[fused::red_index<RG, RT, NW>(buf, rg, lane / NW, lane % NW)]
                             : T(0);
#pragma unroll
        for (int off = NW / 2; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
#pragma unroll
        for (int r = 0; r < RT; ++r) tot[r] = __shfl_sync(0xffffffffu, q, r * NW);
    }
    if (t == 0) {
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const int64_t pr = p0 + r;
            if (pr < npairs) out[pr] = bad[r] ? T(NAN) : tot[r];
        }
    }
}

template <typename T, int G, int NG, int RT, int RG>
cudaError_t launch(const Plan *p, const T *X, int64_t ldx, int64_t nrows, const int64_t *ia,
                   const int64_t *ib, int64_t npairs, T *out, int vec_ok, cudaStream_t st) {
    using C = fused::Cfg<T, G, NG, RT, RG>;
    const int64_t blocks = (npairs + C::ROWS - 1) / C::ROWS;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    mahalanobis_kernel<T, G, NG, RT, RG><<<(unsigned)blocks, C::THREADS, 0, st>>>(
        X, ldx, nrows, ia, ib, npairs, out, (int)p->n, (const T *)p->u, (const T *)p->tau_t,
        p->ldv, (int)p->h, (const T *)p->sign, (const T *)p->d, vec_ok, p->err);
    return cudaGetLastError();
}

template <typename T>
hh_status dispatch(const Plan *p, const void *X, int64_t ldx, int64_t nrows, const int64_t *ia,
                   const int64_t *ib, int64_t npairs, void *out, cudaStream_t st) {
    const int vec = 16 / (int)sizeof(T);
    const int vec_ok = ((uintptr_t)X % 16 == 0) && (ldx % vec == 0);
    const int64_t n = p->n;
    const T *x = (const T *)X;
    T *o = (T *)out;
    cudaError_t e;
#define HH_M(G, NG, RT, RG) e = launch<T, G, NG, RT, RG>(p, x, ldx, nrows, ia, ib, npairs, o, vec_ok, st)
    if (sizeof(T) == 4) {
        if (n <= 128) HH_M(32, 1, 4, 8);
        else if (n <= 256) HH_M(32, 2, 4, 8);
        else if (n <= 512) HH_M(32, 4, 4, 8);
        else if (n <= 1024) HH_M(64, 4, 4, 4);
        else if (n <= 2048) HH_M(128, 4, 4, 2);
        else if (n <= 4096) HH_M(HH_M4096_G, HH_M4096_NG, HH_M4096_RT, HH_M4096_RG);
        else return fail(HH_ERR_UNSUPPORTED, "mahalanobis: n = %lld above 4096 (F32)", (long long)n);
    } else {
        if (n <= 64) HH_M(32, 1, 2, 8);
        else if (n <= 128) HH_M(32, 2, 2, 8);
        else if (n <= 256) HH_M(32, 4, 2, 8);
        else if (n <= 512) HH_M(64, 4, 2, 4);
        else if (n <= 1024) HH_M(128, 4, 2, 2);
        else if (n <= 2048) HH_M(256, 4, 2, 2);
        else if (n <= 4096) HH_M(512, 4, 2, 1);
        else return fail(HH_ERR_UNSUPPORTED, "mahalanobis: n = %lld above 4096 (F64)", (long long)n);
    }
#undef HH_M
    if (e != cudaSuccess) return cuda_fail(e, "mahalanobis launch");
    return HH_OK;
}

}  // namespace

hh_status mahalanobis(const Plan *p, const void *X, int64_t ldx, int64_t nrows, const int64_t *ia,
                      const int64_t *ib, int64_t npairs, void *out, cudaStream_t st) {
    if (p->dtype == HH_F32) return dispatch<float>(p, X, ldx, nrows, ia, ib, npairs, out, st);
    if (p->dtype == HH_F64) return dispatch<double>(p, X, ldx, nrows, ia, ib, npairs, out, st);
    return fail(HH_ERR_UNSUPPORTED, "mahalanobis: F32 and F64 plans only");
}

}  // namespace hh
