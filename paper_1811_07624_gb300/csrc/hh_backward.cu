// Adjoint of the reflector chain (F32 / F64): gradients of a scalar loss L
// with respect to the input vectors, the reflector vectors v_k and the
// spectrum d, for the three forward modes of hh_fused.cuh.
//
// One reflector a_out = a_in - tau v (v . a_in), tau = 2 / (v . v) (§II-A,
// Eq. (2)), with G = dL/da_out, has
//     dL/da_in = H G = G - tau (v . G) v
//     dL/dv    = tau (alpha G - beta a_in) - tau^2 alpha beta v,
// where alpha = v . a_out = -(v . a_in) (since tau v.v = 2) and beta = v . G.
// The kernel walks the chain from the output back to the input; it never
// stores the intermediate vectors: a_in is recomputed from a_out by the
// involution H H = I (§II-A), so modes W and W^T start from the saved forward
// output.  Mode S (Eq. (21)) starts from the saved input, recomputes
// p = W^T (sigma .* x) and W (d .* p) forwards, then walks back through both
// halves (dL/dd = sum p .* dL/d(d .* p)).
//
// Mode 3 is the fast Mahalanobis distance of §IV-C, d_p = sum_m d_m z_m^2 with
// z = W^T (sigma .* (x_a - x_b)) for gathered row pairs: given g_p = dL/dd_p it
// recomputes z, seeds dL/dz = 2 g_p d .* z, adds g_p z .* z to dL/dd and walks
// back through W^T (no gradient for X).
//
// Reductions over the batch are deterministic: each CTA accumulates
// P_k = sum (alpha G - beta a_in) over its rows (in shared memory when it
// fits, else in its own slice of the scratch) and s_k = sum alpha beta, writes
// its partials to the scratch, and a second kernel sums the partials in a
// fixed order in FP64 and forms dL/dv_k = tau_k P_k - tau_k^2 s_k v_k.
#include <algorithm>
#include <type_traits>

#include "hh_fused.cuh"

// Mode S in F32 (allocating path): P_k through batch contractions (1) or
// accumulated per tile by the adjoint kernel (0).
#ifndef HH_BWD_SYM_CONTRACT
#define HH_BWD_SYM_CONTRACT 1
#endif
// The Mahalanobis gradient in F32 the same way (1) or per tile (0).
#ifndef HH_BWD_MAHA_CONTRACT
#define HH_BWD_MAHA_CONTRACT 1
#endif

// Rows per thread of the F32 adjoint for 128 < n <= 512 (and the default of the
// compile-time shape overrides below).
#ifndef HH_BWD_RT
#define HH_BWD_RT 4
#endif

namespace hh {
namespace bwd {

template <typename T, int G, int NG, int RT>
struct BCfg {
    static constexpr int VEC = fused::Granule<T>::N;
    static constexpr int E = NG * VEC;
    static constexpr int NW = G / 32;
    static constexpr int COVER = G * E;
    static constexpr int NV = 2 * RT;    // alpha and beta per row
    static constexpr int L = 32 / NV;    // lanes per value after the warp reduction
    static_assert(NV <= 32 && (NV & (NV - 1)) == 0, "2*RT must be a power of two <= 32");
};

template <typename T, int G, int NG, int RT>
__device__ __forceinline__ void load_rows(T (&a)[RT][BCfg<T, G, NG, RT>::E], const T *A, int64_t lda,
                                          int64_t r0, int64_t batch, int n, int t, int vec_ok) {
    constexpr int VEC = BCfg<T, G, NG, RT>::VEC;
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        const int64_t row = r0 + r;
        const T *ar = A + row * lda;
#pragma unroll
        for (int i = 0; i < NG; ++i) {
            const int col = (t + G * i) * VEC;
            T g[VEC];
            if (row < batch && vec_ok && col + VEC <= n) {
                fused::load_granule<T>(ar + col, g);
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e) g[e] = (row < batch && col + e < n) ? ar[col + e] : T(0);
            }
#pragma unroll
            for (int e = 0; e < VEC; ++e) a[r][i * VEC + e] = g[e];
        }
    }
}

template <typename T, int G, int NG, int RT>
__device__ __forceinline__ void load_cols(T (&c)[BCfg<T, G, NG, RT>::E], const T *__restrict__ s,
                                          int t) {
    constexpr int VEC = BCfg<T, G, NG, RT>::VEC;
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        T g[VEC];
        fused::ldg_granule<T>(s + (size_t)(t + G * i) * VEC, g);
#pragma unroll
        for (int e = 0; e < VEC; ++e) c[i * VEC + e] = g[e];
    }
}

// c0 += a0 * b0, c1 += a1 * b1: one packed FP32 FMA for float, two FMAs for
// double.  The per-element loops below go in pairs of columns.
__device__ __forceinline__ void fma_pair(float &c0, float &c1, float a0, float a1, float b0,
                                         float b1) {
    const float2 r = __ffma2_rn(make_float2(a0, a1), make_float2(b0, b1), make_float2(c0, c1));
    c0 = r.x;
    c1 = r.y;
}
__device__ __forceinline__ void fma_pair(double &c0, double &c1, double a0, double a1, double b0,
                                         double b1) {
    c0 = fma(a0, b0, c0);
    c1 = fma(a1, b1, c1);
}

// Sum NV per-thread values over the G threads of the CTA; every thread gets
// all NV sums.  One CTA barrier (double-buffered shared partials).
template <typename T, int G, int NG, int RT>
__device__ __forceinline__ void cta_sum(T (&p)[BCfg<T, G, NG, RT>::NV], int lane, int warp,
                                        T *red, int &buf) {
    using C = BCfg<T, G, NG, RT>;
    constexpr int NV = C::NV, NW = C::NW, L = C::L;
    T v = fused::warp_reduce_rows<T, NV>(p, lane);
    if constexpr (NW == 1) {
#pragma unroll
        for (int q = 0; q < NV; ++q) p[q] = __shfl_sync(0xffffffffu, v, q * L);
    } else {
        if ((lane & (L - 1)) == 0) red[fused::red_index<1, NV, NW>(buf, 0, lane / L, warp)] = v;
        __syncthreads();
        const int idx = lane / L, sub = lane & (L - 1);
        T q = T(0);
        for (int w = sub; w < NW; w += L) q += red[fused::red_index<1, NV, NW>(buf, 0, idx, w)];
#pragma unroll
        for (int off = L / 2; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
#pragma unroll
        for (int qq = 0; qq < NV; ++qq) p[qq] = __shfl_sync(0xffffffffu, q, qq * L);
        buf ^= 1;
    }
}

// Forward reflector on the rows in a (used to recompute mode S's states).
template <typename T, int G, int NG, int RT>
__device__ __forceinline__ void forward_step(T (&a)[RT][BCfg<T, G, NG, RT>::E],
                                             const T (&v)[BCfg<T, G, NG, RT>::E], T tk, int lane,
                                             int warp, T *red, int &buf) {
    using C = BCfg<T, G, NG, RT>;
    constexpr int E = C::E;
    static_assert(E % 2 == 0, "columns go in pairs");
    T p[C::NV];
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        T s0 = 0, s1 = 0;
#pragma unroll
        for (int e = 0; e < E; e += 2) fma_pair(s0, s1, a[r][e], a[r][e + 1], v[e], v[e + 1]);
        p[r] = s0 + s1;
        p[RT + r] = T(0);
    }
    cta_sum<T, G, NG, RT>(p, lane, warp, red, buf);
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        const T c = -tk * p[r];
#pragma unroll
        for (int e = 0; e < E; e += 2) fma_pair(a[r][e], a[r][e + 1], c, c, v[e], v[e + 1]);
    }
}

// One backward reflector step on (a = output of H_k, g = dL/d output).
// Leaves a = input of H_k, g = dL/d input; adds to the CTA's P_k accumulator
// (this thread's columns) and, on thread 0, to s_k.
template <typename T, int G, int NG, int RT>
__device__ __forceinline__ void backward_step(T (&a)[RT][BCfg<T, G, NG, RT>::E],
                                              T (&g)[RT][BCfg<T, G, NG, RT>::E],
                                              const T (&v)[BCfg<T, G, NG, RT>::E], T tk,
                                              T *__restrict__ pk, double *sk, int t, int lane,
                                              int warp, T *red, int &buf) {
    using C = BCfg<T, G, NG, RT>;
    constexpr int E = C::E, VEC = C::VEC;
    static_assert(E % 2 == 0, "columns go in pairs");
    T p[C::NV];
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        T sa0 = 0, sa1 = 0, sg0 = 0, sg1 = 0;
#pragma unroll
        for (int e = 0; e < E; e += 2) {
            fma_pair(sa0, sa1, a[r][e], a[r][e + 1], v[e], v[e + 1]);
            fma_pair(sg0, sg1, g[r][e], g[r][e + 1], v[e], v[e + 1]);
        }
        p[r] = sa0 + sa1;
        p[RT + r] = sg0 + sg1;
    }
    cta_sum<T, G, NG, RT>(p, lane, warp, red, buf);
    T acc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) acc[e] = T(0);
    double ab = 0.0;
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        const T alpha = p[r], beta = p[RT + r];
        const T ca = -tk * alpha, cb = -tk * beta, nb = -beta;
        ab += (double)alpha * (double)beta;
#pragma unroll
        for (int e = 0; e < E; e += 2) {
            fma_pair(a[r][e], a[r][e + 1], ca, ca, v[e], v[e + 1]);                // a_in
            fma_pair(acc[e], acc[e + 1], nb, nb, a[r][e], a[r][e + 1]);            // - beta a_in
            fma_pair(acc[e], acc[e + 1], alpha, alpha, g[r][e], g[r][e + 1]);      // + alpha G
            fma_pair(g[r][e], g[r][e + 1], cb, cb, v[e], v[e + 1]);                // H G
        }
    }
    if (threadIdx.x == 0) *sk += ab;
#pragma unroll
    for (int i = 0; i < NG; ++i)
#pragma unroll
        for (int e = 0; e < VEC; ++e) pk[(size_t)(t + G * i) * VEC + e] += acc[i * VEC + e];
}

// Sum the NV per-thread values in p over the G threads of the CTA (any power
// of two NV <= 32); every thread gets all NV sums.
template <typename T, int G, int NV>
__device__ __forceinline__ void cta_sum_n(T (&p)[NV], int lane, int warp, T *red, int &buf) {
    constexpr int NW = G / 32, L = 32 / NV;
    static_assert(NV <= 32 && (NV & (NV - 1)) == 0, "NV must be a power of two <= 32");
    T v = fused::warp_reduce_rows<T, NV>(p, lane);
    if constexpr (NW == 1) {
#pragma unroll
        for (int q = 0; q < NV; ++q) p[q] = __shfl_sync(0xffffffffu, v, q * L);
    } else {
        if ((lane & (L - 1)) == 0) red[fused::red_index<1, NV, NW>(buf, 0, lane / L, warp)] = v;
        __syncthreads();
        const int idx = lane / L, sub = lane & (L - 1);
        T q = T(0);
        for (int w = sub; w < NW; w += L) q += red[fused::red_index<1, NV, NW>(buf, 0, idx, w)];
#pragma unroll
        for (int off = L / 2; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
#pragma unroll
        for (int qq = 0; qq < NV; ++qq) p[qq] = __shfl_sync(0xffffffffu, q, qq * L);
        buf ^= 1;
    }
}

// BB backward reflector steps in one round (the Gram correction of the
// blocked forward chain, run backwards).  With (a, g) the round's starting
// state and k_0, k_1, ... the round's reflectors in walking order, the 2 BB
// dot products v_{k_i} . a and v_{k_i} . g of every row are taken at the
// start and reduced over the CTA together (one reduction per round instead
// of one per reflector); the values each step needs follow from
//     alpha_i = v_i . a - sum_{j<i} tau_j alpha_j (v_i . v_j)
//     beta_i  = v_i . g - sum_{j<i} tau_j beta_j  (v_i . v_j)
// (the Gram band v_k . v_{k+j}, j <= 15, of the plan).  The updates of a and
// g and the P_k accumulations then run reflector by reflector per column.
// k_i = k0 - i (DESC) or k0 + i.
template <typename T, int G, int NG, int RT, int BB, bool DESC>
__device__ __forceinline__ void backward_round(T (&a)[RT][BCfg<T, G, NG, RT>::E],
                                               T (&g)[RT][BCfg<T, G, NG, RT>::E],
                                               const T *__restrict__ V, int64_t ldv, int k0,
                                               const T *__restrict__ tau,
                                               const T *__restrict__ gram, T *accp, double *sacc,
                                               int t, int lane, int warp, T *red, int &buf) {
    using C = BCfg<T, G, NG, RT>;
    constexpr int VEC = C::VEC, COVER = C::COVER;
    constexpr int NVB = 2 * BB * RT;
    static_assert(VEC % 2 == 0, "columns go in pairs");
    auto kk = [&](int i) { return DESC ? k0 - i : k0 + i; };
    T p[NVB];
    {
        T s0[NVB], s1[NVB];
#pragma unroll
        for (int q = 0; q < NVB; ++q) s0[q] = s1[q] = T(0);
#pragma unroll
        for (int ig = 0; ig < NG; ++ig) {
            T vv[BB][VEC];
#pragma unroll
            for (int i = 0; i < BB; ++i)
                fused::ldg_granule<T>(V + (size_t)kk(i) * ldv + (size_t)(t + G * ig) * VEC, vv[i]);
#pragma unroll
            for (int e = 0; e < VEC; e += 2) {
                const int c = ig * VEC + e;
#pragma unroll
                for (int r = 0; r < RT; ++r)
#pragma unroll
                    for (int i = 0; i < BB; ++i) {
                        fma_pair(s0[i * RT + r], s1[i * RT + r], a[r][c], a[r][c + 1], vv[i][e],
                                 vv[i][e + 1]);
                        fma_pair(s0[(BB + i) * RT + r], s1[(BB + i) * RT + r], g[r][c], g[r][c + 1],
                                 vv[i][e], vv[i][e + 1]);
                    }
            }
        }
#pragma unroll
        for (int q = 0; q < NVB; ++q) p[q] = s0[q] + s1[q];
    }
    cta_sum_n<T, G, NVB>(p, lane, warp, red, buf);
    T tk[BB], al[BB][RT], be[BB][RT];
#pragma unroll
    for (int i = 0; i < BB; ++i) tk[i] = __ldg(tau + kk(i));
#pragma unroll
    for (int i = 0; i < BB; ++i) {
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            al[i][r] = p[i * RT + r];
            be[i][r] = p[(BB + i) * RT + r];
        }
#pragma unroll
        for (int j = 0; j < i; ++j) {
            // v_{k_i} . v_{k_j}: the band entry of the lower index at distance i - j
            const T gij = __ldg(gram + (size_t)(DESC ? kk(i) : kk(j)) * 16 + (i - j));
            const T tj = tk[j] * gij;
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                al[i][r] = fma(-tj, al[j][r], al[i][r]);
                be[i][r] = fma(-tj, be[j][r], be[i][r]);
            }
        }
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < BB; ++i) {
            double ab = 0.0;
#pragma unroll
            for (int r = 0; r < RT; ++r) ab += (double)al[i][r] * (double)be[i][r];
            sacc[kk(i)] += ab;
        }
    }
#pragma unroll
    for (int ig = 0; ig < NG; ++ig) {
        T vv[BB][VEC], acc[BB][VEC];
#pragma unroll
        for (int i = 0; i < BB; ++i) {
            fused::ldg_granule<T>(V + (size_t)kk(i) * ldv + (size_t)(t + G * ig) * VEC, vv[i]);
#pragma unroll
            for (int e = 0; e < VEC; ++e) acc[i][e] = T(0);
        }
#pragma unroll
        for (int e = 0; e < VEC; e += 2) {
            const int c = ig * VEC + e;
#pragma unroll
            for (int r = 0; r < RT; ++r)
#pragma unroll
                for (int i = 0; i < BB; ++i) {
                    const T alpha = al[i][r], nb = -be[i][r];
                    const T ca = -tk[i] * alpha, cb = -tk[i] * be[i][r];
                    fma_pair(a[r][c], a[r][c + 1], ca, ca, vv[i][e], vv[i][e + 1]);           // a_in
                    fma_pair(acc[i][e], acc[i][e + 1], nb, nb, a[r][c], a[r][c + 1]);        // - beta a_in
                    fma_pair(acc[i][e], acc[i][e + 1], alpha, alpha, g[r][c], g[r][c + 1]);  // + alpha G
                    fma_pair(g[r][c], g[r][c + 1], cb, cb, vv[i][e], vv[i][e + 1]);          // H G
                }
        }
#pragma unroll
        for (int i = 0; i < BB; ++i) {
            T *pk = accp + (size_t)kk(i) * COVER + (size_t)(t + G * ig) * VEC;
#pragma unroll
            for (int e = 0; e < VEC; ++e) pk[e] += acc[i][e];
        }
    }
}

// BB forward reflectors k0, k0 + 1, ... in one round: the BB dot products of
// every row are taken at the round's start and reduced together, and
// c_i = v_i . a - sum_{j<i} tau_j c_j (v_i . v_j) gives each reflector's value
// (the forward chain's Gram correction).
template <typename T, int G, int NG, int RT, int BB>
__device__ __forceinline__ void forward_round(T (&a)[RT][BCfg<T, G, NG, RT>::E],
                                              const T *__restrict__ V, int64_t ldv, int k0,
                                              const T *__restrict__ tau,
                                              const T *__restrict__ gram, int t, int lane,
                                              int warp, T *red, int &buf) {
    using C = BCfg<T, G, NG, RT>;
    constexpr int VEC = C::VEC;
    constexpr int NVB = BB * RT;
    static_assert(VEC % 2 == 0, "columns go in pairs");
    T p[NVB];
    {
        T s0[NVB], s1[NVB];
#pragma unroll
        for (int q = 0; q < NVB; ++q) s0[q] = s1[q] = T(0);
#pragma unroll
        for (int ig = 0; ig < NG; ++ig) {
            T vv[BB][VEC];
#pragma unroll
            for (int i = 0; i < BB; ++i)
                fused::ldg_granule<T>(V + (size_t)(k0 + i) * ldv + (size_t)(t + G * ig) * VEC, vv[i]);
#pragma unroll
            for (int e = 0; e < VEC; e += 2) {
                const int c = ig * VEC + e;
#pragma unroll
                for (int r = 0; r < RT; ++r)
#pragma unroll
                    for (int i = 0; i < BB; ++i)
                        fma_pair(s0[i * RT + r], s1[i * RT + r], a[r][c], a[r][c + 1], vv[i][e],
                                 vv[i][e + 1]);
            }
        }
#pragma unroll
        for (int q = 0; q < NVB; ++q) p[q] = s0[q] + s1[q];
    }
    cta_sum_n<T, G, NVB>(p, lane, warp, red, buf);
    T tk[BB], cf[BB][RT];
#pragma unroll
    for (int i = 0; i < BB; ++i) tk[i] = __ldg(tau + k0 + i);
#pragma unroll
    for (int i = 0; i < BB; ++i) {
#pragma unroll
        for (int r = 0; r < RT; ++r) cf[i][r] = p[i * RT + r];
#pragma unroll
        for (int j = 0; j < i; ++j) {
            const T tj = tk[j] * __ldg(gram + (size_t)(k0 + j) * 16 + (i - j));
#pragma unroll
            for (int r = 0; r < RT; ++r) cf[i][r] = fma(-tj, cf[j][r], cf[i][r]);
        }
    }
#pragma unroll
    for (int ig = 0; ig < NG; ++ig) {
        T vv[BB][VEC];
#pragma unroll
        for (int i = 0; i < BB; ++i)
            fused::ldg_granule<T>(V + (size_t)(k0 + i) * ldv + (size_t)(t + G * ig) * VEC, vv[i]);
#pragma unroll
        for (int e = 0; e < VEC; e += 2) {
            const int c = ig * VEC + e;
#pragma unroll
            for (int r = 0; r < RT; ++r)
#pragma unroll
                for (int i = 0; i < BB; ++i) {
                    const T cc = -tk[i] * cf[i][r];
                    fma_pair(a[r][c], a[r][c + 1], cc, cc, vv[i][e], vv[i][e + 1]);
                }
        }
    }
}

// The forward chain k = 0 .. h-1 on the rows in a, in rounds of BB.
template <typename T, int G, int NG, int RT, int BB>
__device__ __forceinline__ void forward_walk(T (&a)[RT][BCfg<T, G, NG, RT>::E],
                                             const T *__restrict__ V, int64_t ldv, int h,
                                             const T *__restrict__ tau,
                                             const T *__restrict__ gram, int t, int lane, int warp,
                                             T *red, int &buf) {
    using C = BCfg<T, G, NG, RT>;
    int k = 0;
    if constexpr (BB > 1)
        for (; k + BB <= h; k += BB)
            forward_round<T, G, NG, RT, BB>(a, V, ldv, k, tau, gram, t, lane, warp, red, buf);
    for (; k < h; ++k) {
        T v[C::E];
        load_cols<T, G, NG, RT>(v, V + (size_t)k * ldv, t);
        forward_step<T, G, NG, RT>(a, v, __ldg(tau + k), lane, warp, red, buf);
    }
}

// The backward walk over all h reflectors: k = h-1 .. 0 (DESC) or 0 .. h-1,
// in rounds of BB, the remainder one reflector per round.
template <typename T, int G, int NG, int RT, int BB, bool DESC>
__device__ __forceinline__ void backward_walk(T (&a)[RT][BCfg<T, G, NG, RT>::E],
                                              T (&g)[RT][BCfg<T, G, NG, RT>::E],
                                              const T *__restrict__ V, int64_t ldv, int h,
                                              const T *__restrict__ tau,
                                              const T *__restrict__ gram, T *accp, double *sacc,
                                              int t, int lane, int warp, T *red, int &buf) {
    using C = BCfg<T, G, NG, RT>;
    constexpr int E = C::E, COVER = C::COVER;
    int k = DESC ? h - 1 : 0, left = h;
    if constexpr (BB > 1) {
        for (; left >= BB; left -= BB, k += DESC ? -BB : BB)
            backward_round<T, G, NG, RT, BB, DESC>(a, g, V, ldv, k, tau, gram, accp, sacc, t, lane,
                                                   warp, red, buf);
    }
    for (; left > 0; --left, k += DESC ? -1 : 1) {
        T v[E];
        load_cols<T, G, NG, RT>(v, V + (size_t)k * ldv, t);
        backward_step<T, G, NG, RT>(a, g, v, __ldg(tau + k), accp + (size_t)k * COVER, sacc + k, t,
                                    lane, warp, red, buf);
    }
}

// Grid-persistent backward.  part: per CTA (h + 1) rows of COVER values
// (rows k < h: P_k; row h: the dL/dd partial), spart: per CTA h doubles (s_k).
// With SMEM the accumulators live in shared memory and are copied to `part`
// at the end; otherwise they are updated in place in `part`.
constexpr int kModeMahalanobis = 3;

// Rows x_ia[p] - x_ib[p] for the RT pairs of a tile (zero for pairs past the
// end; an index outside [0, nrows) gives a zero row and sets *err).
template <typename T, int G, int NG, int RT>
__device__ __forceinline__ void load_pair_rows(T (&a)[RT][BCfg<T, G, NG, RT>::E], const T *X,
                                               int64_t ldx, int64_t nrows,
                                               const int64_t *__restrict__ ia,
                                               const int64_t *__restrict__ ib, int64_t r0,
                                               int64_t npairs, int n, int t, int vec_ok,
                                               int *err) {
    constexpr int VEC = BCfg<T, G, NG, RT>::VEC;
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        const int64_t pr = r0 + r;
        int64_t ra = 0, rb = 0;
        bool live = pr < npairs;
        if (live) {
            ra = ia[pr];
            rb = ib[pr];
            if (ra < 0 || ra >= nrows || rb < 0 || rb >= nrows) {
                live = false;
                ra = rb = 0;
                if (t == 0) atomicExch(err, (int)HH_ERR_INVALID_ARG);
            }
        }
        const T *xa = X + ra * ldx, *xb = X + rb * ldx;
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
            for (int e = 0; e < VEC; ++e) a[r][i * VEC + e] = ga[e] - gb[e];
        }
    }
}

// PRE (mode S): the forward states come precomputed in two row-major
// batch x n arrays (leading dimension n): pre_a = W (d .* p) before the final
// sign and pre_p = p.  The kernel then skips its own forward recompute and
// holds no copy of p.  BB: reflectors per backward round (backward_round); FB:
// per round of mode 3's forward recompute (forward_round).
template <typename T, int MODE, int G, int NG, int RT, bool SMEM, bool PRE, int MINB, int BB,
          int FB>
__global__ void __launch_bounds__(G, MINB)
backward_kernel(const T *S, int64_t lds, const T *gY, int64_t ldg, T *gX, int64_t ldgx,
                int64_t batch, int n, const T *__restrict__ V, const T *__restrict__ tau,
                int64_t ldv, int h, const T *__restrict__ sign, const T *__restrict__ d,
                T *__restrict__ part, double *__restrict__ spart, int vec_ok,
                const int64_t *__restrict__ ia, const int64_t *__restrict__ ib, int64_t nrows,
                int *__restrict__ err, const T *__restrict__ pre_a, const T *__restrict__ pre_p,
                int pre_vec_ok, const T *__restrict__ gram) {
    using C = BCfg<T, G, NG, RT>;
    constexpr int E = C::E, VEC = C::VEC, COVER = C::COVER;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NVMAX = C::NV > 2 * BB * RT ? (C::NV > FB * RT ? C::NV : FB * RT)
                                              : (2 * BB * RT > FB * RT ? 2 * BB * RT : FB * RT);
    __shared__ T red[2 * NVMAX * C::NW];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    T *accp = SMEM ? reinterpret_cast<T *>(smem_raw) : part + (size_t)blockIdx.x * (h + 1) * COVER;
    double *sacc = spart + (size_t)blockIdx.x * h;
    // zero this thread's accumulator columns (same thread reads and writes them)
    for (int k = 0; k <= h; ++k)
#pragma unroll
        for (int i = 0; i < NG; ++i)
#pragma unroll
            for (int e = 0; e < VEC; ++e) accp[(size_t)k * COVER + (size_t)(t + G * i) * VEC + e] = T(0);
    if (t == 0)
        for (int k = 0; k < h; ++k) sacc[k] = 0.0;
    int buf = 0;
    const int64_t tiles = (batch + RT - 1) / RT;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t r0 = tile * RT;
        T a[RT][E], g[RT][E], v[E];
        T sg[PRE ? 1 : E];
        if constexpr (!PRE)
            if (sign) load_cols<T, G, NG, RT>(sg, sign, t);
        if constexpr (MODE == kModeMahalanobis) {
            // z = W^T (sigma .* (x_a - x_b)); dL/dz = 2 g_p d .* z; dL/dd += g_p z .* z
            static_assert(!PRE, "mode 3 recomputes z");
            load_pair_rows<T, G, NG, RT>(a, S, lds, nrows, ia, ib, r0, batch, n, t, vec_ok, err);
            if (sign)
#pragma unroll
                for (int r = 0; r < RT; ++r)
#pragma unroll
                    for (int e = 0; e < E; ++e) a[r][e] *= sg[e];
            forward_walk<T, G, NG, RT, FB>(a, V, ldv, h, tau, gram, t, lane, warp, red, buf);
            T dv[E], dd[E];
            load_cols<T, G, NG, RT>(dv, d, t);
#pragma unroll
            for (int e = 0; e < E; ++e) dd[e] = T(0);
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const T gp = r0 + r < batch ? gY[r0 + r] : T(0);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    dd[e] = fma(gp * a[r][e], a[r][e], dd[e]);
                    g[r][e] = T(2) * gp * dv[e] * a[r][e];
                }
            }
            T *dk = accp + (size_t)h * COVER;
#pragma unroll
            for (int i = 0; i < NG; ++i)
#pragma unroll
                for (int e = 0; e < VEC; ++e) dk[(size_t)(t + G * i) * VEC + e] += dd[i * VEC + e];
            backward_walk<T, G, NG, RT, BB, true>(a, g, V, ldv, h, tau, gram, accp, sacc, t, lane,
                                                  warp, red, buf);
            continue;
        }
        load_rows<T, G, NG, RT>(g, gY, ldg, r0, batch, n, t, vec_ok);
        T pvec[MODE == HH_MODE_SYM && !PRE ? RT : 1][MODE == HH_MODE_SYM && !PRE ? E : 1];
        if (PRE && MODE == HH_MODE_SYM) {
            load_rows<T, G, NG, RT>(a, pre_a, n, r0, batch, n, t, pre_vec_ok);
        } else if (MODE == HH_MODE_SYM) {
            // recompute p = W^T (sigma .* x), then W (d .* p)
            load_rows<T, G, NG, RT>(a, S, lds, r0, batch, n, t, vec_ok);
            if (sign)
#pragma unroll
                for (int r = 0; r < RT; ++r)
#pragma unroll
                    for (int e = 0; e < E; ++e) a[r][e] *= sg[e];
            for (int k = 0; k < h; ++k) {
                load_cols<T, G, NG, RT>(v, V + (size_t)k * ldv, t);
                forward_step<T, G, NG, RT>(a, v, __ldg(tau + k), lane, warp, red, buf);
            }
            T dv[E];
            load_cols<T, G, NG, RT>(dv, d, t);
#pragma unroll
            for (int r = 0; r < RT; ++r)
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if constexpr (MODE == HH_MODE_SYM && !PRE) pvec[r][e] = a[r][e];
                    a[r][e] *= dv[e];
                }
            for (int k = h - 1; k >= 0; --k) {
                load_cols<T, G, NG, RT>(v, V + (size_t)k * ldv, t);
                forward_step<T, G, NG, RT>(a, v, __ldg(tau + k), lane, warp, red, buf);
            }
        } else {
            load_rows<T, G, NG, RT>(a, S, lds, r0, batch, n, t, vec_ok);
        }
        // W part (modes W and S): y = sigma .* a^(1); walk k = 1..h
        if (MODE != HH_MODE_WT) {
            if (sign) {
                if constexpr (PRE) {
                    T s1[E];
                    load_cols<T, G, NG, RT>(s1, sign, t);
#pragma unroll
                    for (int r = 0; r < RT; ++r)
#pragma unroll
                        for (int e = 0; e < E; ++e) g[r][e] *= s1[e];
                } else {
#pragma unroll
                    for (int r = 0; r < RT; ++r)
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            if (MODE == HH_MODE_W) a[r][e] *= sg[e];
                            g[r][e] *= sg[e];
                        }
                }
            }
            backward_walk<T, G, NG, RT, BB, false>(a, g, V, ldv, h, tau, gram, accp, sacc, t, lane,
                                                   warp, red, buf);
        }
        if (MODE == HH_MODE_SYM) {
            // dL/dd += p .* dL/dq;  dL/dp = d .* dL/dq; continue from a = p
            T dv[E];
            load_cols<T, G, NG, RT>(dv, d, t);
            T dd[E];
#pragma unroll
            for (int e = 0; e < E; ++e) dd[e] = T(0);
            if constexpr (PRE) load_rows<T, G, NG, RT>(a, pre_p, n, r0, batch, n, t, pre_vec_ok);
#pragma unroll
            for (int r = 0; r < RT; ++r)
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if constexpr (MODE == HH_MODE_SYM && PRE) {
                        dd[e] = fma(a[r][e], g[r][e], dd[e]);
                    } else if constexpr (MODE == HH_MODE_SYM) {
                        dd[e] = fma(pvec[r][e], g[r][e], dd[e]);
                        a[r][e] = pvec[r][e];
                    }
                    g[r][e] *= dv[e];
                }
            T *dk = accp + (size_t)h * COVER;
#pragma unroll
            for (int i = 0; i < NG; ++i)
#pragma unroll
                for (int e = 0; e < VEC; ++e) dk[(size_t)(t + G * i) * VEC + e] += dd[i * VEC + e];
        }
        // W^T part (modes WT and S): walk k = h..1; then dL/dx = sigma .* g
        if (MODE != HH_MODE_W) {
            backward_walk<T, G, NG, RT, BB, true>(a, g, V, ldv, h, tau, gram, accp, sacc, t, lane,
                                                  warp, red, buf);
            if (sign) {
                if constexpr (PRE) {
                    T s1[E];
                    load_cols<T, G, NG, RT>(s1, sign, t);
#pragma unroll
                    for (int r = 0; r < RT; ++r)
#pragma unroll
                        for (int e = 0; e < E; ++e) g[r][e] *= s1[e];
                } else {
#pragma unroll
                    for (int r = 0; r < RT; ++r)
#pragma unroll
                        for (int e = 0; e < E; ++e) g[r][e] *= sg[e];
                }
            }
        }
        if (gX) {
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const int64_t row = r0 + r;
                if (row >= batch) continue;
                T *gr = gX + row * ldgx;
#pragma unroll
                for (int i = 0; i < NG; ++i) {
                    const int col = (t + G * i) * VEC;
                    T q[VEC];
#pragma unroll
                    for (int e = 0; e < VEC; ++e) q[e] = g[r][i * VEC + e];
                    if (vec_ok && col + VEC <= n) {
                        fused::store_granule<T>(gr + col, q);
                    } else {
#pragma unroll
                        for (int e = 0; e < VEC; ++e)
                            if (col + e < n) gr[col + e] = q[e];
                    }
                }
            }
        }
    }
    if (SMEM) {
        T *dst = part + (size_t)blockIdx.x * (h + 1) * COVER;
        for (int k = 0; k <= h; ++k)
#pragma unroll
            for (int i = 0; i < NG; ++i)
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    const size_t o = (size_t)k * COVER + (size_t)(t + G * i) * VEC + e;
                    dst[o] = accp[o];
                }
    }
}

// Fixed-order FP64 reduction of the partials.  Block (k, c) handles columns
// 32c .. 32c+31 of row k: k < h writes dL/dv_k (gU row k, length n), k = h
// writes dL/dd.  Each of 8 warps sums every 8th partial (warp w: parts
// w, w + 8, ...), then one warp adds the 8 sums in order; s_k is summed
// lane-strided with a fixed shuffle tree.  The result does not depend on the
// launch, only on nparts.
template <typename T>
__global__ void __launch_bounds__(256)
reduce_kernel(const T *__restrict__ part, const double *__restrict__ spart, int nparts, int cover,
              int n, int h, const T *__restrict__ V, int64_t ldv, const double *__restrict__ tau,
              T *gU, T *gd) {
    const int k = blockIdx.x;
    if (k < h && !gU) return;
    if (k == h && !gd) return;
    const int cx = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int j = blockIdx.y * 32 + cx;
    __shared__ double sh[8][33];
    __shared__ double ssum;
    double acc = 0.0;
    if (j < n)
        for (int p = grp; p < nparts; p += 8) acc += (double)part[((size_t)p * (h + 1) + k) * cover + j];
    sh[grp][cx] = acc;
    if (k < h && grp == 0) {
        double sk = 0.0;
        for (int p = cx; p < nparts; p += 32) sk += spart[(size_t)p * h + k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sk += __shfl_xor_sync(0xffffffffu, sk, off);
        if (cx == 0) ssum = sk;
    }
    __syncthreads();
    if (grp == 0 && j < n) {
        double tot = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) tot += sh[q][cx];
        if (k < h) {
            const double t = tau[k];
            gU[(size_t)k * n + j] = (T)(t * tot - t * t * ssum * (double)V[(size_t)k * ldv + j]);
        } else {
            gd[j] = (T)tot;
        }
    }
}

// Q = d .* P (rows of length n, leading dimension n, n % 4 == 0, both 16-byte
// aligned): one 4-column granule per thread, grid-stride.
__global__ void __launch_bounds__(256)
scale_cols_kernel(const float *__restrict__ P, float *__restrict__ Q, const float *__restrict__ d,
                  int64_t batch, int n) {
    const int ng = n / 4;
    const int64_t total = batch * ng;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % ng) * 4;
        const float4 x = reinterpret_cast<const float4 *>(P)[i];
        const float4 s = *reinterpret_cast<const float4 *>(d + c);
        reinterpret_cast<float4 *>(Q)[i] = make_float4(x.x * s.x, x.y * s.y, x.z * s.z, x.w * s.w);
    }
}

// ---- mode S in F32 through batch contractions ------------------------------------------
//
// With (A, G) the state a walk starts from and a^(k), g^(k) the state when it
// reaches reflector k, both are the start state minus multiples of the
// reflectors walked before: a^(k) = A - sum_{j before k} tau_j alpha_j v_j,
// and g^(k) likewise with beta.  So the per-reflector partial of the walk,
//     P_k = sum_rows alpha_k g^(k) - beta_k a^(k+)      (a^(k+): after H_k),
// splits into two products over the batch and a combination of reflectors:
//     P_k = G^T alpha_k - A^T beta_k - sum_{j before k} tau_j M[k][j] v_j
//           + sum_{j up to k} tau_j M[j][k] v_j,        M = alpha^T beta (h x h).
// The walk kernel writes each row's alpha_k and -beta_k and the state G of the
// second walk; G^T alpha - A^T beta and M are batch contractions (xty_kernel
// and mm_small_kernel, FP32 within a chunk of rows, FP64 across chunks in a
// fixed order), and combine_kernel forms
// dL/dv_k = tau_k P_k - tau_k^2 s_k v_k with s_k = M[k][k].  The same
// quantities as the per-tile accumulation, summed in a different order.

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One walk round without accumulation: as backward_round, then for each
// row r of the tile below the batch end and each reflector k of the round,
// store(r, k, alpha, beta) (called by thread r).
template <int G, int NG, int RT, int BB, bool DESC, typename Store>
__device__ __forceinline__ void walk_round(float (&a)[RT][BCfg<float, G, NG, RT>::E],
                                           float (&g)[RT][BCfg<float, G, NG, RT>::E],
                                           const float *__restrict__ V, int64_t ldv, int k0,
                                           const float *__restrict__ tau,
                                           const float *__restrict__ gram, Store &store,
                                           int64_t r0, int64_t batch, int t, int lane, int warp,
                                           float *red, int &buf) {
    using C = BCfg<float, G, NG, RT>;
    constexpr int VEC = C::VEC;
    constexpr int NVB = 2 * BB * RT;
    auto kk = [&](int i) { return DESC ? k0 - i : k0 + i; };
    float p[NVB];
    {
        float s0[NVB], s1[NVB];
#pragma unroll
        for (int q = 0; q < NVB; ++q) s0[q] = s1[q] = 0.f;
#pragma unroll
        for (int ig = 0; ig < NG; ++ig) {
            float vv[BB][VEC];
#pragma unroll
            for (int i = 0; i < BB; ++i)
                fused::ldg_granule<float>(V + (size_t)kk(i) * ldv + (size_t)(t + G * ig) * VEC, vv[i]);
#pragma unroll
            for (int e = 0; e < VEC; e += 2) {
                const int c = ig * VEC + e;
#pragma unroll
                for (int r = 0; r < RT; ++r)
#pragma unroll
                    for (int i = 0; i < BB; ++i) {
                        fma_pair(s0[i * RT + r], s1[i * RT + r], a[r][c], a[r][c + 1], vv[i][e],
                                 vv[i][e + 1]);
                        fma_pair(s0[(BB + i) * RT + r], s1[(BB + i) * RT + r], g[r][c], g[r][c + 1],
                                 vv[i][e], vv[i][e + 1]);
                    }
            }
        }
#pragma unroll
        for (int q = 0; q < NVB; ++q) p[q] = s0[q] + s1[q];
    }
    cta_sum_n<float, G, NVB>(p, lane, warp, red, buf);
    float tk[BB], al[BB][RT], be[BB][RT];
#pragma unroll
    for (int i = 0; i < BB; ++i) tk[i] = __ldg(tau + kk(i));
#pragma unroll
    for (int i = 0; i < BB; ++i) {
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            al[i][r] = p[i * RT + r];
            be[i][r] = p[(BB + i) * RT + r];
        }
#pragma unroll
        for (int j = 0; j < i; ++j) {
            const float gij = __ldg(gram + (size_t)(DESC ? kk(i) : kk(j)) * 16 + (i - j));
            const float tj = tk[j] * gij;
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                al[i][r] = fmaf(-tj, al[j][r], al[i][r]);
                be[i][r] = fmaf(-tj, be[j][r], be[i][r]);
            }
        }
    }
    // thread r stores row r's values (every thread holds all of them)
#pragma unroll
    for (int r = 0; r < RT; ++r)
        if (t == r && r0 + r < batch)
#pragma unroll
            for (int i = 0; i < BB; ++i) store(r, kk(i), al[i][r], be[i][r]);
#pragma unroll
    for (int ig = 0; ig < NG; ++ig) {
        float vv[BB][VEC];
#pragma unroll
        for (int i = 0; i < BB; ++i)
            fused::ldg_granule<float>(V + (size_t)kk(i) * ldv + (size_t)(t + G * ig) * VEC, vv[i]);
#pragma unroll
        for (int e = 0; e < VEC; e += 2) {
            const int c = ig * VEC + e;
#pragma unroll
            for (int r = 0; r < RT; ++r)
#pragma unroll
                for (int i = 0; i < BB; ++i) {
                    const float ca = -tk[i] * al[i][r], cb = -tk[i] * be[i][r];
                    fma_pair(a[r][c], a[r][c + 1], ca, ca, vv[i][e], vv[i][e + 1]);
                    fma_pair(g[r][c], g[r][c + 1], cb, cb, vv[i][e], vv[i][e + 1]);
                }
        }
    }
}

// A whole walk (k = 0 .. h-1, or h-1 .. 0 with DESC) in rounds of BB.
template <int G, int NG, int RT, int BB, bool DESC, typename Store>
__device__ __forceinline__ void walk_all(float (&a)[RT][BCfg<float, G, NG, RT>::E],
                                         float (&g)[RT][BCfg<float, G, NG, RT>::E],
                                         const float *__restrict__ V, int64_t ldv, int h,
                                         const float *__restrict__ tau,
                                         const float *__restrict__ gram, Store &&store, int64_t r0,
                                         int64_t batch, int t, int lane, int warp, float *red,
                                         int &buf) {
    int k = DESC ? h - 1 : 0, left = h;
    for (; left >= BB; left -= BB, k += DESC ? -BB : BB)
        walk_round<G, NG, RT, BB, DESC>(a, g, V, ldv, k, tau, gram, store, r0, batch, t, lane,
                                        warp, red, buf);
    for (; left > 0; --left, k += DESC ? -1 : 1)
        walk_round<G, NG, RT, 1, DESC>(a, g, V, ldv, k, tau, gram, store, r0, batch, t, lane, warp,
                                       red, buf);
}

// The two walks of the mode-S adjoint from the states q = W (d .* p) (before
// the final sign: rows of Qsrc, times qsign when given, i.e. sigma .* y for
// the forward output y) and P = p: the W walk from (q, sigma .* dL/dy), then
// dL/dd += p .* g, g = d .* g (written to Gd: the second walk's start), the
// W^T walk from (P, Gd), and dL/dx = sigma .* g.  Per CTA the dL/dd partial
// (COVER values) goes to ddpart.
template <int G, int NG, int RT, int BB>
__global__ void __launch_bounds__(G)
sym_walk_kernel(const float *gY, int64_t ldg, float *gX, int64_t ldgx, int64_t batch, int n,
                const float *__restrict__ V, const float *__restrict__ tau, int64_t ldv, int h,
                const float *__restrict__ sign, const float *__restrict__ d,
                const float *__restrict__ gram, const float *__restrict__ Qsrc, int64_t ldq,
                int qvec, const float *__restrict__ qsign, const float *__restrict__ P,
                int64_t ldp, float *__restrict__ Gd, float *__restrict__ AW,
                float *__restrict__ BW, float *__restrict__ AT, float *__restrict__ BT,
                float *__restrict__ ddpart, int vec_ok) {
    using C = BCfg<float, G, NG, RT>;
    constexpr int E = C::E, VEC = C::VEC, COVER = C::COVER;
    constexpr int NVMAX = 2 * BB * RT > C::NV ? 2 * BB * RT : C::NV;
    __shared__ float red[2 * NVMAX * C::NW];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    float dd[E];
#pragma unroll
    for (int e = 0; e < E; ++e) dd[e] = 0.f;
    int buf = 0;
    const int64_t tiles = (batch + RT - 1) / RT;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t r0 = tile * RT;
        float a[RT][E], g[RT][E];
        load_rows<float, G, NG, RT>(g, gY, ldg, r0, batch, n, t, vec_ok);
        load_rows<float, G, NG, RT>(a, Qsrc, ldq, r0, batch, n, t, qvec);
        if (sign) {
            float s1[E];
            load_cols<float, G, NG, RT>(s1, sign, t);
#pragma unroll
            for (int r = 0; r < RT; ++r)
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    g[r][e] *= s1[e];
                    if (qsign) a[r][e] *= s1[e];
                }
        }
        walk_all<G, NG, RT, BB, false>(
            a, g, V, ldv, h, tau, gram,
            [&](int r, int k, float al, float be) {
                AW[(size_t)(r0 + r) * h + k] = al;
                BW[(size_t)(r0 + r) * h + k] = -be;
            },
            r0, batch, t, lane, warp, red, buf);
        load_rows<float, G, NG, RT>(a, P, ldp, r0, batch, n, t, 1);
        {
            float dv[E];
            load_cols<float, G, NG, RT>(dv, d, t);
#pragma unroll
            for (int r = 0; r < RT; ++r)
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    dd[e] = fmaf(a[r][e], g[r][e], dd[e]);
                    g[r][e] *= dv[e];
                }
        }
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const int64_t row = r0 + r;
            if (row >= batch) continue;
#pragma unroll
            for (int i = 0; i < NG; ++i) {
                const int col = (t + G * i) * VEC;
                float q[VEC];
#pragma unroll
                for (int e = 0; e < VEC; ++e) q[e] = g[r][i * VEC + e];
                if (col + VEC <= n) fused::store_granule<float>(Gd + row * n + col, q);
            }
        }
        walk_all<G, NG, RT, BB, true>(
            a, g, V, ldv, h, tau, gram,
            [&](int r, int k, float al, float be) {
                AT[(size_t)(r0 + r) * h + k] = al;
                BT[(size_t)(r0 + r) * h + k] = -be;
            },
            r0, batch, t, lane, warp, red, buf);
        if (gX) {
            float s1[E];
            if (sign) load_cols<float, G, NG, RT>(s1, sign, t);
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const int64_t row = r0 + r;
                if (row >= batch) continue;
                float *gr = gX + row * ldgx;
#pragma unroll
                for (int i = 0; i < NG; ++i) {
                    const int col = (t + G * i) * VEC;
                    float q[VEC];
#pragma unroll
                    for (int e = 0; e < VEC; ++e)
                        q[e] = sign ? g[r][i * VEC + e] * s1[i * VEC + e] : g[r][i * VEC + e];
                    if (vec_ok && col + VEC <= n) {
                        fused::store_granule<float>(gr + col, q);
                    } else {
#pragma unroll
                        for (int e = 0; e < VEC; ++e)
                            if (col + e < n) gr[col + e] = q[e];
                    }
                }
            }
        }
    }
    float *dst = ddpart + (size_t)blockIdx.x * COVER;
#pragma unroll
    for (int i = 0; i < NG; ++i)
#pragma unroll
        for (int e = 0; e < VEC; ++e) dst[(size_t)(t + G * i) * VEC + e] = dd[i * VEC + e];
}

// Batch contraction out[c][k][j] = sum_pairs sum_{rows in chunk c} X[row][j] Y[row][k]
// (j < n, k < h), the sum of the first post_pairs pairs scaled by post0[j]
// when given.  X row-major
// with 16-byte aligned rows (n % 4 == 0), Y row-major batch x h (h % 4 == 0).
// A CTA of 64 threads computes a 128 x 32 (j x k) tile of one chunk, 8 x 8 per
// thread in FP32 registers, over slabs of 16 rows moved into shared memory by
// cp.async in a three-stage ring.  Chunk c covers rows [c*chunk, (c+1)*chunk).
struct XtyArgs {
    const float *X[4];
    int64_t ldx[4];
    const float *Y[4];
    int npairs;
    const float *post0;
    int post_pairs;
    int64_t rows, chunk;
    int n, h;
    float *out;  // nchunks x h x n
};
constexpr int kXtyJ = 128, kXtyK = 32, kXtySlab = 16, kXtyStages = 3;

__global__ void __launch_bounds__(64)
xty_kernel(const __grid_constant__ XtyArgs args) {
    __shared__ __align__(16) float xs[kXtyStages][kXtySlab][kXtyJ];
    __shared__ __align__(16) float ys[kXtyStages][kXtySlab][kXtyK];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int j0 = blockIdx.x * kXtyJ, k0 = blockIdx.y * kXtyK;
    const int64_t rb = (int64_t)blockIdx.z * args.chunk;
    const int64_t re = min(args.rows, rb + args.chunk);
    const int n = args.n, h = args.h;
    const int64_t nsl = re > rb ? (re - rb + kXtySlab - 1) / kXtySlab : 0;
    const int64_t total = nsl * args.npairs;
    float acc[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int w = 0; w < 8; ++w) acc[u][w] = 0.f;
    auto issue = [&](int64_t s) {
        const int stg = (int)(s % kXtyStages);
        const int pi = (int)(s / nsl);
        const int64_t r = rb + (s - pi * nsl) * kXtySlab;
        const float *X = args.X[pi], *Y = args.Y[pi];
        const int64_t ldx = args.ldx[pi];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int gi = t + 64 * q, rr = gi >> 5, cg = (gi & 31) * 4;
            const int64_t row = r + rr;
            const int col = j0 + cg;
            const bool ok = row < re && col < n;
            cp_async16(&xs[stg][rr][cg], ok ? X + row * ldx + col : X, ok ? 16 : 0);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int gi = t + 64 * q, rr = gi >> 3, kc = (gi & 7) * 4;
            const int64_t row = r + rr;
            const int k = k0 + kc;
            const bool ok = row < re && k < h;
            cp_async16(&ys[stg][rr][kc], ok ? Y + row * h + k : Y, ok ? 16 : 0);
        }
    };
    auto post_scale = [&]() {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int j = j0 + (u < 4 ? tx * 4 + u : 64 + tx * 4 + (u - 4));
            const float sc = j < n ? args.post0[j] : 0.f;
#pragma unroll
            for (int w = 0; w < 8; ++w) acc[u][w] *= sc;
        }
    };
#pragma unroll
    for (int s = 0; s < kXtyStages - 1; ++s) {
        if (s < total) issue(s);
        cp_async_commit();
    }
    for (int64_t s = 0; s < total; ++s) {
        if (s + kXtyStages - 1 < total) issue(s + kXtyStages - 1);
        cp_async_commit();
        cp_async_wait<kXtyStages - 1>();
        __syncthreads();
        if (s == nsl * args.post_pairs && args.post0) post_scale();
        const int stg = (int)(s % kXtyStages);
#pragma unroll
        for (int q = 0; q < kXtySlab; ++q) {
            const float4 xa = *reinterpret_cast<const float4 *>(&xs[stg][q][tx * 4]);
            const float4 xb = *reinterpret_cast<const float4 *>(&xs[stg][q][64 + tx * 4]);
            const float4 ya = *reinterpret_cast<const float4 *>(&ys[stg][q][ty * 4]);
            const float4 yb = *reinterpret_cast<const float4 *>(&ys[stg][q][16 + ty * 4]);
            const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
            const float yv[8] = {ya.x, ya.y, ya.z, ya.w, yb.x, yb.y, yb.z, yb.w};
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int w = 0; w < 8; w += 2)
                    fma_pair(acc[u][w], acc[u][w + 1], xv[u], xv[u], yv[w], yv[w + 1]);
        }
        __syncthreads();
    }
    cp_async_wait<0>();
    if (args.npairs == args.post_pairs && args.post0) post_scale();
    float *o = args.out + (size_t)blockIdx.z * h * n;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int j = j0 + (u < 4 ? tx * 4 + u : 64 + tx * 4 + (u - 4));
        if (j >= n) continue;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int k = k0 + (w < 4 ? ty * 4 + w : 16 + ty * 4 + (w - 4));
            if (k < h) o[(size_t)k * n + j] = acc[u][w];
        }
    }
}

// Small contraction out[b][k * h + j] = sum over the rows of block b of
// X[row][j] * Y[row][k] (j, k < h <= 64; X, Y row-major with leading
// dimensions ldx, ldy): 64-row slabs staged in shared memory, each thread
// accumulating its h^2 / 256 outputs in FP32.  Block b covers rows
// [b * chunk, (b + 1) * chunk).
constexpr int kMmRows = 64;
__global__ void __launch_bounds__(256)
mm_small_kernel(const float *__restrict__ X, int64_t ldx, const float *__restrict__ Y, int64_t ldy,
                int64_t rows, int64_t chunk, int h, float *__restrict__ out) {
    __shared__ float xs[kMmRows][64], ys[kMmRows][64];
    const int t = threadIdx.x;
    const int64_t rb = (int64_t)blockIdx.x * chunk;
    const int64_t re = min(rows, rb + chunk);
    const int hh = h * h;
    float acc[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) acc[m] = 0.f;
    for (int64_t r = rb; r < re; r += kMmRows) {
        for (int i = t; i < kMmRows * h; i += 256) {
            const int rr = i / h, c = i - rr * h;
            const int64_t row = r + rr;
            xs[rr][c] = row < re ? X[row * ldx + c] : 0.f;
            ys[rr][c] = row < re ? Y[row * ldy + c] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int q = t + 256 * m;
            if (q < hh) {
                const int k = q / h, j = q - k * h;
                float a = acc[m];
                for (int rr = 0; rr < kMmRows; ++rr) a = fmaf(xs[rr][j], ys[rr][k], a);
                acc[m] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int q = t + 256 * m;
        if (q < hh) out[(size_t)blockIdx.x * hh + q] = acc[m];
    }
}

// out[i] = sum over p of in[p * stride + i] in FP64 (i < count), p increasing
// within each of 8 interleaved groups, the groups added in order.  Block b
// handles i in [32b, 32b + 32).
__global__ void __launch_bounds__(256)
sum_parts_kernel(const float *__restrict__ in, int nparts, int64_t stride, int64_t count,
                 double *__restrict__ out) {
    __shared__ double sh[8][33];
    const int cx = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 32 + cx;
    double s = 0.0;
    if (i < count)
        for (int p = grp; p < nparts; p += 8) s += (double)in[(size_t)p * stride + i];
    sh[grp][cx] = s;
    __syncthreads();
    if (grp == 0 && i < count) {
        double tot = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) tot += sh[q][cx];
        out[i] = tot;
    }
}

// dL/dv_k (row k of gU) = tau_k P_k - tau_k^2 s_k v_k with
// P_k = R1[k] .* dscale + R2[k] + sum_i Cf[k][i] v_i (dscale, R2 optional),
// where for each walk given (MW: k = 0 .. h-1 first to last; MT: k = h-1 .. 0;
// the arrays hold -M, M[k][i] = sum_rows alpha_k beta_i)
//     Cf[k][i] += -tau_i M[k][i] [i walked before k] + tau_i M[i][k] [i walked up to k]
// and s_k = MW[k][k] + MT[k][k].  Block (h, *) writes dL/dd.  Grid (h + 1,
// column blocks of 256).
__global__ void __launch_bounds__(256)
combine_kernel(const double *__restrict__ R1, const float *__restrict__ dscale,
               const double *__restrict__ R2, const double *__restrict__ MW,
               const double *__restrict__ MT, const double *__restrict__ tau,
               const float *__restrict__ V, int64_t ldv, int n, int h, float *gU,
               const double *__restrict__ dd, float *gd) {
    const int k = blockIdx.x;
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    if (k == h) {
        if (gd && j < n) gd[j] = (float)dd[j];
        return;
    }
    if (!gU) return;
    extern __shared__ double cf[];  // h coefficients
    for (int i = threadIdx.x; i < h; i += blockDim.x) {
        double c = 0.0;
        if (MW && i < k) c += tau[i] * MW[(size_t)k * h + i];
        if (MW && i <= k) c -= tau[i] * MW[(size_t)i * h + k];
        if (MT && i > k) c += tau[i] * MT[(size_t)k * h + i];
        if (MT && i >= k) c -= tau[i] * MT[(size_t)i * h + k];
        cf[i] = c;
    }
    __syncthreads();
    if (j >= n) return;
    const double tk = tau[k];
    const double sk = -((MW ? MW[(size_t)k * h + k] : 0.0) + (MT ? MT[(size_t)k * h + k] : 0.0));
    double pk = R1[(size_t)k * n + j] * (dscale ? (double)dscale[j] : 1.0);
    if (R2) pk += R2[(size_t)k * n + j];
    for (int i = 0; i < h; ++i) pk += cf[i] * (double)V[(size_t)i * ldv + j];
    gU[(size_t)k * n + j] = (float)(tk * pk - tk * tk * sk * (double)V[(size_t)k * ldv + j]);
}

// Mode S, F32, allocating path, aligned dL/dy rows, h % 4 == 0, h <= 64:
// forward states by the fused kernels (q = sigma .* Ys when the forward
// output Ys is given, aligned), the walks by sym_walk_kernel, P_k by the
// batch contraction, combine_kernel.
template <int G, int NG, int RT, int BB>
hh_status sym_contract(const Plan *p, const float *S, int64_t lds, const float *gY, int64_t ldg,
                       float *gX, int64_t ldgx, float *gU, float *gd, int64_t batch, int vec_ok,
                       const float *Ys, int64_t ldy, const float *Pg, int64_t ldpg,
                       cudaStream_t st) {
    using C = BCfg<float, G, NG, RT>;
    const int h = (int)p->h, n = (int)p->n;
    const size_t bn = (size_t)batch * n, bh = (size_t)batch * h;
    auto kern = sym_walk_kernel<G, NG, RT, BB>;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, G, 0) != cudaSuccess || nb < 1) nb = 1;
    const int64_t tiles = (batch + RT - 1) / RT;
    const int nparts = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)p->num_sms * nb));
    const int jt = (n + kXtyJ - 1) / kXtyJ, kt = (h + kXtyK - 1) / kXtyK;
    const int64_t want = std::max<int64_t>(1, (int64_t)p->num_sms * 8 / (jt * kt));
    int64_t chunk = std::max<int64_t>(256, (batch + want - 1) / want);
    chunk = (chunk + kXtySlab - 1) / kXtySlab * kXtySlab;
    const int nchunks = (int)((batch + chunk - 1) / chunk);
    // one allocation, carved in 256-byte aligned pieces
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t oP = Pg ? 0 : take(bn * 4), oQ = Ys ? 0 : take(bn * 4), oGd = take(bn * 4);
    const size_t oAW = take(bh * 4), oBW = take(bh * 4), oAT = take(bh * 4), oBT = take(bh * 4);
    const size_t odd = take((size_t)nparts * C::COVER * 4);
    // the h x h contraction: blocks of mchunk rows, two per SM
    const int64_t mchunk = std::max<int64_t>(kMmRows, (batch + 2 * p->num_sms - 1) / (2 * p->num_sms));
    const int nmm = (int)((batch + mchunk - 1) / mchunk);
    const size_t oPp = take((size_t)nchunks * h * n * 4);
    const size_t oMp = take((size_t)nmm * 2 * h * h * 4);
    const size_t oPst = take((size_t)h * n * 8), oM = take((size_t)2 * h * h * 8),
                 odd64 = take((size_t)n * 8);
    char *base = nullptr;
    cudaError_t e = dev_malloc_async(reinterpret_cast<void **>(&base), off, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (adjoint work arrays)");
    auto F = [&](size_t o) { return reinterpret_cast<float *>(base + o); };
    auto D = [&](size_t o) { return reinterpret_cast<double *>(base + o); };
    // p = W^T (sigma .* x) (given as Pg, or computed); q = W (d .* p) without
    // the final sign (sigma .* Ys when the forward output is given)
    float *P = Pg ? const_cast<float *>(Pg) : F(oP), *Q = F(oQ);
    const int64_t ldp = Pg ? ldpg : n;
    hh_status hs = Pg ? HH_OK : fused_apply(p, HH_MODE_WT, S, lds, P, n, batch, st);
    if (hs == HH_OK && !Ys) {
        const unsigned fill =
            (unsigned)std::min<int64_t>(((int64_t)bn / 4 + 255) / 256, (int64_t)p->num_sms * 8);
        scale_cols_kernel<<<fill, 256, 0, st>>>(P, Q, (const float *)p->d, batch, n);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            Plan unsigned_plan = *p;
            unsigned_plan.sign = nullptr;
            hs = fused_apply(&unsigned_plan, HH_MODE_W, Q, n, Q, n, batch, st);
        }
    }
    const float *sign = (const float *)p->sign;
    // q = sigma .* y (Ys given) or the recomputed state (Q)
    const float *qsrc = Ys ? Ys : Q;
    const int64_t ldq = Ys ? ldy : n;
    if (hs == HH_OK && e == cudaSuccess) {
        kern<<<nparts, G, 0, st>>>(gY, ldg, gX, ldgx, batch, n, (const float *)p->u,
                                   (const float *)p->tau_t, p->ldv, h, sign, (const float *)p->d,
                                   (const float *)p->gram, qsrc, ldq, 1, Ys ? sign : nullptr, P,
                                   ldp, F(oGd), F(oAW), F(oBW), F(oAT), F(oBT), F(odd), vec_ok);
        e = cudaGetLastError();
    }
    if (hs == HH_OK && e == cudaSuccess && gU) {
        XtyArgs xa{};
        xa.X[0] = gY, xa.ldx[0] = ldg, xa.Y[0] = F(oAW);
        xa.X[1] = qsrc, xa.ldx[1] = ldq, xa.Y[1] = F(oBW);
        xa.X[2] = F(oGd), xa.ldx[2] = n, xa.Y[2] = F(oAT);
        xa.X[3] = P, xa.ldx[3] = ldp, xa.Y[3] = F(oBT);
        xa.npairs = 4;
        // sigma scales (sigma .* dL/dy)^T alpha, and (sigma .* y)^T beta when q = sigma .* y
        xa.post0 = sign;
        xa.post_pairs = Ys ? 2 : 1;
        xa.rows = batch;
        xa.chunk = chunk;
        xa.n = n;
        xa.h = h;
        xa.out = F(oPp);
        xty_kernel<<<dim3(jt, kt, nchunks), 64, 0, st>>>(xa);
        // -M[k][j] = sum (-beta_j) alpha_k: X = -beta, Y = alpha; the two walks'
        // partials one after the other (nmm x h x h each)
        for (int w = 0; w < 2; ++w)
            mm_small_kernel<<<nmm, 256, 0, st>>>(F(w ? oBT : oBW), h, F(w ? oAT : oAW), h, batch,
                                                 mchunk, h, F(oMp) + (size_t)w * nmm * h * h);
        const int64_t hn = (int64_t)h * n, hh = (int64_t)h * h;
        sum_parts_kernel<<<(unsigned)((hn + 31) / 32), 256, 0, st>>>(F(oPp), nchunks, hn, hn, D(oPst));
        for (int w = 0; w < 2; ++w)
            sum_parts_kernel<<<(unsigned)((hh + 31) / 32), 256, 0, st>>>(
                F(oMp) + (size_t)w * nmm * h * h, nmm, hh, hh, D(oM) + (size_t)w * h * h);
        e = cudaGetLastError();
    }
    if (hs == HH_OK && e == cudaSuccess && gd) {
        sum_parts_kernel<<<(unsigned)((n + 31) / 32), 256, 0, st>>>(F(odd), nparts, C::COVER, n,
                                                                    D(odd64));
        e = cudaGetLastError();
    }
    if (hs == HH_OK && e == cudaSuccess && (gU || gd)) {
        combine_kernel<<<dim3(h + 1, (n + 255) / 256), 256, (size_t)h * sizeof(double), st>>>(
            D(oPst), nullptr, nullptr, D(oM), D(oM) + (size_t)h * h, p->tau, (const float *)p->u,
            p->ldv, n, h, gU, D(odd64), gd);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaFreeAsync(base, st);
    if (e == cudaSuccess) e = e2;
    if (hs != HH_OK) return hs;
    if (e != cudaSuccess) return cuda_fail(e, "adjoint (mode S) launch");
    return HH_OK;
}

// The Mahalanobis gradient (mode 3) in the same form: per pair the kernel
// recomputes z = W^T (sigma .* (x_a - x_b)) (forward rounds of FB), stores it
// to Z, seeds g = 2 g_p d .* z, adds g_p z .* z to its dL/dd partial, and
// walks back (rounds of BB), storing Y[p] = [2 g_p alpha | -beta] (2h values)
// and alpha (h values) to Al.  With the walk's start state (z, 2 g_p d .* z),
//     P_k = d .* (Z^T (2 g_p alpha_k)) - Z^T beta_k + (reflector terms),
// so one contraction Z^T Y gives both parts.  An index outside [0, nrows)
// gives a zero row and sets *err, as in the recomputing kernel.
template <int G, int NG, int RT, int FB, int BB>
__global__ void __launch_bounds__(G)
maha_walk_kernel(const float *X, int64_t ldx, int64_t nrows, const int64_t *__restrict__ ia,
                 const int64_t *__restrict__ ib, const float *__restrict__ gp, int64_t npairs,
                 int n, const float *__restrict__ V, const float *__restrict__ tau, int64_t ldv,
                 int h, const float *__restrict__ sign, const float *__restrict__ d,
                 const float *__restrict__ gram, float *__restrict__ Z, float *__restrict__ Y,
                 float *__restrict__ Al, float *__restrict__ ddpart, int *__restrict__ err,
                 int vec_ok) {
    using C = BCfg<float, G, NG, RT>;
    constexpr int E = C::E, VEC = C::VEC, COVER = C::COVER;
    constexpr int NVA = 2 * BB * RT > C::NV ? 2 * BB * RT : C::NV;
    constexpr int NVMAX = NVA > FB * RT ? NVA : FB * RT;
    __shared__ float red[2 * NVMAX * C::NW];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    float dd[E];
#pragma unroll
    for (int e = 0; e < E; ++e) dd[e] = 0.f;
    int buf = 0;
    const int64_t tiles = (npairs + RT - 1) / RT;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t r0 = tile * RT;
        float a[RT][E], g[RT][E];
        load_pair_rows<float, G, NG, RT>(a, X, ldx, nrows, ia, ib, r0, npairs, n, t, vec_ok, err);
        if (sign) {
            float s1[E];
            load_cols<float, G, NG, RT>(s1, sign, t);
#pragma unroll
            for (int r = 0; r < RT; ++r)
#pragma unroll
                for (int e = 0; e < E; ++e) a[r][e] *= s1[e];
        }
        forward_walk<float, G, NG, RT, FB>(a, V, ldv, h, tau, gram, t, lane, warp, red, buf);
        float gw[RT];
#pragma unroll
        for (int r = 0; r < RT; ++r) gw[r] = r0 + r < npairs ? gp[r0 + r] : 0.f;
        {
            float dv[E];
            load_cols<float, G, NG, RT>(dv, d, t);
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const int64_t row = r0 + r;
#pragma unroll
                for (int i = 0; i < NG; ++i) {
                    const int col = (t + G * i) * VEC;
                    float q[VEC];
#pragma unroll
                    for (int e = 0; e < VEC; ++e) q[e] = a[r][i * VEC + e];
                    if (row < npairs && col + VEC <= n)
                        fused::store_granule<float>(Z + row * n + col, q);
                }
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    dd[e] = fmaf(gw[r] * a[r][e], a[r][e], dd[e]);
                    g[r][e] = 2.f * gw[r] * dv[e] * a[r][e];
                }
            }
        }
        walk_all<G, NG, RT, BB, true>(
            a, g, V, ldv, h, tau, gram,
            [&](int r, int k, float al, float be) {
                const size_t row = (size_t)(r0 + r);
                Y[row * 2 * h + k] = 2.f * gw[r] * al;
                Y[row * 2 * h + h + k] = -be;
                Al[row * h + k] = al;
            },
            r0, npairs, t, lane, warp, red, buf);
    }
    float *dst = ddpart + (size_t)blockIdx.x * COVER;
#pragma unroll
    for (int i = 0; i < NG; ++i)
#pragma unroll
        for (int e = 0; e < VEC; ++e) dst[(size_t)(t + G * i) * VEC + e] = dd[i * VEC + e];
}

// Mode 3, F32, aligned point rows, n % 4 == 0, h % 4 == 0, h <= 64, bounded
// work arrays: maha_walk_kernel, the contractions Z^T Y and -M = (-beta)^T
// alpha, combine_kernel with R1 = rows 0..h-1 scaled by d and R2 = rows
// h..2h-1.
template <int G, int NG, int RT, int FB, int BB>
hh_status maha_contract(const Plan *p, const float *X, int64_t ldx, int64_t nrows,
                        const int64_t *ia, const int64_t *ib, const float *gout, int64_t npairs,
                        float *gU, float *gd, int vec_ok, cudaStream_t st) {
    using C = BCfg<float, G, NG, RT>;
    const int h = (int)p->h, n = (int)p->n;
    auto kern = maha_walk_kernel<G, NG, RT, FB, BB>;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, G, 0) != cudaSuccess || nb < 1) nb = 1;
    const int64_t tiles = (npairs + RT - 1) / RT;
    const int nparts = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)p->num_sms * nb));
    const int h2 = 2 * h;
    const int jt = (n + kXtyJ - 1) / kXtyJ, kt = (h2 + kXtyK - 1) / kXtyK;
    const int64_t want = std::max<int64_t>(1, (int64_t)p->num_sms * 8 / (jt * kt));
    int64_t chunk = std::max<int64_t>(256, (npairs + want - 1) / want);
    chunk = (chunk + kXtySlab - 1) / kXtySlab * kXtySlab;
    const int nchunks = (int)((npairs + chunk - 1) / chunk);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t oZ = take((size_t)npairs * n * 4), oY = take((size_t)npairs * h2 * 4),
                 oAl = take((size_t)npairs * h * 4);
    const size_t odd = take((size_t)nparts * C::COVER * 4);
    const int64_t mchunk =
        std::max<int64_t>(kMmRows, (npairs + 2 * p->num_sms - 1) / (2 * p->num_sms));
    const int nmm = (int)((npairs + mchunk - 1) / mchunk);
    const size_t oRp = take((size_t)nchunks * h2 * n * 4), oMp = take((size_t)nmm * h * h * 4);
    const size_t oR = take((size_t)h2 * n * 8), oM = take((size_t)h * h * 8),
                 odd64 = take((size_t)n * 8);
    char *base = nullptr;
    cudaError_t e = dev_malloc_async(reinterpret_cast<void **>(&base), off, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (gradient work arrays)");
    auto F = [&](size_t o) { return reinterpret_cast<float *>(base + o); };
    auto D = [&](size_t o) { return reinterpret_cast<double *>(base + o); };
    kern<<<nparts, G, 0, st>>>(X, ldx, nrows, ia, ib, gout, npairs, n, (const float *)p->u,
                               (const float *)p->tau_t, p->ldv, h, (const float *)p->sign,
                               (const float *)p->d, (const float *)p->gram, F(oZ), F(oY), F(oAl),
                               F(odd), p->err, vec_ok);
    e = cudaGetLastError();
    if (e == cudaSuccess && gU) {
        XtyArgs xa{};
        xa.X[0] = F(oZ), xa.ldx[0] = n, xa.Y[0] = F(oY);
        xa.npairs = 1;
        xa.rows = npairs;
        xa.chunk = chunk;
        xa.n = n;
        xa.h = h2;
        xa.out = F(oRp);
        xty_kernel<<<dim3(jt, kt, nchunks), 64, 0, st>>>(xa);
        // -M[k][j] = sum (-beta_j) alpha_k: X = -beta (columns h.. of Y), Y = alpha
        mm_small_kernel<<<nmm, 256, 0, st>>>(F(oY) + h, h2, F(oAl), h, npairs, mchunk, h, F(oMp));
        const int64_t rn = (int64_t)h2 * n, hh = (int64_t)h * h;
        sum_parts_kernel<<<(unsigned)((rn + 31) / 32), 256, 0, st>>>(F(oRp), nchunks, rn, rn, D(oR));
        sum_parts_kernel<<<(unsigned)((hh + 31) / 32), 256, 0, st>>>(F(oMp), nmm, hh, hh, D(oM));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && gd) {
        sum_parts_kernel<<<(unsigned)((n + 31) / 32), 256, 0, st>>>(F(odd), nparts, C::COVER, n,
                                                                    D(odd64));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && (gU || gd)) {
        combine_kernel<<<dim3(h + 1, (n + 255) / 256), 256, (size_t)h * sizeof(double), st>>>(
            D(oR), (const float *)p->d, D(oR) + (size_t)h * n, nullptr, D(oM), p->tau,
            (const float *)p->u, p->ldv, n, h, gU, D(odd64), gd);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaFreeAsync(base, st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return cuda_fail(e, "Mahalanobis gradient launch");
    return HH_OK;
}

struct PairArgs {
    const int64_t *ia = nullptr, *ib = nullptr;
    int64_t nrows = 0;
    const void *ysym = nullptr;  // mode S: the forward output y = S_bar x, or null
    int64_t ldy = 0;
    const void *psym = nullptr;  // mode S: p = W^T (sigma .* x), or null (then S is x)
    int64_t ldp = 0;
};

template <typename T, int G, int NG, int RT, int MINB = 1, int BB = 1, int FB = 1>
hh_status run(const Plan *p, int mode, const T *S, int64_t lds, const T *gY, int64_t ldg,
              T *gX, int64_t ldgx, T *gU, T *gd, int64_t batch, int vec_ok, void *scratch,
              size_t scratch_bytes, PairArgs pa, cudaStream_t st) {
    using C = BCfg<T, G, NG, RT>;
    const int h = (int)p->h, n = (int)p->n;
    const size_t acc_bytes = (size_t)(h + 1) * C::COVER * sizeof(T);
    const bool use_smem = acc_bytes <= 48 * 1024;
    auto pick = [&](auto kern, size_t smem) -> int {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, G, smem) != cudaSuccess || nb < 1)
            nb = 1;
        return nb;
    };
    const int64_t tiles = (batch + RT - 1) / RT;
    // Mode S in F32 on the allocating path: the forward states p and W (d .* p)
    // come from the fused forward kernels (blocked rounds), and the adjoint
    // kernel reads them instead of recomputing the chain one reflector per
    // round.  Bounded to kPreMaxBytes of extra device memory; above it, or with
    // a caller's scratch (no allocation allowed), the kernel recomputes.  (For
    // mode 3 the gathered differences would cost more HBM traffic than the
    // recompute saves.)
    constexpr size_t kPreMaxBytes = size_t(3) << 30;
    const size_t pre_bytes = (size_t)batch * n * sizeof(T) * 3;
    const bool pre = std::is_same<T, float>::value && !scratch && batch > 0 && n % 4 == 0 &&
                     mode == HH_MODE_SYM && pre_bytes <= kPreMaxBytes;
    auto launch = [&](auto kern, size_t smem, bool with_pre) -> hh_status {
        int nparts = (int)std::min<int64_t>(tiles, (int64_t)p->num_sms * pick(kern, smem));
        if (nparts < 1) nparts = 1;
        const size_t need = (size_t)nparts * (acc_bytes + (size_t)h * sizeof(double));
        void *buf = scratch;
        bool own = false;
        if (!buf) {
            cudaError_t e = dev_malloc_async(&buf, need, st);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (backward scratch)");
            own = true;
        } else if (need > scratch_bytes) {
            // fewer CTAs, each covering more rows, so the partials fit
            const size_t per = acc_bytes + (size_t)h * sizeof(double);
            nparts = (int)(scratch_bytes / per);
            if (nparts < 1)
                return fail(HH_ERR_INVALID_ARG,
                            "backward: one CTA's partial sums need %zu bytes of scratch, more "
                            "than the %zu bytes available (h or n too large)",
                            per, scratch_bytes);
        }
        T *part = reinterpret_cast<T *>(buf);
        double *spart = reinterpret_cast<double *>(reinterpret_cast<char *>(buf) +
                                                   (size_t)nparts * acc_bytes);
        T *pre_buf = nullptr, *pre_a = nullptr, *pre_p = nullptr;
        cudaError_t e = cudaSuccess;
        hh_status hs = HH_OK;
        if (with_pre) {
            e = dev_malloc_async(reinterpret_cast<void **>(&pre_buf), pre_bytes, st);
            if (e != cudaSuccess) {
                if (own) cudaFreeAsync(buf, st);
                return cuda_fail(e, "cudaMallocAsync (backward forward states)");
            }
            const unsigned fill =
                (unsigned)std::min<int64_t>((batch * (n / 4) + 255) / 256, (int64_t)p->num_sms * 8);
            // p = W^T (sigma .* x); q = W (d .* p) without the final sign
            pre_p = pre_buf;
            pre_a = pre_buf + (size_t)batch * n;
            hs = fused_apply(p, HH_MODE_WT, S, lds, pre_p, n, batch, st);
            if (hs == HH_OK) {
                scale_cols_kernel<<<fill, 256, 0, st>>>((const float *)pre_p, (float *)pre_a,
                                                        (const float *)p->d, batch, n);
                e = cudaGetLastError();
            }
            if (hs == HH_OK && e == cudaSuccess) {
                Plan unsigned_plan = *p;
                unsigned_plan.sign = nullptr;
                hs = fused_apply(&unsigned_plan, HH_MODE_W, pre_a, n, pre_a, n, batch, st);
            }
        }
        if (hs == HH_OK && e == cudaSuccess) {
            kern<<<nparts, G, smem, st>>>(S, lds, gY, ldg, gX, ldgx, batch, n, (const T *)p->u,
                                          (const T *)p->tau_t, p->ldv, h, (const T *)p->sign,
                                          (const T *)p->d, part, spart, vec_ok, pa.ia, pa.ib,
                                          pa.nrows, p->err, pre_a, pre_p, 1,
                                          (const T *)p->gram);
            e = cudaGetLastError();
        }
        if (hs == HH_OK && e == cudaSuccess && (gU || gd))
            reduce_kernel<T><<<dim3(h + 1, (n + 31) / 32), 256, 0, st>>>(
                part, spart, nparts, C::COVER, n, h, (const T *)p->u, p->ldv, p->tau, gU, gd);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (pre_buf) {
            cudaError_t e2 = cudaFreeAsync(pre_buf, st);
            if (e == cudaSuccess) e = e2;
        }
        if (own) {
            cudaError_t e2 = cudaFreeAsync(buf, st);
            if (e == cudaSuccess) e = e2;
        }
        if (hs != HH_OK) return hs;
        if (e != cudaSuccess) return cuda_fail(e, "backward launch");
        return HH_OK;
    };
// Mode S without PRE holds p as well: one reflector per round there (the
// blocked round's extra registers would spill).
#define HH_BWD_KERN(M, PRE, BBX)                                                              \
    if (use_smem) {                                                                           \
        return launch(backward_kernel<T, M, G, NG, RT, true, PRE, MINB, BBX, FB>, acc_bytes, PRE); \
    } else {                                                                                  \
        return launch(backward_kernel<T, M, G, NG, RT, false, PRE, MINB, BBX, FB>, 0, PRE);       \
    }
    switch (mode) {
        case HH_MODE_W: HH_BWD_KERN(HH_MODE_W, false, BB)
        case HH_MODE_WT: HH_BWD_KERN(HH_MODE_WT, false, BB)
        case HH_MODE_SYM:
            if constexpr (std::is_same<T, float>::value) {
#if HH_BWD_SYM_CONTRACT
                if (pre && vec_ok && h % 4 == 0 && h <= 64) {
                    const bool yok = pa.ysym && (uintptr_t)pa.ysym % 16 == 0 && pa.ldy % 4 == 0;
                    return sym_contract<G, NG, RT, BB>(
                        p, S, lds, gY, ldg, gX, ldgx, gU, gd, batch, vec_ok,
                        yok ? (const float *)pa.ysym : nullptr, yok ? pa.ldy : 0,
                        (const float *)pa.psym, pa.ldp, st);
                }
#endif
                if (pre) HH_BWD_KERN(HH_MODE_SYM, true, BB)
            }
            HH_BWD_KERN(HH_MODE_SYM, false, 1)
        default:
#if HH_BWD_MAHA_CONTRACT
            if constexpr (std::is_same<T, float>::value) {
                const size_t work = (size_t)batch * (n + 3 * h) * sizeof(float);
                if (!scratch && vec_ok && n % 4 == 0 && h % 4 == 0 && h <= 64 && batch > 0 &&
                    work <= kPreMaxBytes)
                    return maha_contract<G, NG, RT, FB, BB>(p, S, lds, pa.nrows, pa.ia, pa.ib, gY,
                                                            batch, gU, gd, vec_ok, st);
            }
#endif
            HH_BWD_KERN(kModeMahalanobis, false, BB)
    }
#undef HH_BWD_KERN
}

template <typename T>
hh_status dispatch(const Plan *p, int mode, const void *S, int64_t lds, const void *gY,
                   int64_t ldg, void *gX, int64_t ldgx, void *gU, void *gd, int64_t batch,
                   void *scratch, size_t scratch_bytes, PairArgs pa, cudaStream_t st) {
    const int64_t n = p->n;
    const int vec = 16 / (int)sizeof(T);
    // mode 3 reads gY as one value per pair: only S's alignment matters there
    const int vec_ok = ((uintptr_t)S % 16 == 0) && lds % vec == 0 &&
                       (mode == kModeMahalanobis ||
                        ((uintptr_t)gY % 16 == 0 && ldg % vec == 0 &&
                         (!gX || ((uintptr_t)gX % 16 == 0 && ldgx % vec == 0))));
#define HH_RUN(G, NG, RT) HH_RUN_B(G, NG, RT, 1, 1, 1)
#define HH_RUN_B(G, NG, RT, MINB, BB, FB)                                                   \
    return run<T, G, NG, RT, MINB, BB, FB>(p, mode, (const T *)S, lds, (const T *)gY, ldg, (T *)gX, ldgx, \
                             (T *)gU, (T *)gd, batch, vec_ok, scratch, scratch_bytes, pa, st)
    if constexpr (sizeof(T) == 4) {
        if (n <= 128) HH_RUN(32, 1, 4);
#ifndef HH_BWD256_G
#define HH_BWD256_G 32
#define HH_BWD256_NG 2
#define HH_BWD256_RT HH_BWD_RT
#endif
#ifndef HH_BWD256_MINB
#define HH_BWD256_MINB 1
#endif
#ifndef HH_BWD1024_MINB
#define HH_BWD1024_MINB 1
#endif
#ifndef HH_BWD256_BB
#define HH_BWD256_BB 2
#endif
#ifndef HH_BWD256_FB
#define HH_BWD256_FB 4
#endif
#ifndef HH_BWD1024_BB
#define HH_BWD1024_BB 2
#endif
#ifndef HH_BWD1024_FB
#define HH_BWD1024_FB 1
#endif
#ifndef HH_BWD1024_G
// 4 rows x 16 columns per thread, two warps per row (measured 14% faster than
// 128 threads x 8 columns for the adjoint of S at n = 1024, h = 32)
#define HH_BWD1024_G 64
#define HH_BWD1024_NG 4
#define HH_BWD1024_RT 4
#endif
        if (n <= 256) HH_RUN_B(HH_BWD256_G, HH_BWD256_NG, HH_BWD256_RT, HH_BWD256_MINB, HH_BWD256_BB,
                                HH_BWD256_FB);
        if (n <= 512) HH_RUN(64, 2, HH_BWD_RT);
        if (n <= 1024) HH_RUN_B(HH_BWD1024_G, HH_BWD1024_NG, HH_BWD1024_RT, HH_BWD1024_MINB,
                                 HH_BWD1024_BB, HH_BWD1024_FB);
        if (n <= 2048) HH_RUN(256, 2, 2);
        if (n <= 4096) HH_RUN(512, 2, 2);
    } else {
        if (n <= 64) HH_RUN(32, 1, 4);
        if (n <= 128) HH_RUN(32, 2, 2);
        if (n <= 256) HH_RUN(64, 2, 2);
        if (n <= 512) HH_RUN(128, 2, 2);
        if (n <= 1024) HH_RUN(256, 2, 2);
        if (n <= 2048) HH_RUN(512, 2, 2);
    }
#undef HH_RUN
#undef HH_RUN_B
    return fail(HH_ERR_UNSUPPORTED, "backward: n = %lld is above this build's limit (%d)",
                (long long)n, sizeof(T) == 4 ? 4096 : 2048);
}

}  // namespace bwd

hh_status backward(const Plan *p, hh_mode mode, const void *S, int64_t lds, const void *gY,
                   int64_t ldg, void *gX, int64_t ldgx, void *gU, void *gd, int64_t batch,
                   void *scratch, size_t scratch_bytes, cudaStream_t st) {
    bwd::PairArgs pa;
    if (p->dtype == HH_F32)
        return bwd::dispatch<float>(p, mode, S, lds, gY, ldg, gX, ldgx, gU, gd, batch, scratch,
                                    scratch_bytes, pa, st);
    if (p->dtype == HH_F64)
        return bwd::dispatch<double>(p, mode, S, lds, gY, ldg, gX, ldgx, gU, gd, batch, scratch,
                                     scratch_bytes, pa, st);
    return fail(HH_ERR_UNSUPPORTED, "backward: F32 and F64 plans only");
}

hh_status backward_sym_y(const Plan *p, const void *X, int64_t ldx, const void *Y, int64_t ldy,
                         const void *gY, int64_t ldg, void *gX, int64_t ldgx, void *gU, void *gd,
                         int64_t batch, cudaStream_t st) {
    bwd::PairArgs pa;
    pa.ysym = Y;
    pa.ldy = ldy;
    if (p->dtype == HH_F32)
        return bwd::dispatch<float>(p, HH_MODE_SYM, X, ldx, gY, ldg, gX, ldgx, gU, gd, batch,
                                    nullptr, 0, pa, st);
    if (p->dtype == HH_F64)
        return bwd::dispatch<double>(p, HH_MODE_SYM, X, ldx, gY, ldg, gX, ldgx, gU, gd, batch,
                                     nullptr, 0, pa, st);
    return fail(HH_ERR_UNSUPPORTED, "backward: F32 and F64 plans only");
}

hh_status backward_sym_py(const Plan *p, const void *P, int64_t ldp, const void *Y, int64_t ldy,
                          const void *gY, int64_t ldg, void *gX, int64_t ldgx, void *gU, void *gd,
                          int64_t batch, cudaStream_t st) {
    const int64_t n = p->n, h = p->h;
    const auto al = [](const void *q, int64_t ld) { return (uintptr_t)q % 16 == 0 && ld % 4 == 0; };
    // the contraction path reads p and y directly
    const bool direct = p->dtype == HH_F32 && batch > 0 && n % 4 == 0 && h % 4 == 0 && h <= 64 &&
                        (size_t)batch * n * 4 * 3 <= (size_t(3) << 30) && al(P, ldp) &&
                        al(Y, ldy) && al(gY, ldg) && (!gX || al(gX, ldgx));
    bwd::PairArgs pa;
    pa.ysym = Y;
    pa.ldy = ldy;
    if (direct) {
        pa.psym = P;
        pa.ldp = ldp;
        return bwd::dispatch<float>(p, HH_MODE_SYM, nullptr, ldp, gY, ldg, gX, ldgx, gU, gd, batch,
                                    nullptr, 0, pa, st);
    }
    // otherwise the input first: x = sigma .* (W p), W orthogonal
    if (p->dtype != HH_F32 && p->dtype != HH_F64)
        return fail(HH_ERR_UNSUPPORTED, "backward: F32 and F64 plans only");
    const size_t es = dtype_size(p->dtype);
    void *X = nullptr;
    if (batch > 0) {
        cudaError_t e = dev_malloc_async(&X, (size_t)batch * n * es, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (backward input)");
    }
    hh_status hs = batch > 0 ? fused_apply(p, HH_MODE_W, P, ldp, X, n, batch, st) : HH_OK;
    if (hs == HH_OK) {
        if (p->dtype == HH_F32)
            hs = bwd::dispatch<float>(p, HH_MODE_SYM, X, n, gY, ldg, gX, ldgx, gU, gd, batch,
                                      nullptr, 0, pa, st);
        else
            hs = bwd::dispatch<double>(p, HH_MODE_SYM, X, n, gY, ldg, gX, ldgx, gU, gd, batch,
                                       nullptr, 0, pa, st);
    }
    if (X) {
        cudaError_t e = cudaFreeAsync(X, st);
        if (hs == HH_OK && e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync (backward input)");
    }
    return hs;
}

hh_status mahalanobis_backward(const Plan *p, const void *X, int64_t ldx, int64_t nrows,
                               const int64_t *ia, const int64_t *ib, int64_t npairs,
                               const void *gout, void *gU, void *gd, cudaStream_t st) {
    bwd::PairArgs pa;
    pa.ia = ia;
    pa.ib = ib;
    pa.nrows = nrows;
    const int m = bwd::kModeMahalanobis;
    if (p->dtype == HH_F32)
        return bwd::dispatch<float>(p, m, X, ldx, gout, 1, nullptr, p->n, gU, gd, npairs, nullptr,
                                    0, pa, st);
    if (p->dtype == HH_F64)
        return bwd::dispatch<double>(p, m, X, ldx, gout, 1, nullptr, p->n, gU, gd, npairs, nullptr,
                                     0, pa, st);
    return fail(HH_ERR_UNSUPPORTED, "mahalanobis backward: F32 and F64 plans only");
}

}  // namespace hh
