// Fused reflector-chain kernels (CUDA cores, F32 / F64).
//
// One pass over X: every vector is read once and written once; all h
// reflectors are applied while the vector sits in registers.  Per reflector
// (§II-A, Eq. (2): H_k = I - tau_k v_k v_k^T, tau_k = 2 / v_k^T v_k):
//     c = tau_k (v_k . x)   (warp-shuffle dot product, then across warps)
//     x <- x - c v_k
// which is the paper's 4n operations per reflector (§II-A).  The modes run
// the chain in the orders of Eq. (1) and Eq. (21):
//     W   : k = h..1, then y = sigma .* x
//     WT  : x = sigma .* x, then k = 1..h
//     SYM : sigma, k = 1..h, x = d .* x, k = h..1, sigma
//
// Thread layout.  A CTA holds RG row groups; a row group is G threads (G/32
// warps) that share RT rows.  Thread t of a group owns NG 16-byte granules of
// every one of its rows: granule t + G*i, i < NG, so a warp's loads and stores
// are 512-byte contiguous runs.  Per reflector a thread loads its NG granules
// of v_k once and reuses them for RT rows (dot and update).  The RT partial
// dot products of a warp are reduced with a transposing shuffle tree (each
// lane ends with one row's warp sum), then across the group's warps through
// shared memory with one barrier per reflector (double-buffered).
#pragma once

#include "hh_internal.cuh"

namespace hh {
namespace fused {

template <typename T>
struct Granule;
template <>
struct Granule<float> {
    using type = float4;
    static constexpr int N = 4;
};
template <>
struct Granule<double> {
    using type = double2;
    static constexpr int N = 2;
};

template <typename T>
__device__ __forceinline__ void load_granule(const T *p, T (&v)[Granule<T>::N]);
template <>
__device__ __forceinline__ void load_granule<float>(const float *p, float (&v)[4]) {
    float4 q = __ldcs(reinterpret_cast<const float4 *>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <>
__device__ __forceinline__ void load_granule<double>(const double *p, double (&v)[2]) {
    double2 q = __ldcs(reinterpret_cast<const double2 *>(p));
    v[0] = q.x; v[1] = q.y;
}
template <typename T>
__device__ __forceinline__ void ldg_granule(const T *p, T (&v)[Granule<T>::N]);
template <>
__device__ __forceinline__ void ldg_granule<float>(const float *p, float (&v)[4]) {
    float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <>
__device__ __forceinline__ void ldg_granule<double>(const double *p, double (&v)[2]) {
    double2 q = __ldg(reinterpret_cast<const double2 *>(p));
    v[0] = q.x; v[1] = q.y;
}
template <typename T>
__device__ __forceinline__ void store_granule(T *p, const T (&v)[Granule<T>::N]);
template <>
__device__ __forceinline__ void store_granule<float>(float *p, const float (&v)[4]) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
}
template <>
__device__ __forceinline__ void store_granule<double>(double *p, const double (&v)[2]) {
    __stcs(reinterpret_cast<double2 *>(p), make_double2(v[0], v[1]));
}

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

// Transposing warp reduction of RT values per lane.  On return every lane holds
// the warp-wide sum of p[r] with r = lane >> (5 - log2(RT)).
template <typename T, int RT>
__device__ __forceinline__ T warp_reduce_rows(T (&p)[RT], int lane) {
    constexpr int L = ilog2(RT);
    static_assert((1 << L) == RT && RT <= 32, "RT must be a power of two <= 32");
#pragma unroll
    for (int s = 0; s < L; ++s) {
        const int off = 16 >> s;
        const int half = RT >> (s + 1);
        const bool hi = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            T send = hi ? p[i] : p[i + half];
            T keep = hi ? p[i + half] : p[i];
            p[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    T v = p[0];
#pragma unroll
    for (int off = 16 >> L; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Flat index of a cross-warp partial in a reduction buffer laid out as
// [2 buffers][RG groups][NV values][NW warps].  The buffers are plain 1-D shared
// arrays indexed by this function: a 4-D __shared__ array indexed the same way
// gave wrong partial sums in one kernel of this library.
template <int RG, int NV, int NW>
__device__ __forceinline__ int red_index(int buf, int rg, int v, int w) {
    return ((buf * RG + rg) * NV + v) * NW + w;
}

template <typename T, int G, int NG, int RT, int RG>
struct Cfg {
    static constexpr int VEC = Granule<T>::N;
    static constexpr int E = NG * VEC;   // elements of one row held by a thread
    static constexpr int NW = G / 32;    // warps per row group
    static constexpr int THREADS = G * RG;
    static constexpr int ROWS = RT * RG; // rows per CTA
    static constexpr int COVER = G * E;  // columns covered
    static_assert(G % 32 == 0, "G must be a multiple of 32");
    static_assert(RT * NW <= 32, "cross-warp reduction uses one lane per (row, warp)");
};

// Apply reflector H_k = I - tk vk vk^T to the RT rows held in x.
template <typename T, int G, int NG, int RT, int RG>
__device__ __forceinline__ void reflect(T (&x)[RT][Cfg<T, G, NG, RT, RG>::E],
                                        const T *__restrict__ uk, T tk, int t, int lane, int warp,
                                        int rg, T *red, int &buf) {
    using C = Cfg<T, G, NG, RT, RG>;
    constexpr int VEC = C::VEC, E = C::E, NW = C::NW;
    T u[E];
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        T g[VEC];
        ldg_granule<T>(uk + (size_t)(t + G * i) * VEC, g);
#pragma unroll
        for (int e = 0; e < VEC; ++e) u[i * VEC + e] = g[e];
    }
    T p[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        T s0 = 0, s1 = 0;
#pragma unroll
        for (int e = 0; e < E; e += 2) {
            s0 = fma(x[r][e], u[e], s0);
            if (e + 1 < E) s1 = fma(x[r][e + 1], u[e + 1], s1);
        }
        p[r] = s0 + s1;
    }
    T v = warp_reduce_rows<T, RT>(p, lane);
    constexpr int SH = 5 - ilog2(RT);  // lanes per row after the reduction = 1 << SH
    T c[RT];
    if constexpr (NW == 1) {
#pragma unroll
        for (int r = 0; r < RT; ++r) c[r] = tk * __shfl_sync(0xffffffffu, v, r << SH);
    } else {
        if ((lane & ((1 << SH) - 1)) == 0) red[red_index<RG, RT, NW>(buf, rg, lane >> SH, warp)] = v;
        __syncthreads();
        // lane l < RT*NW reads partial (row l / NW, warp l % NW); segments of NW lanes sum.
        T q = lane < RT * NW ? red[red_index<RG, RT, NW>(buf, rg, lane / NW, lane % NW)] : T(0);
#pragma unroll
        for (int off = NW / 2; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
#pragma unroll
        for (int r = 0; r < RT; ++r) c[r] = tk * __shfl_sync(0xffffffffu, q, r * NW);
        buf ^= 1;
    }
#pragma unroll
    for (int r = 0; r < RT; ++r) {
#pragma unroll
        for (int e = 0; e < E; ++e) x[r][e] = fma(-c[r], u[e], x[r][e]);
    }
}

template <typename T, int G, int NG, int RT, int RG>
__device__ __forceinline__ void scale_cols(T (&x)[RT][Cfg<T, G, NG, RT, RG>::E],
                                           const T *__restrict__ s, int t) {
    using C = Cfg<T, G, NG, RT, RG>;
    constexpr int VEC = C::VEC;
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        T g[VEC];
        ldg_granule<T>(s + (size_t)(t + G * i) * VEC, g);
#pragma unroll
        for (int r = 0; r < RT; ++r)
#pragma unroll
            for (int e = 0; e < VEC; ++e) x[r][i * VEC + e] *= g[e];
    }
}

// X and Y may be the same buffer (each thread reads its elements before it
// writes them, and no two threads share an element).
template <typename T, int MODE, int G, int NG, int RT, int RG>
__global__ void __launch_bounds__(G *RG)
fused_chain_kernel(const T *X, int64_t ldx, T *Y, int64_t ldy, int64_t batch, int n,
                   const T *__restrict__ U, const T *__restrict__ tau, int64_t ldv, int h,
                   const T *__restrict__ sign, const T *__restrict__ d, int vec_ok) {
    using C = Cfg<T, G, NG, RT, RG>;
    constexpr int VEC = C::VEC, E = C::E, NW = C::NW;
    __shared__ T red[2 * RG * RT * NW];
    const int tid = threadIdx.x;
    const int rg = tid / G;
    const int t = tid - rg * G;
    const int warp = t >> 5, lane = t & 31;
    const int64_t row0 = ((int64_t)blockIdx.x * RG + rg) * RT;
    int buf = 0;

    T x[RT][E];
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        const int64_t row = row0 + r;
        const T *xr = X + row * ldx;
#pragma unroll
        for (int i = 0; i < NG; ++i) {
            const int col = (t + G * i) * VEC;
            T g[VEC];
            if (row < batch && vec_ok && col + VEC <= n) {
                load_granule<T>(xr + col, g);
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e) g[e] = (row < batch && col + e < n) ? xr[col + e] : T(0);
            }
#pragma unroll
            for (int e = 0; e < VEC; ++e) x[r][i * VEC + e] = g[e];
        }
    }

    if (MODE != HH_MODE_W && sign) scale_cols<T, G, NG, RT, RG>(x, sign, t);
    if (MODE != HH_MODE_W) {
        for (int k = 0; k < h; ++k)
            reflect<T, G, NG, RT, RG>(x, U + (size_t)k * ldv, __ldg(tau + k), t, lane, warp, rg,
                                      red, buf);
    }
    if (MODE == HH_MODE_SYM) scale_cols<T, G, NG, RT, RG>(x, d, t);
    if (MODE != HH_MODE_WT) {
        for (int k = h - 1; k >= 0; --k)
            reflect<T, G, NG, RT, RG>(x, U + (size_t)k * ldv, __ldg(tau + k), t, lane, warp, rg,
                                      red, buf);
    }
    if (MODE != HH_MODE_WT && sign) scale_cols<T, G, NG, RT, RG>(x, sign, t);

#pragma unroll
    for (int r = 0; r < RT; ++r) {
        const int64_t row = row0 + r;
        if (row >= batch) continue;
        T *yr = Y + row * ldy;
#pragma unroll
        for (int i = 0; i < NG; ++i) {
            const int col = (t + G * i) * VEC;
            T g[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) g[e] = x[r][i * VEC + e];
            if (vec_ok && col + VEC <= n) {
                store_granule<T>(yr + col, g);
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (col + e < n) yr[col + e] = g[e];
            }
        }
    }
}

// Rows too long for registers: one CTA per row, the row kept in Y (global),
// re-read and re-written once per reflector.  Correct for any n; only meant
// for n beyond the register-tiled configurations.
template <typename T, int MODE>
__global__ void __launch_bounds__(512)
wide_chain_kernel(const T *X, int64_t ldx, T *Y, int64_t ldy, int64_t batch, int64_t n,
                  const T *__restrict__ U, const T *__restrict__ tau, int64_t ldv, int h,
                  const T *__restrict__ sign, const T *__restrict__ d) {
    __shared__ T red[32];
    __shared__ T bc;
    const int64_t row = blockIdx.x;
    if (row >= batch) return;
    const T *xr = X + row * ldx;
    T *yr = Y + row * ldy;
    auto block_sum = [&](T v) -> T {
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x < 32) {
            T q = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : T(0);
            for (int off = 16; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
            if (threadIdx.x == 0) bc = q;
        }
        __syncthreads();
        T r = bc;
        __syncthreads();
        return r;
    };
    auto reflect1 = [&](int k) {
        const T *uk = U + (size_t)k * ldv;
        T s = 0;
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s = fma(yr[j], uk[j], s);
        T c = tau[k] * block_sum(s);
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) yr[j] = fma(-c, uk[j], yr[j]);
        __syncthreads();
    };
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        T v = xr[j];
        if (MODE != HH_MODE_W && sign) v *= sign[j];
        yr[j] = v;
    }
    __syncthreads();
    if (MODE != HH_MODE_W)
        for (int k = 0; k < h; ++k) reflect1(k);
    if (MODE == HH_MODE_SYM) {
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) yr[j] *= d[j];
        __syncthreads();
    }
    if (MODE != HH_MODE_WT)
        for (int k = h - 1; k >= 0; --k) reflect1(k);
    if (MODE != HH_MODE_WT && sign)
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) yr[j] *= sign[j];
}

template <typename T, int G, int NG, int RT, int RG>
cudaError_t launch_cfg(hh_mode mode, const T *X, int64_t ldx, T *Y, int64_t ldy, int64_t batch,
                       int n, const T *U, const T *tau, int64_t ldv, int h, const T *sign,
                       const T *d, int vec_ok, cudaStream_t st) {
    using C = Cfg<T, G, NG, RT, RG>;
    const int64_t blocks = (batch + C::ROWS - 1) / C::ROWS;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)blocks);
    switch (mode) {
        case HH_MODE_W:
            fused_chain_kernel<T, HH_MODE_W, G, NG, RT, RG>
                <<<grid, C::THREADS, 0, st>>>(X, ldx, Y, ldy, batch, n, U, tau, ldv, h, sign, d, vec_ok);
            break;
        case HH_MODE_WT:
            fused_chain_kernel<T, HH_MODE_WT, G, NG, RT, RG>
                <<<grid, C::THREADS, 0, st>>>(X, ldx, Y, ldy, batch, n, U, tau, ldv, h, sign, d, vec_ok);
            break;
        default:
            fused_chain_kernel<T, HH_MODE_SYM, G, NG, RT, RG>
                <<<grid, C::THREADS, 0, st>>>(X, ldx, Y, ldy, batch, n, U, tau, ldv, h, sign, d, vec_ok);
            break;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_wide(hh_mode mode, const T *X, int64_t ldx, T *Y, int64_t ldy, int64_t batch,
                        int64_t n, const T *U, const T *tau, int64_t ldv, int h, const T *sign,
                        const T *d, cudaStream_t st) {
    if (batch > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)batch);
    switch (mode) {
        case HH_MODE_W:
            wide_chain_kernel<T, HH_MODE_W><<<grid, 512, 0, st>>>(X, ldx, Y, ldy, batch, n, U, tau, ldv, h, sign, d);
            break;
        case HH_MODE_WT:
            wide_chain_kernel<T, HH_MODE_WT><<<grid, 512, 0, st>>>(X, ldx, Y, ldy, batch, n, U, tau, ldv, h, sign, d);
            break;
        default:
            wide_chain_kernel<T, HH_MODE_SYM><<<grid, 512, 0, st>>>(X, ldx, Y, ldy, batch, n, U, tau, ldv, h, sign, d);
            break;
    }
    return cudaGetLastError();
}

}  // namespace fused
}  // namespace hh
