// Staged, blocked F32 reflector-chain kernel.
//
// The chain of §II-A (Eq. (1)-(2)) applied to tiles of vectors held in
// registers, B consecutive reflectors per synchronisation round.  For the
// reflectors j = 1..B of a block, in the order they act, the sequential updates
//     c_j = tau_j (v_j . x_{j-1}),  x_j = x_{j-1} - c_j v_j
// are regrouped so that all dot products use the block's input x:
//     z_j = v_j . x,   c_j = tau_j (z_j - sum_{i<j} c_i (v_i . v_j)),
//     x_B = x - sum_j c_j v_j,
// which is the same arithmetic reordered (the Gram entries v_i . v_j are
// computed in FP64 when the plan is created).  The B*RT dot products of a
// block are reduced together: one transposing warp shuffle, one barrier and
// one cross-warp combine per block instead of per reflector.
//
// Each vector is read from HBM once and written once: tiles are prefetched
// into shared memory by the bulk-copy engine (cp.async.bulk + mbarrier) while
// the previous tile is computed; reflector values are read through L1.
//
// Layout.  Persistent CTAs, as many per SM as fit.  A CTA is RG row groups of
// G threads, each group with its own barrier; thread t of a group owns
// granules t + G*i (i < NG) of 4 floats of each of its RT rows, so one loaded
// reflector value feeds 2*RT FMAs.  Pairs of columns use the packed FP32 FMA.
// Wide tiles (32 columns x 4 rows per thread) double the arithmetic per
// shuffle reduction and per barrier; they need up to 255 registers, so they
// run with half the resident warps.
//
// Waits on the mbarrier are bounded (about a second of clock cycles).  On
// expiry the kernel records HH_ERR_TIMEOUT in *err, waits once more (bounded)
// for that copy, marks the CTA aborted so no further wait blocks, and runs to
// the end without trusting its data.
#pragma once

#include <type_traits>

#include "hh_fused.cuh"

namespace hh {
namespace staged {

constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz
constexpr int kGramBand = 16;                    // Gram entries stored per reflector

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global memory into this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int G, int NG, int RT, int RG, int B>
struct SCfg {
    static constexpr int E = NG * 4;      // floats of one row held by a thread
    static constexpr int E2 = E / 2;      // float2 pairs
    static constexpr int NW = G / 32;     // warps per row group
    static constexpr int THREADS = G * RG;
    static constexpr int ROWS = RT * RG;  // rows per tile
    static constexpr int COVER = G * E;   // columns covered
    static constexpr int NV = B * RT;     // dot products reduced together
    static constexpr int L = 32 / NV;     // lanes holding one value after the warp reduction
    // Wide tiles (32 columns x 4 or more rows per thread) run with up to 255
    // registers per thread: fewer warps, each with twice the work per shuffle
    // reduction and per barrier.  Other tiles are capped at 128 registers so
    // that 16 warps stay resident.
    static constexpr bool WIDE = E >= 32 && RT >= 4;
    static constexpr int MINB = WIDE ? (256 / THREADS > 0 ? 256 / THREADS : 1)
                                     : (512 / THREADS > 0 ? 512 / THREADS : 1);
    // keep the block's reflector values in registers between dot and update
    static constexpr bool KEEP = B * E <= (WIDE ? 64 : 32);
    static_assert(G % 32 == 0, "G must be a multiple of 32");
    static_assert(NV <= 32 && (NV & (NV - 1)) == 0, "B*RT must be a power of two <= 32");
    static_assert(B >= 1 && B <= kGramBand, "block larger than the stored Gram band");
};

template <int G, int NG, int RT, int RG, int B>
__device__ __forceinline__ void scale2(float2 (&x)[RT][SCfg<G, NG, RT, RG, B>::E2],
                                       const float *__restrict__ s, int t) {
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        float4 q = __ldg(reinterpret_cast<const float4 *>(s) + (t + G * i));
        const float2 lo = make_float2(q.x, q.y), hi = make_float2(q.z, q.w);
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            x[r][2 * i] = __fmul2_rn(x[r][2 * i], lo);
            x[r][2 * i + 1] = __fmul2_rn(x[r][2 * i + 1], hi);
        }
    }
}

// Scale the columns of the held rows by s; only the first `act` granule
// indices (a warp-uniform count) are touched.
template <int G, int NG, int RT, int RG, int B>
__device__ __forceinline__ void scale2_part(float2 (&x)[RT][SCfg<G, NG, RT, RG, B>::E2],
                                            const float *__restrict__ s, int t, int act) {
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        if (i >= act) break;
        float4 q = __ldg(reinterpret_cast<const float4 *>(s) + (t + G * i));
        const float2 lo = make_float2(q.x, q.y), hi = make_float2(q.z, q.w);
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            x[r][2 * i] = __fmul2_rn(x[r][2 * i], lo);
            x[r][2 * i + 1] = __fmul2_rn(x[r][2 * i + 1], hi);
        }
    }
}

// Dot products and update of one reflector over the granules i >= I0 (I0 a
// compile-time count), in the same order as over all of them: one packed
// accumulator per row, elements ascending.
template <int I0, int RT, int E2>
__device__ __forceinline__ void dot_from(const float2 (&x)[RT][E2], const float2 (&uj)[E2],
                                         float *p) {
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int e = 2 * I0; e < E2; ++e) a = __ffma2_rn(x[r][e], uj[e], a);
        p[r] = a.x + a.y;
    }
}
template <int I0, int RT, int E2>
__device__ __forceinline__ void update_from(float2 (&x)[RT][E2], const float2 (&uj)[E2],
                                            const float *c) {
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        const float2 cc = make_float2(c[r], c[r]);
#pragma unroll
        for (int e = 2 * I0; e < E2; ++e) x[r][e] = __ffma2_rn(uj[e], cc, x[r][e]);
    }
}
// Apply h reflectors to the RT rows in x, ascending (k = 0..h-1) or descending
// (k = h-1..0), in blocks of B.  With TR, start[k] is the first column where
// v_k may be non-zero (the reflectors of a partial QR factorization, §II-D,
// have k leading zeros): a block skips the granule indices i whose 4G columns
// all lie before the smallest start of its reflectors, in the dot products
// and in the update (a warp-uniform branch).  The skipped terms are exact
// zeros, so the result is the same as without skipping.  With PART, granule
// indices i >= act (warp-uniform: the warp's columns there lie past n) are
// neither read nor computed, so a tile shape wider than n costs n columns of
// arithmetic and reads nothing past the reflectors' rows (the batched launch).
template <int G, int NG, int RT, int RG, int B, bool TR = false, bool PART = false>
__device__ __forceinline__ void chain(
    float2 (&x)[RT][SCfg<G, NG, RT, RG, B>::E2], bool asc, int h, const float *__restrict__ V,
    int64_t ldv, const float *__restrict__ tau, const float *__restrict__ gram, int t, int lane,
    int warp, int rg, float *red, int &buf, const int *__restrict__ start = nullptr,
    int act = NG) {
    constexpr bool RANGED = TR || PART;
    using C = SCfg<G, NG, RT, RG, B>;
    constexpr int E2 = C::E2, NW = C::NW, NV = C::NV, L = C::L;
    // Values of reflector j of the block starting at s (zeros past h).
    auto load_block_u = [&](int s0, int j, float2(&dst)[E2]) {
        const bool ok = s0 + j < h;
        const int k = asc ? s0 + j : h - 1 - s0 - j;
        const float4 *row = reinterpret_cast<const float4 *>(V + (size_t)(ok ? k : 0) * ldv);
#pragma unroll
        for (int i = 0; i < NG; ++i) {
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ok && (!PART || i < act)) q = __ldg(row + (t + G * i));
            dst[2 * i] = make_float2(q.x, q.y);
            dst[2 * i + 1] = make_float2(q.z, q.w);
        }
    };
    // Reflector values: all B kept in registers between the dot and the
    // update phase (KEEP), or one at a time and read again for the update.
    // Kept values are software-pipelined: reflector j of the next block is
    // loaded as soon as the update with reflector j of this block is issued,
    // so its latency hides behind the rest of the update instead of stalling
    // the next block's dot products.
    constexpr int KB = C::KEEP ? B : 1;
    float2 u[KB][E2];
    if constexpr (C::KEEP) {
#pragma unroll
        for (int j = 0; j < B; ++j) load_block_u(0, j, u[j]);
    }
    // tau and the Gram entries of the block starting at s0 (zeros past h),
    // read before the block's reduction so that their latency is not exposed
    // between the barrier and the update.
    auto load_coef = [&](int s0, float(&tk)[B], float(&gv)[B][B]) {
        const int nb0 = h - s0 < B ? h - s0 : B;
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int kj = asc ? s0 + j : h - 1 - s0 - j;
            tk[j] = j < nb0 ? __ldg(tau + kj) : 0.f;
#pragma unroll
            for (int i = 0; i < B; ++i) {
                const int ki = asc ? s0 + i : h - 1 - s0 - i;
                gv[j][i] = (i > j && i < nb0)
                               ? __ldg(gram + (size_t)(asc ? kj : ki) * kGramBand + (i - j))
                               : 0.f;
            }
        }
    };
    // One round of B reflectors starting at s; granule indices below the
    // compile-time I0 are left out (zero-prefix skipping; 0 otherwise).
    auto round = [&](auto i0c, int s) {
        constexpr int I0 = decltype(i0c)::value;
        (void)I0;
            const int nb = h - s < B ? h - s : B;
            float tk[B], gv[B][B];
            load_coef(s, tk, gv);
            auto load_u = [&](int j, float2(&dst)[E2]) { load_block_u(s, j, dst); };
            float p[NV];
    #pragma unroll
            for (int j = 0; j < B; ++j) {
                if constexpr (!C::KEEP) load_u(j, u[0]);
                const float2(&uj)[E2] = u[C::KEEP ? j : 0];
                if constexpr (TR && !PART) {
                    dot_from<I0, RT, E2>(x, uj, p + j * RT);
                } else if constexpr (RANGED) {
                    // the same summation order per row, skipped granules left out
                    float2 a[RT];
    #pragma unroll
                    for (int r = 0; r < RT; ++r) a[r] = make_float2(0.f, 0.f);
    #pragma unroll
                    for (int i = 0; i < NG; ++i) {
                        if (PART && i >= act) continue;
    #pragma unroll
                        for (int r = 0; r < RT; ++r) {
                            a[r] = __ffma2_rn(x[r][2 * i], uj[2 * i], a[r]);
                            a[r] = __ffma2_rn(x[r][2 * i + 1], uj[2 * i + 1], a[r]);
                        }
                    }
    #pragma unroll
                    for (int r = 0; r < RT; ++r) p[j * RT + r] = a[r].x + a[r].y;
                } else {
                    // one packed accumulator per row
    #pragma unroll
                    for (int r = 0; r < RT; ++r) {
                        float2 a = make_float2(0.f, 0.f);
    #pragma unroll
                        for (int e = 0; e < E2; ++e) a = __ffma2_rn(x[r][e], uj[e], a);
                        p[j * RT + r] = a.x + a.y;
                    }
                }
            }
            float v = fused::warp_reduce_rows<float, NV>(p, lane);  // lane holds value lane / L
            float z[NV];
            if constexpr (NW == 1) {
    #pragma unroll
                for (int q = 0; q < NV; ++q) z[q] = __shfl_sync(0xffffffffu, v, q * L);
            } else {
                if ((lane & (L - 1)) == 0) red[fused::red_index<RG, NV, NW>(buf, rg, lane / L, warp)] = v;
                // only this row group's warps meet here (named barrier 1 + rg with
                // several groups), so row groups do not wait for one another
                if constexpr (RG > 1)
                    asm volatile("bar.sync %0, %1;" ::"r"(1 + rg), "n"(G) : "memory");
                else
                    __syncthreads();
                const int idx = lane / L, sub = lane & (L - 1);
                float q = 0.f;
    #pragma unroll
                for (int w = sub; w < NW; w += L) q += red[fused::red_index<RG, NV, NW>(buf, rg, idx, w)];
    #pragma unroll
                for (int off = L / 2; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
    #pragma unroll
                for (int qq = 0; qq < NV; ++qq) z[qq] = __shfl_sync(0xffffffffu, q, qq * L);
                buf ^= 1;
            }
            // Coefficients in the order the reflectors act, stored negated:
            // c_j = -tau_j (z_j - sum_{i<j} c_i g_ij), resolved left to right.  The
            // Gram entries are uniform scalars read through L1 (the smaller index
            // of each pair addresses the band).
            float c[B][RT];
    #pragma unroll
            for (int j = 0; j < B; ++j)
    #pragma unroll
                for (int r = 0; r < RT; ++r) c[j][r] = z[j * RT + r];
    #pragma unroll
            for (int j = 0; j < B; ++j) {
    #pragma unroll
                for (int r = 0; r < RT; ++r) c[j][r] *= -tk[j];
    #pragma unroll
                for (int i = j + 1; i < B; ++i) {
    #pragma unroll
                    for (int r = 0; r < RT; ++r) c[i][r] = fmaf(c[j][r], gv[j][i], c[i][r]);
                }
            }
    #pragma unroll
            for (int j = 0; j < B; ++j) {
                if constexpr (!C::KEEP) load_u(j, u[0]);
                const float2(&uj)[E2] = u[C::KEEP ? j : 0];
                if constexpr (TR && !PART) {
                    float cj[RT];
    #pragma unroll
                    for (int r = 0; r < RT; ++r) cj[r] = c[j][r];
                    update_from<I0, RT, E2>(x, uj, cj);
                } else if constexpr (RANGED) {
    #pragma unroll
                    for (int i = 0; i < NG; ++i) {
                        if (PART && i >= act) continue;
    #pragma unroll
                        for (int r = 0; r < RT; ++r) {
                            const float2 cc = make_float2(c[j][r], c[j][r]);
                            x[r][2 * i] = __ffma2_rn(uj[2 * i], cc, x[r][2 * i]);
                            x[r][2 * i + 1] = __ffma2_rn(uj[2 * i + 1], cc, x[r][2 * i + 1]);
                        }
                    }
                } else {
    #pragma unroll
                    for (int r = 0; r < RT; ++r) {
                        const float2 cc = make_float2(c[j][r], c[j][r]);
    #pragma unroll
                        for (int e = 0; e < E2; ++e) x[r][e] = __ffma2_rn(uj[e], cc, x[r][e]);
                    }
                }
                if constexpr (C::KEEP) load_block_u(s + B, j, u[j]);
            }
    };
    if constexpr (TR && !PART) {
        static_assert(NG <= 8, "zero-prefix skipping covers at most 8 granule indices");
        // Rounds are taken in runs with the same skipped prefix, each run by an
        // instantiation for its prefix, so the loops stay fully unrolled.
        auto i0_of = [&](int s0) {
            int mn = 0x7fffffff;
#pragma unroll
            for (int j = 0; j < B; ++j)
                if (s0 + j < h) {
                    const int st0 = __ldg(start + (asc ? s0 + j : h - 1 - s0 - j));
                    mn = st0 < mn ? st0 : mn;
                }
            const int q = mn / (4 * G);
            return q < NG ? q : NG;
        };
        int s = 0;
        while (s < h) {
            const int i0 = i0_of(s);
            int e = s + B;
            while (e < h && i0_of(e) == i0) e += B;
            switch (i0) {
#define HH_RUN_CASE(I)                                                                   \
    case I:                                                                              \
        if constexpr (I <= NG)                                                           \
            for (; s < e; s += B) round(std::integral_constant<int, (I <= NG ? I : 0)>{}, s); \
        break;
                HH_RUN_CASE(0) HH_RUN_CASE(1) HH_RUN_CASE(2) HH_RUN_CASE(3) HH_RUN_CASE(4)
                HH_RUN_CASE(5) HH_RUN_CASE(6) HH_RUN_CASE(7) HH_RUN_CASE(8)
#undef HH_RUN_CASE
                default: s = e; break;
            }
        }
    } else {
        for (int s = 0; s < h; s += B) round(std::integral_constant<int, 0>{}, s);
    }
}

// Requirements (checked by the launcher): n % 4 == 0, n <= COVER, X and Y rows
// and bases 16-byte aligned, V rows padded with zeros to ldv >= COVER, ldv % 4
// == 0, ROWS*n floats of dynamic shared memory.
// Registers: at most 128 per thread (16 resident warps per SM), or 255 for wide
// tiles (8 warps per SM).
template <int MODE, int G, int NG, int RT, int RG, int B, bool TR = false>
__global__ void __launch_bounds__(G *RG, (SCfg<G, NG, RT, RG, B>::MINB))
staged_chain_kernel(const float *X, int64_t ldx, float *Y, int64_t ldy, int64_t batch, int n,
                    const float *__restrict__ V, const float *__restrict__ tau, int64_t ldv,
                    int h, const float *__restrict__ gram, const float *__restrict__ sign,
                    const float *__restrict__ d, int *__restrict__ err,
                    const int *__restrict__ start) {
    using C = SCfg<G, NG, RT, RG, B>;
    constexpr int E2 = C::E2, ROWS = C::ROWS;
    extern __shared__ __align__(128) float stage[];  // ROWS x n
    __shared__ __align__(8) uint64_t full_bar;
    __shared__ __align__(16) float red[2 * RG * C::NV * C::NW];
    __shared__ int aborted;

    const int tid = threadIdx.x;
    const int rg = tid / G;
    const int t = tid - rg * G;
    const int warp = t >> 5, lane = t & 31;
    const int64_t tiles = (batch + ROWS - 1) / ROWS;
    int64_t tile = blockIdx.x;
    if (tile >= tiles) return;
    const uint32_t row_bytes = (uint32_t)n * 4u;

    auto issue_tile = [&](int64_t tl) {
        const int64_t r0 = tl * ROWS;
        const int64_t left = batch - r0;
        const int nvalid = left < ROWS ? (int)left : ROWS;
        mbar_expect_tx(&full_bar, row_bytes * (uint32_t)nvalid);
        for (int r = 0; r < nvalid; ++r)
            bulk_g2s(stage + (size_t)r * n, X + (r0 + r) * ldx, row_bytes, &full_bar);
    };

    if (tid == 0) {
        aborted = 0;
        mbar_init(&full_bar, 1);
        fence_proxy_async();
        issue_tile(tile);
    }
    __syncthreads();

    uint32_t phase = 0;
    int buf = 0;
    for (; tile < tiles; tile += gridDim.x) {
        if (!*(volatile int *)&aborted && !mbar_wait_bounded(&full_bar, phase)) {
            atomicExch(err, (int)HH_ERR_TIMEOUT);
            mbar_wait_bounded(&full_bar, phase);  // give the copy in flight one more chance
            *(volatile int *)&aborted = 1;
        }
        phase ^= 1;
        const int64_t r0 = tile * ROWS;
        float2 x[RT][E2];
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const int lr = rg * RT + r;
            const bool valid = r0 + lr < batch;
            const float *srow = stage + (size_t)lr * n;
#pragma unroll
            for (int i = 0; i < NG; ++i) {
                const int col = (t + G * i) * 4;
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                if (valid && col < n) q = *reinterpret_cast<const float4 *>(srow + col);
                x[r][2 * i] = make_float2(q.x, q.y);
                x[r][2 * i + 1] = make_float2(q.z, q.w);
            }
        }
        __syncthreads();  // every thread has its rows: the stage may be refilled
        if (tid == 0 && tile + gridDim.x < tiles && !aborted) {
            fence_proxy_async();
            issue_tile(tile + gridDim.x);
        }

        if (MODE != HH_MODE_W && sign) scale2<G, NG, RT, RG, B>(x, sign, t);
        // W: k = h..1; W^T: k = 1..h; S: k = 1..h, scale by d, k = h..1 (one
        // loop, so the chain is instantiated once per kernel).
        for (int half = 0; half < (MODE == HH_MODE_SYM ? 2 : 1); ++half) {
            if (half == 1) scale2<G, NG, RT, RG, B>(x, d, t);
            const bool asc = MODE != HH_MODE_W && half == 0;
            chain<G, NG, RT, RG, B, TR>(x, asc, h, V, ldv, tau, gram, t, lane, warp, rg, red, buf,
                                        start);
        }
        if (MODE != HH_MODE_WT && sign) scale2<G, NG, RT, RG, B>(x, sign, t);

#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const int64_t row = r0 + rg * RT + r;
            if (row >= batch) continue;
            float *yr = Y + row * ldy;
#pragma unroll
            for (int i = 0; i < NG; ++i) {
                const int col = (t + G * i) * 4;
                if (col < n)
                    __stcs(reinterpret_cast<float4 *>(yr + col),
                           make_float4(x[r][2 * i].x, x[r][2 * i].y, x[r][2 * i + 1].x,
                                       x[r][2 * i + 1].y));
            }
        }
    }
}

// start: per-reflector first possibly non-zero column, or null; with it the
// kernels skip zero prefixes (TR).
template <int G, int NG, int RT, int RG, int B>
cudaError_t launch(hh_mode mode, const float *X, int64_t ldx, float *Y, int64_t ldy,
                   int64_t batch, int n, const float *V, const float *tau, int64_t ldv, int h,
                   const float *gram, const float *sign, const float *d, int *err, int num_sms,
                   cudaStream_t st, const int *start = nullptr) {
    using C = SCfg<G, NG, RT, RG, B>;
    const size_t smem = (size_t)C::ROWS * n * sizeof(float);
    const int64_t tiles = (batch + C::ROWS - 1) / C::ROWS;
    // Per kernel (one entry per mode) and device: the shared-memory opt-in at
    // the largest stage this configuration can need, and the resident CTAs per
    // SM there (a lower bound for smaller stages), both set on first use.
    static PerDevice state[6];
    auto run = [&](auto kern, int slot) -> cudaError_t {
        int per_sm = 1;
        cudaError_t e = per_device(state[slot], per_sm, [&](int &v) -> cudaError_t {
            const size_t smax = (size_t)C::ROWS * C::COVER * sizeof(float);
            cudaError_t e2 =
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
            if (e2 != cudaSuccess) return e2;
            int nb = 0;
            e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, C::THREADS, smax);
            if (e2 != cudaSuccess) return e2;
            v = nb > 0 ? nb : 1;
            return cudaSuccess;
        });
        if (e != cudaSuccess) return e;
        const int64_t slots = (int64_t)num_sms * per_sm;
        const int grid = (int)(tiles < slots ? tiles : slots);
        kern<<<grid, C::THREADS, smem, st>>>(X, ldx, Y, ldy, batch, n, V, tau, ldv, h, gram, sign,
                                             d, err, start);
        return cudaGetLastError();
    };
    if (start) {
        switch (mode) {
            case HH_MODE_W: return run(staged_chain_kernel<HH_MODE_W, G, NG, RT, RG, B, true>, 3);
            case HH_MODE_WT: return run(staged_chain_kernel<HH_MODE_WT, G, NG, RT, RG, B, true>, 4);
            default: return run(staged_chain_kernel<HH_MODE_SYM, G, NG, RT, RG, B, true>, 5);
        }
    }
    switch (mode) {
        case HH_MODE_W: return run(staged_chain_kernel<HH_MODE_W, G, NG, RT, RG, B>, 0);
        case HH_MODE_WT: return run(staged_chain_kernel<HH_MODE_WT, G, NG, RT, RG, B>, 1);
        default: return run(staged_chain_kernel<HH_MODE_SYM, G, NG, RT, RG, B>, 2);
    }
}

}  // namespace staged
}  // namespace hh
