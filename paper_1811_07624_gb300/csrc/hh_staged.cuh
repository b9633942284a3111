// Staged F32 reflector-chain kernel: the fused chain of hh_fused.cuh with the
// vectors and the reflectors moved through shared memory by the bulk-copy
// engine (cp.async.bulk + mbarrier), so the arithmetic loop reads registers
// and shared memory only.
//
// Per reflector (§II-A, Eq. (2)): c = tau_k (v_k . x), x <- x - c v_k, in the
// mode orders of Eq. (1) / Eq. (21).  Each vector is read from HBM once (into
// shared memory, then registers) and written once (registers -> HBM).
//
// Layout.  Persistent CTAs, as many per SM as fit.  A CTA is RG row groups of
// G threads; thread t of a group owns granules t + G*i (i < NG) of 4 floats of
// each of its RT rows, so one reflector value loaded from shared memory feeds
// 2*RT FMAs.  The RT partial dot products are reduced by a transposing warp
// shuffle, then across the group's G/32 warps through shared memory behind one
// CTA barrier per chain step.  Pairs of columns use the packed FP32 FMA.
//
// Shared memory: `stage` receives the CTA's next tile of rows while the
// current tile is computed in registers.  `ring` holds reflector vectors
// (padded to COVER floats): when all h fit (resident) they are loaded once per
// CTA; otherwise S slots stream the chain steps, and the slot used by step
// g-1 is refilled (with step g-1+S) right after step g's barrier, which every
// thread passes only after it finished step g-1.
//
// Waits on an mbarrier are bounded (about a second of clock cycles).  On
// expiry the kernel records HH_ERR_TIMEOUT in *err, waits once more (bounded)
// for that copy, marks the CTA aborted so no further wait blocks, and runs to
// the end without trusting its data.
#pragma once

#include "hh_fused.cuh"

namespace hh {
namespace staged {

constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz
constexpr int kMaxSlots = 64;

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

template <int G, int NG, int RT, int RG>
struct SCfg {
    static constexpr int E = NG * 4;      // floats of one row held by a thread
    static constexpr int E2 = E / 2;      // float2 pairs
    static constexpr int NW = G / 32;
    static constexpr int THREADS = G * RG;
    static constexpr int ROWS = RT * RG;  // rows per tile
    static constexpr int COVER = G * E;   // padded reflector length in shared memory
    static_assert(G % 32 == 0 && RT * NW <= 32, "bad staged configuration");
    static_assert(RG == 1 || NW == 1, "several row groups only with one warp each");
};

// Floats of the tile stage (ROWS rows of n), rounded up to 128 bytes.
template <int G, int NG, int RT, int RG>
__host__ __device__ constexpr size_t stage_floats(int n) {
    return ((size_t)SCfg<G, NG, RT, RG>::ROWS * n + 31) / 32 * 32;
}

template <int G, int NG, int RT, int RG>
__device__ __forceinline__ void scale2(float2 (&x)[RT][SCfg<G, NG, RT, RG>::E2],
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

// Requirements (checked by the launcher): n % 4 == 0, n <= COVER, X and Y rows
// and bases 16-byte aligned, V rows padded with zeros to ldv >= COVER, ldv % 4
// == 0, 1 <= S <= kMaxSlots, and stage + S*COVER floats of dynamic shared memory.
template <int MODE, int G, int NG, int RT, int RG>
__global__ void __launch_bounds__(G *RG)
staged_chain_kernel(const float *X, int64_t ldx, float *Y, int64_t ldy, int64_t batch, int n,
                    const float *__restrict__ V, const float *__restrict__ tau, int64_t ldv,
                    int h, const float *__restrict__ sign, const float *__restrict__ d, int S,
                    int *__restrict__ err) {
    using C = SCfg<G, NG, RT, RG>;
    constexpr int E2 = C::E2, NW = C::NW, ROWS = C::ROWS, COVER = C::COVER;
    extern __shared__ __align__(128) float smem[];
    float *stage = smem;                                  // ROWS x n
    float *ring = smem + stage_floats<G, NG, RT, RG>(n);  // S x COVER
    __shared__ __align__(8) uint64_t full_bar;
    __shared__ __align__(8) uint64_t vbar[kMaxSlots];
    __shared__ float red[2][RG][RT][NW];
    __shared__ int aborted;

    const int tid = threadIdx.x;
    const int rg = tid / G;
    const int t = tid - rg * G;
    const int warp = t >> 5, lane = t & 31;
    const int64_t tiles = (batch + ROWS - 1) / ROWS;
    int64_t tile = blockIdx.x;
    if (tile >= tiles) return;
    const uint32_t row_bytes = (uint32_t)n * 4u;
    const bool resident = S >= h;
    const int steps = MODE == HH_MODE_SYM ? 2 * h : h;
    const int64_t my_tiles = (tiles - 1 - blockIdx.x) / gridDim.x + 1;
    const int64_t total_steps = my_tiles * steps;
    auto kof = [&](int s) {
        return MODE == HH_MODE_W ? h - 1 - s
                                 : (MODE == HH_MODE_WT ? s : (s < h ? s : 2 * h - 1 - s));
    };
    auto issue_tile = [&](int64_t tl) {
        const int64_t r0 = tl * ROWS;
        const int64_t left = batch - r0;
        const int nvalid = left < ROWS ? (int)left : ROWS;
        mbar_expect_tx(&full_bar, row_bytes * (uint32_t)nvalid);
        for (int r = 0; r < nvalid; ++r)
            bulk_g2s(stage + (size_t)r * n, X + (r0 + r) * ldx, row_bytes, &full_bar);
    };
    auto issue_reflector = [&](int k, int slot) {
        mbar_expect_tx(&vbar[slot], COVER * 4u);
        bulk_g2s(ring + (size_t)slot * COVER, V + (size_t)k * ldv, COVER * 4u, &vbar[slot]);
    };
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (*(volatile int *)&aborted) return;
        if (!mbar_wait_bounded(bar, parity)) {
            atomicExch(err, (int)HH_ERR_TIMEOUT);
            mbar_wait_bounded(bar, parity);  // give the copy in flight one more chance to land
            *(volatile int *)&aborted = 1;
        }
    };

    if (tid == 0) {
        aborted = 0;
        mbar_init(&full_bar, 1);
        const int nslots = resident ? (h > 0 ? h : 1) : S;
        for (int j = 0; j < nslots; ++j) mbar_init(&vbar[j], 1);
        fence_proxy_async();
        issue_tile(tile);
        if (resident) {
            for (int k = 0; k < h; ++k) issue_reflector(k, k);
        } else {
            int si = 0;
            for (int64_t gg = 0; gg < S && gg < total_steps; ++gg) {
                issue_reflector(kof(si), (int)gg);
                si = si + 1 == steps ? 0 : si + 1;
            }
        }
    }
    __syncthreads();

    uint32_t phase = 0;
    int buf = 0;
    int64_t g = 0;  // this CTA's chain-step counter
    // Ring bookkeeping without divisions: the slot and phase parity of the
    // current step, the slot of the previous step, and (thread 0) the next
    // global step to copy in and its position in the chain.
    int slot_c = 0, slot_prev = 0;
    uint32_t par_c = 0;
    int64_t g_issue = S;
    int s_issue = steps > 0 ? S % steps : 0;
    for (; tile < tiles; tile += gridDim.x) {
        wait(&full_bar, phase);
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
        if (tid == 0 && tile + gridDim.x < tiles) {
            fence_proxy_async();
            issue_tile(tile + gridDim.x);
        }

        if (MODE != HH_MODE_W && sign) scale2<G, NG, RT, RG>(x, sign, t);
        for (int s = 0; s < steps; ++s, ++g) {
            if (MODE == HH_MODE_SYM && s == h) scale2<G, NG, RT, RG>(x, d, t);
            const int k = kof(s);
            const int slot = resident ? k : slot_c;
            wait(&vbar[slot], resident ? 0u : par_c);
            const float4 *vk = reinterpret_cast<const float4 *>(ring + (size_t)slot * COVER);
            float2 u[E2];
#pragma unroll
            for (int i = 0; i < NG; ++i) {
                const float4 q = vk[t + G * i];
                u[2 * i] = make_float2(q.x, q.y);
                u[2 * i + 1] = make_float2(q.z, q.w);
            }
            float p[RT];
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
#pragma unroll
                for (int e = 0; e < E2; e += 2) {
                    a = __ffma2_rn(x[r][e], u[e], a);
                    if (e + 1 < E2) b = __ffma2_rn(x[r][e + 1], u[e + 1], b);
                }
                a = __fadd2_rn(a, b);
                p[r] = a.x + a.y;
            }
            const float tk = __ldg(tau + k);
            float v = fused::warp_reduce_rows<float, RT>(p, lane);
            constexpr int SH = 5 - fused::ilog2(RT);
            float c[RT];
            if constexpr (NW > 1) {
                if ((lane & ((1 << SH) - 1)) == 0) red[buf][rg][lane >> SH][warp] = v;
            }
            if (NW > 1 || !resident) __syncthreads();
            // every thread finished step g-1: its slot may be refilled with step g-1+S
            if (!resident && tid == 0 && g >= 1 && g_issue < total_steps) {
                fence_proxy_async();
                issue_reflector(kof(s_issue), slot_prev);
                ++g_issue;
                s_issue = s_issue + 1 == steps ? 0 : s_issue + 1;
            }
            if (!resident) {
                slot_prev = slot_c;
                if (++slot_c == S) {
                    slot_c = 0;
                    par_c ^= 1u;
                }
            }
            if constexpr (NW == 1) {
#pragma unroll
                for (int r = 0; r < RT; ++r) c[r] = -tk * __shfl_sync(0xffffffffu, v, r << SH);
            } else {
                float q = lane < RT * NW ? red[buf][rg][lane / NW][lane % NW] : 0.f;
#pragma unroll
                for (int off = NW / 2; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
#pragma unroll
                for (int r = 0; r < RT; ++r) c[r] = -tk * __shfl_sync(0xffffffffu, q, r * NW);
                buf ^= 1;
            }
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const float2 cc = make_float2(c[r], c[r]);
#pragma unroll
                for (int e = 0; e < E2; ++e) x[r][e] = __ffma2_rn(u[e], cc, x[r][e]);
            }
        }
        if (MODE == HH_MODE_SYM && h == 0) scale2<G, NG, RT, RG>(x, d, t);
        if (MODE != HH_MODE_WT && sign) scale2<G, NG, RT, RG>(x, sign, t);

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

// Slots of the reflector ring: all h when they fit in `budget` bytes next to
// the stage (loaded once per CTA), else as many as fit, at least 2.
template <int G, int NG, int RT, int RG>
int ring_slots(int n, int h, size_t budget) {
    using C = SCfg<G, NG, RT, RG>;
    const size_t st = stage_floats<G, NG, RT, RG>(n) * sizeof(float);
    const size_t slot = (size_t)C::COVER * sizeof(float);
    if (h <= kMaxSlots && st + (size_t)h * slot <= budget) return h > 0 ? h : 1;
    long long s = budget > st ? (long long)((budget - st) / slot) : 0;
    if (s < 2) s = 2;
    if (s > kMaxSlots) s = kMaxSlots;
    return (int)s;
}

template <int G, int NG, int RT, int RG>
cudaError_t launch(hh_mode mode, const float *X, int64_t ldx, float *Y, int64_t ldy,
                   int64_t batch, int n, const float *V, const float *tau, int64_t ldv, int h,
                   const float *sign, const float *d, int *err, int num_sms, size_t budget,
                   cudaStream_t st) {
    using C = SCfg<G, NG, RT, RG>;
    const int S = ring_slots<G, NG, RT, RG>(n, h, budget);
    const size_t smem = (stage_floats<G, NG, RT, RG>(n) + (size_t)S * C::COVER) * sizeof(float);
    if (smem > 226 * 1024) return cudaErrorInvalidConfiguration;
    const int64_t tiles = (batch + C::ROWS - 1) / C::ROWS;
    // The shared-memory opt-in is a per-kernel attribute (one entry per mode),
    // raised when a call needs more than any earlier one; the resident-CTA
    // count depends on this call's shared memory.
    static size_t attr_set[3] = {0, 0, 0};
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e;
        if (smem > attr_set[mode]) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr_set[mode] = smem;
        }
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, C::THREADS, smem);
        if (e != cudaSuccess) return e;
        if (nb < 1) return cudaErrorInvalidConfiguration;
        const int64_t slots = (int64_t)num_sms * nb;
        const int grid = (int)(tiles < slots ? tiles : slots);
        kern<<<grid, C::THREADS, smem, st>>>(X, ldx, Y, ldy, batch, n, V, tau, ldv, h, sign, d, S,
                                             err);
        return cudaGetLastError();
    };
    switch (mode) {
        case HH_MODE_W: return run(staged_chain_kernel<HH_MODE_W, G, NG, RT, RG>);
        case HH_MODE_WT: return run(staged_chain_kernel<HH_MODE_WT, G, NG, RT, RG>);
        default: return run(staged_chain_kernel<HH_MODE_SYM, G, NG, RT, RG>);
    }
}

}  // namespace staged
}  // namespace hh
