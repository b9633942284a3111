// Staged F32 reflector-chain kernel: the fused chain of hh_fused.cuh with the
// next tile of vectors prefetched into shared memory by the bulk-copy engine
// (cp.async.bulk + mbarrier) while the current tile is computed in registers.
//
// Per reflector (§II-A, Eq. (2)): c = tau_k (v_k . x), x <- x - c v_k, in the
// mode orders of Eq. (1) / Eq. (21).  Each vector is read from HBM once (into
// shared memory, then registers) and written once (registers -> HBM).
//
// Layout: persistent CTAs (as many per SM as fit), RG row groups of G threads; thread t of
// a group owns granules t + G*i (i < NG) of 4 floats of each of its RT rows.
// Within a group the RT partial dot products are reduced by a transposing warp
// shuffle, then across the group's G/32 warps through shared memory behind a
// named barrier (one per group, so groups run independently).  Arithmetic on
// pairs of columns uses the packed FP32 FMA (fma.rn.f32x2).
//
// Waits on the mbarrier are bounded (~1 s of clock cycles); on expiry the
// kernel records HH_ERR_TIMEOUT in *err, waits once more (bounded) for its
// copy, and returns.
#pragma once

#include "hh_fused.cuh"

namespace hh {
namespace staged {

constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

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

// Bounded wait: true when the phase with the given parity completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
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

__device__ __forceinline__ void named_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int G, int NG, int RT, int RG>
struct SCfg {
    static constexpr int E = NG * 4;      // floats of one row held by a thread
    static constexpr int E2 = E / 2;      // float2 pairs
    static constexpr int NW = G / 32;
    static constexpr int THREADS = G * RG;
    static constexpr int ROWS = RT * RG;  // rows per tile
    static constexpr int COVER = G * E;
    static_assert(G % 32 == 0 && RT * NW <= 32, "bad staged configuration");
};

// Pull the cache lines of a reflector a thread group will need soon into L1:
// a warp's granules of one reflector are NG runs of 512 bytes (4 lines each);
// lane j < 4*NG fetches line j % 4 of run j / 4.
template <int G, int NG>
__device__ __forceinline__ void prefetch_reflector(const float *vk, int warp, int lane) {
    if (lane < 4 * NG) {
        const char *p = reinterpret_cast<const char *>(vk) +
                        16 * ((size_t)warp * 32 + (size_t)G * (lane >> 2)) + 128 * (lane & 3);
        asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
    }
}

template <int G, int NG, int RT, int RG>
__device__ __forceinline__ void reflect2(float2 (&x)[RT][SCfg<G, NG, RT, RG>::E2],
                                         const float *__restrict__ vk, float tk,
                                         const float *vpre, int t, int lane, int warp, int rg,
                                         float (*red)[RG][RT][SCfg<G, NG, RT, RG>::NW], int &buf) {
    using C = SCfg<G, NG, RT, RG>;
    constexpr int E2 = C::E2, NW = C::NW;
    if (vpre) prefetch_reflector<G, NG>(vpre, warp, lane);
    float2 u[E2];
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        float4 q = __ldg(reinterpret_cast<const float4 *>(vk) + (t + G * i));
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
    float v = fused::warp_reduce_rows<float, RT>(p, lane);
    constexpr int SH = 5 - fused::ilog2(RT);
    float c[RT];
    if constexpr (NW == 1) {
#pragma unroll
        for (int r = 0; r < RT; ++r) c[r] = -tk * __shfl_sync(0xffffffffu, v, r << SH);
    } else {
        if ((lane & ((1 << SH) - 1)) == 0) red[buf][rg][lane >> SH][warp] = v;
        named_bar(1 + rg, G);
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

// Requirements (checked by the launcher): n % 4 == 0, n <= COVER, X rows and
// base 16-byte aligned, ROWS * n * 4 bytes of dynamic shared memory.
template <int MODE, int G, int NG, int RT, int RG>
__global__ void __launch_bounds__(G *RG)
staged_chain_kernel(const float *X, int64_t ldx, float *Y, int64_t ldy, int64_t batch, int n,
                    const float *__restrict__ V, const float *__restrict__ tau, int64_t ldv,
                    int h, const float *__restrict__ sign, const float *__restrict__ d,
                    int *__restrict__ err) {
    using C = SCfg<G, NG, RT, RG>;
    constexpr int E2 = C::E2, NW = C::NW, ROWS = C::ROWS;
    extern __shared__ __align__(128) float stage[];  // ROWS x n
    __shared__ __align__(8) uint64_t full_bar;
    __shared__ float red[2][RG][RT][NW];
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    const int rg = tid / G;
    const int t = tid - rg * G;
    const int warp = t >> 5, lane = t & 31;
    const int64_t tiles = (batch + ROWS - 1) / ROWS;
    int64_t tile = blockIdx.x;
    if (tile >= tiles) return;
    const uint32_t row_bytes = (uint32_t)n * 4u;

    auto issue = [&](int64_t tl) {
        const int64_t r0 = tl * ROWS;
        const int64_t left = batch - r0;
        const int nvalid = left < ROWS ? (int)left : ROWS;
        mbar_expect_tx(&full_bar, row_bytes * (uint32_t)nvalid);
        for (int r = 0; r < nvalid; ++r)
            bulk_g2s(stage + (size_t)r * n, X + (r0 + r) * ldx, row_bytes, &full_bar);
    };

    if (tid == 0) {
        abort_flag = 0;
        mbar_init(&full_bar, 1);
        fence_proxy_async();
        issue(tile);
    }
    __syncthreads();

    uint32_t phase = 0;
    int buf = 0;
    for (; tile < tiles; tile += gridDim.x) {
        const bool ok = mbar_wait_bounded(&full_bar, phase);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(err, (int)HH_ERR_TIMEOUT);
                mbar_wait_bounded(&full_bar, phase);  // let the copy in flight land
            }
            __syncthreads();
            return;
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
        if (tid == 0 && tile + gridDim.x < tiles) {
            fence_proxy_async();
            issue(tile + gridDim.x);
        }

        if (MODE != HH_MODE_W && sign) scale2<G, NG, RT, RG>(x, sign, t);
        // One loop over the chain steps of the mode (a single loop body keeps the
        // symmetric mode within the register budget): W runs k = h..1, W^T runs
        // k = 1..h, S runs k = 1..h, scales by d, then k = h..1.
        const int steps = MODE == HH_MODE_SYM ? 2 * h : h;
        auto kof = [&](int s) {
            return MODE == HH_MODE_W ? h - 1 - s
                                     : (MODE == HH_MODE_WT ? s : (s < h ? s : 2 * h - 1 - s));
        };
        for (int s = 0; s < steps; ++s) {
            if (MODE == HH_MODE_SYM && s == h) scale2<G, NG, RT, RG>(x, d, t);
            const int k = kof(s);
            const float *vpre = s + 2 < steps ? V + (size_t)kof(s + 2) * ldv : nullptr;
            reflect2<G, NG, RT, RG>(x, V + (size_t)k * ldv, __ldg(tau + k), vpre, t, lane, warp,
                                    rg, red, buf);
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
    (void)abort_flag;
}

template <int G, int NG, int RT, int RG>
cudaError_t launch(hh_mode mode, const float *X, int64_t ldx, float *Y, int64_t ldy,
                   int64_t batch, int n, const float *V, const float *tau, int64_t ldv, int h,
                   const float *sign, const float *d, int *err, int num_sms, cudaStream_t st) {
    using C = SCfg<G, NG, RT, RG>;
    const size_t smem = (size_t)C::ROWS * n * sizeof(float);
    const int64_t tiles = (batch + C::ROWS - 1) / C::ROWS;
    // The shared-memory opt-in and the resident-CTA count are per kernel: one
    // entry per mode, filled on first use (the count at the largest stage).
    static bool attr_done[3] = {false, false, false};
    static int per_sm[3] = {0, 0, 0};
    auto run = [&](auto kern) -> cudaError_t {
        if (!attr_done[mode]) {
            const size_t smax = (size_t)C::ROWS * C::COVER * sizeof(float);
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smax);
            if (e != cudaSuccess) return e;
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, C::THREADS, smax);
            if (e != cudaSuccess) return e;
            per_sm[mode] = nb > 0 ? nb : 1;
            attr_done[mode] = true;
        }
        const int64_t slots = (int64_t)num_sms * per_sm[mode];
        const int grid = (int)(tiles < slots ? tiles : slots);
        kern<<<grid, C::THREADS, smem, st>>>(X, ldx, Y, ldy, batch, n, V, tau, ldv, h, sign, d,
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
