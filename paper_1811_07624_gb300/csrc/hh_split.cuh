// Column-split F32 reflector-chain kernel on clusters of CL CTAs (two in the
// configuration the library dispatches; CL = 1 keeps all of V in one CTA and
// needs no exchange when a row group is one warp).
//
// The arithmetic is the staged kernel's: the chain of §II-A (Eq. (1)-(2)),
// B consecutive reflectors per round, with the dot products of a round taken
// against the round's input and the sequential coefficients recovered exactly
// from the FP64 Gram entries,
//     z_j = v_j . x,   c_j = tau_j (z_j - sum_{i<j} c_i (v_i . v_j)),
//     x <- x - sum_j c_j v_j.
// What changes is where the reflector values come from.  The two CTAs of a
// cluster split every vector's columns in half, and each keeps its half of all
// h reflectors resident in shared memory for the whole persistent kernel, so
// inside the loop no reflector value is read from L2.  The price is one
// exchange per round: each warp's dot products cover its share of one half of
// the columns.  After a shuffle reduction inside the warp, every warp stores
// its partial sums into a receive slot of its own CTA (shared store, then an
// mbarrier arrival) and into the same slot of the peer CTA through
// distributed shared memory (st.async, completing bytes on the peer's
// mbarrier).  One barrier phase per round thus gathers all partial sums of
// both CTAs, with no named barrier between the warps, and both CTAs add them
// in the same fixed order, so both halves of a vector see bit-identical
// coefficients.
//
// Vectors go from HBM straight into registers (16-byte loads, each warp
// reading 512-byte runs); while a tile is computed the bulk-copy engine
// prefetches the row group's next tile into L2, and results leave with
// streaming stores.  Each vector is read once and written once.
//
// Layout.  A CTA is RG row groups of G threads; thread t of a group owns
// granules t + G*i (i < NG) of 4 floats, within this CTA's half, of each of
// the group's RT rows.  Row group rg of both CTAs of cluster c walks the same
// tiles of RT rows, c*RG + rg + k*(clusters*RG).
//
// Waits are bounded (about a second of clock cycles).  On expiry the thread
// records HH_ERR_TIMEOUT in *err and stops waiting; control flow stays
// uniform (every thread runs every round), so no barrier is left unmatched,
// and the kernel ends with a cluster barrier so that no CTA leaves while its
// peer may still store into it.
#pragma once

#include "hh_staged.cuh"

namespace hh {
namespace split {

using staged::bulk_g2s;
using staged::fence_proxy_async;
using staged::kGramBand;
using staged::kWaitCycles;
using staged::mbar_expect_tx;
using staged::mbar_init;
using staged::smem_u32;

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// Address of the same shared-memory variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
// Store one float into a peer CTA's shared memory; the store completes 4 bytes
// of the transaction count of the peer's mbarrier at `bar`.
__device__ __forceinline__ void st_async_f32(uint32_t addr, float v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(
                     addr),
                 "r"(__float_as_uint(v)), "r"(bar)
                 : "memory");
}
// Arrive on a local mbarrier (release at CTA scope), optionally raising the
// phase's expected transaction bytes first.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void fence_mbarrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;" ::
            : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// Phase-parity wait with acquire at cluster scope (the phase is completed by
// a peer CTA's stores), bounded by about a second of clock cycles.
__device__ __forceinline__ bool try_wait_cluster(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool wait_cluster_bounded(uint64_t *bar, uint32_t parity) {
    if (try_wait_cluster(bar, parity)) return true;
    const long long t0 = clock64();
    while (!try_wait_cluster(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

template <int G, int NG, int RT, int RG, int B>
struct XCfg {
    static constexpr int E = NG * 4;      // floats of one row held by a thread
    static constexpr int E2 = E / 2;      // float2 pairs
    static constexpr int NW = G / 32;     // warps per row group
    static constexpr int THREADS = G * RG;
    static constexpr int HALF = G * E;    // columns owned by one CTA of the pair
    static constexpr int NV = B * RT;     // dot products reduced together
    static constexpr int L = 32 / NV;     // lanes holding one value after the warp reduction
    static_assert(G % 32 == 0, "G must be a multiple of 32");
    static_assert(NV <= 32 && (NV & (NV - 1)) == 0, "B*RT must be a power of two <= 32");
    static_assert(B >= 1 && B <= kGramBand, "block larger than the stored Gram band");
};

// Scale the held columns (this CTA's half, starting at column c0) by s.
template <int G, int NG, int RT, int RG, int B>
__device__ __forceinline__ void scale_half(float2 (&x)[RT][XCfg<G, NG, RT, RG, B>::E2],
                                           const float *__restrict__ s, int c0, int t) {
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        float4 q = __ldg(reinterpret_cast<const float4 *>(s + c0) + (t + G * i));
        const float2 lo = make_float2(q.x, q.y), hi = make_float2(q.z, q.w);
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            x[r][2 * i] = __fmul2_rn(x[r][2 * i], lo);
            x[r][2 * i + 1] = __fmul2_rn(x[r][2 * i + 1], hi);
        }
    }
}

// Per-row-group exchange state: the round counter selects the receive buffer
// (round & 1) and the phase parity of its mbarrier ((round >> 1) & 1).
template <int CL>
struct Exchange {
    uint32_t round;
    uint32_t rank;               // this CTA's rank in the cluster
    uint32_t peer_slot[CL > 1 ? CL - 1 : 1];  // the other CTAs' receive slots (shared::cluster)
    uint32_t peer_bar[CL > 1 ? CL - 1 : 1];   // ... and their receive mbarriers
    bool waiting;                // false once a wait of this thread expired
};

// Apply h reflectors, ascending (k = 0..h-1) or descending, to the RT rows in
// x, B per round.  vs holds this CTA's half of every reflector (row k at
// vs + k*HALF).  With PART, granule indices i >= act (warp-uniform: their
// columns lie past this CTA's share of n) are neither read nor computed; the
// remaining terms are summed in the same order.
template <int G, int NG, int RT, int RG, int B, int CL, bool PART = false>
__device__ __forceinline__ void chain(float2 (&x)[RT][XCfg<G, NG, RT, RG, B>::E2], bool asc, int h,
                                      const float *vs, const float *__restrict__ tau,
                                      const float *__restrict__ gram, int t, int lane, int warp,
                                      float *slot, uint64_t *bars, Exchange<CL> &xc, int *err,
                                      int act = NG) {
    using C = XCfg<G, NG, RT, RG, B>;
    constexpr int E2 = C::E2, NW = C::NW, NV = C::NV, L = C::L, HALF = C::HALF;
    (void)NW;
    (void)act;
    auto load_u = [&](int s0, int j, float2(&dst)[E2]) {
        const bool ok = s0 + j < h;
        const int k = asc ? s0 + j : h - 1 - s0 - j;
        const float4 *row = reinterpret_cast<const float4 *>(vs + (size_t)(ok ? k : 0) * HALF);
#pragma unroll
        for (int i = 0; i < NG; ++i) {
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ok && (!PART || i < act)) q = row[t + G * i];
            dst[2 * i] = make_float2(q.x, q.y);
            dst[2 * i + 1] = make_float2(q.z, q.w);
        }
    };
    for (int s = 0; s < h; s += B) {
        const int nb = h - s < B ? h - s : B;
        // tau and the Gram entries of the round (uniform scalars through L1),
        // read before the reduction so their latency is not exposed after it
        float tk[B], gv[B][B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int kj = asc ? s + j : h - 1 - s - j;
            tk[j] = j < nb ? __ldg(tau + kj) : 0.f;
#pragma unroll
            for (int i = 0; i < B; ++i) {
                const int ki = asc ? s + i : h - 1 - s - i;
                gv[j][i] = (i > j && i < nb)
                               ? __ldg(gram + (size_t)(asc ? kj : ki) * kGramBand + (i - j))
                               : 0.f;
            }
        }
        float p[NV];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            float2 u[E2];
            load_u(s, j, u);
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                float2 a = make_float2(0.f, 0.f);
                if constexpr (PART) {
#pragma unroll
                    for (int i = 0; i < NG; ++i) {
                        if (i >= act) continue;
                        a = __ffma2_rn(x[r][2 * i], u[2 * i], a);
                        a = __ffma2_rn(x[r][2 * i + 1], u[2 * i + 1], a);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < E2; ++e) a = __ffma2_rn(x[r][e], u[e], a);
                }
                p[j * RT + r] = a.x + a.y;
            }
        }
        float q = fused::warp_reduce_rows<float, NV>(p, lane);  // lane holds value lane / L
        const int idx = lane / L, sub = lane & (L - 1);
        // q: this warp's part of value idx, held by the L lanes of idx.  Every
        // warp posts its part into slot [b][rank][warp][idx] of every CTA of
        // the cluster: its own with a shared store and an arrival, the others'
        // with st.async, which completes bytes on their mbarriers.  Once a
        // CTA's barrier phase completes it holds all CL*NW parts, and every
        // CTA adds them in the same fixed order.
        float zz;
        if constexpr (CL == 1 && NW == 1) {
            zz = q;  // one warp holds all columns: the shuffle reduction is the whole sum
            (void)slot;
            (void)bars;
            (void)err;
        } else {
            const uint32_t b = xc.round & 1u, par = (xc.round >> 1) & 1u;
            if (sub == 0) {
                const uint32_t off = ((b * CL + xc.rank) * NW + warp) * NV + idx;
                slot[off] = q;
#pragma unroll
                for (int pc = 0; pc < CL - 1; ++pc)
                    st_async_f32(xc.peer_slot[pc] + off * 4u, q, xc.peer_bar[pc] + b * 8u);
            }
            __syncwarp();
            if (lane == 0) {
                if (warp == 0)
                    mbar_arrive_expect_tx(bars + b, (CL - 1) * NW * NV * 4u);  // + the others' parts
                else
                    mbar_arrive(bars + b);
            }
            if (xc.waiting && !wait_cluster_bounded(bars + b, par)) {
                atomicExch(err, (int)HH_ERR_TIMEOUT);
                xc.waiting = false;
            }
            zz = 0.f;
#pragma unroll
            for (int c = 0; c < CL; ++c)
#pragma unroll
                for (int w = 0; w < NW; ++w) zz += slot[((b * CL + c) * NW + w) * NV + idx];
        }
        ++xc.round;
        float z[NV];
#pragma unroll
        for (int qq = 0; qq < NV; ++qq) z[qq] = __shfl_sync(0xffffffffu, zz, qq * L);
        // coefficients in the order the reflectors act, stored negated
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
            float2 u[E2];
            load_u(s, j, u);
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const float2 cc = make_float2(c[j][r], c[j][r]);
                if constexpr (PART) {
#pragma unroll
                    for (int i = 0; i < NG; ++i) {
                        if (i >= act) continue;
                        x[r][2 * i] = __ffma2_rn(u[2 * i], cc, x[r][2 * i]);
                        x[r][2 * i + 1] = __ffma2_rn(u[2 * i + 1], cc, x[r][2 * i + 1]);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < E2; ++e) x[r][e] = __ffma2_rn(u[e], cc, x[r][e]);
                }
            }
        }
    }
}

// Requirements (checked by the launcher): HALF < n <= 2*HALF, n % 4 == 0, X and
// Y rows and bases 16-byte aligned, V rows zero padded to ldv >= 2*HALF,
// ldv % 4 == 0, h*HALF floats of dynamic shared memory.  Launched as clusters
// of two CTAs (cluster rank = the half of the columns a CTA owns).
template <int MODE, int G, int NG, int RT, int RG, int B, int CL, int MINB, bool KP = false>
__global__ void __launch_bounds__(G *RG, MINB)
split_chain_kernel(const float *X, int64_t ldx, float *Y, int64_t ldy, int64_t batch, int n,
                   const float *__restrict__ V, const float *__restrict__ tau, int64_t ldv, int h,
                   const float *__restrict__ gram, const float *__restrict__ sign,
                   const float *__restrict__ d, int *__restrict__ err, float *__restrict__ P,
                   int64_t ldp) {
    using C = XCfg<G, NG, RT, RG, B>;
    constexpr int E2 = C::E2, NV = C::NV, HALF = C::HALF;
    extern __shared__ __align__(128) float vs[];  // h x HALF: this CTA's half of every reflector
    __shared__ __align__(8) uint64_t vbar;
    // per row group, two buffers of 2 CTAs x NW warps x NV partial dot products,
    // each completed on its own mbarrier (NW local arrivals + the peer's bytes)
    __shared__ __align__(8) uint64_t rbar[RG][2];
    __shared__ __align__(16) float rslot[RG][2 * CL * C::NW * NV];

    const int tid = threadIdx.x;
    const int rg = tid / G;
    const int t = tid - rg * G;
    const int warp = t >> 5, lane = t & 31;
    const uint32_t rank = cluster_rank();
    const int c0 = (int)rank * HALF;  // first column of this CTA's half
    const int64_t cid = cluster_id(), ncl = cluster_count();
    const int ncols = n - c0 < HALF ? n - c0 : HALF;  // columns of this half inside n

    if (tid == 0) {
        mbar_init(&vbar, 1);
        for (int g = 0; g < RG; ++g) {
            mbar_init(&rbar[g][0], C::NW);
            mbar_init(&rbar[g][1], C::NW);
        }
        fence_mbarrier_init();
        fence_proxy_async();
        if (h > 0) {
            mbar_expect_tx(&vbar, (uint32_t)h * HALF * 4u);
            for (int k = 0; k < h; ++k)
                bulk_g2s(vs + (size_t)k * HALF, V + (size_t)k * ldv + c0, HALF * 4u, &vbar);
        }
    }
    // every mbarrier of the cluster is initialised before any peer stores into it
    cluster_sync();
    Exchange<CL> xc;
    xc.round = 0;
    xc.rank = rank;
#pragma unroll
    for (int pc = 0; pc < CL - 1; ++pc) {
        const uint32_t other = (rank + 1u + (uint32_t)pc) % (uint32_t)CL;
        xc.peer_slot[pc] = peer_addr(smem_u32(&rslot[rg][0]), other);
        xc.peer_bar[pc] = peer_addr(smem_u32(&rbar[rg][0]), other);
    }
    xc.waiting = true;
    if (h > 0 && !wait_cluster_bounded(&vbar, 0)) {
        atomicExch(err, (int)HH_ERR_TIMEOUT);
        wait_cluster_bounded(&vbar, 0);  // give the copy in flight one more chance
        xc.waiting = false;
    }

    const int64_t rtiles = (batch + RT - 1) / RT;
    for (int64_t tl = cid * RG + rg; tl < rtiles; tl += ncl * RG) {
        const int64_t r0 = tl * RT;
        // the group's next tile into L2 while this one is computed
        if (t == 0) {
            const int64_t nr0 = (tl + ncl * RG) * RT;
#pragma unroll
            for (int r = 0; r < RT; ++r)
                if (ncols > 0 && nr0 + r < batch)
                    prefetch_l2(X + (nr0 + r) * ldx + c0, (uint32_t)ncols * 4u);
        }
        float2 x[RT][E2];
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const bool valid = r0 + r < batch;
            const float *xr = X + (r0 + r) * ldx + c0;
#pragma unroll
            for (int i = 0; i < NG; ++i) {
                const int col = (t + G * i) * 4;
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                if (valid && col < ncols) q = __ldcs(reinterpret_cast<const float4 *>(xr + col));
                x[r][2 * i] = make_float2(q.x, q.y);
                x[r][2 * i + 1] = make_float2(q.z, q.w);
            }
        }
        if (MODE != HH_MODE_W && sign) scale_half<G, NG, RT, RG, B>(x, sign, c0, t);
        // W: k = h..1; W^T: k = 1..h; S: k = 1..h, scale by d, k = h..1
        for (int half = 0; half < (MODE == HH_MODE_SYM ? 2 : 1); ++half) {
            if (half == 1) {
                // mode S with P (KP): p = W^T (sigma .* x), the state between the halves
                if constexpr (KP)
#pragma unroll
                    for (int r = 0; r < RT; ++r) {
                        if (r0 + r >= batch) continue;
                        float *pr = P + (r0 + r) * ldp + c0;
#pragma unroll
                        for (int i = 0; i < NG; ++i) {
                            const int col = (t + G * i) * 4;
                            if (col < ncols)
                                __stcs(reinterpret_cast<float4 *>(pr + col),
                                       make_float4(x[r][2 * i].x, x[r][2 * i].y,
                                                   x[r][2 * i + 1].x, x[r][2 * i + 1].y));
                        }
                    }
                scale_half<G, NG, RT, RG, B>(x, d, c0, t);
            }
            const bool asc = MODE != HH_MODE_W && half == 0;
            chain<G, NG, RT, RG, B, CL>(x, asc, h, vs, tau, gram, t, lane, warp, &rslot[rg][0],
                                        &rbar[rg][0], xc, err);
        }
        if (MODE != HH_MODE_WT && sign) scale_half<G, NG, RT, RG, B>(x, sign, c0, t);
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            if (r0 + r >= batch) continue;
            float *yr = Y + (r0 + r) * ldy + c0;
#pragma unroll
            for (int i = 0; i < NG; ++i) {
                const int col = (t + G * i) * 4;
                if (col < ncols)
                    __stcs(reinterpret_cast<float4 *>(yr + col),
                           make_float4(x[r][2 * i].x, x[r][2 * i].y, x[r][2 * i + 1].x,
                                       x[r][2 * i + 1].y));
            }
        }
    }
    // no CTA leaves while its peer may still store into its receive slots
    __syncthreads();
    cluster_sync();
}

// Largest dynamic shared memory a launch may request (h*HALF floats): one CTA
// per SM may take 200 KiB, two take 100 KiB each.
template <int MINB>
constexpr size_t max_smem() {
    return MINB >= 2 ? 100 * 1024 : 200 * 1024;
}

template <int G, int NG, int RT, int RG, int B, int MINB = 1>
constexpr int max_h() {
    return (int)(max_smem<MINB>() / (XCfg<G, NG, RT, RG, B>::HALF * sizeof(float)));
}

// Per configuration, kernel (W, W^T, S, S keeping p) and device: the
// shared-memory opt-in at the largest request and the co-resident clusters
// measured with it.
template <int G, int NG, int RT, int RG, int B, int CL, int MINB>
inline PerDevice g_state[4];

template <int G, int NG, int RT, int RG, int B, int CL, int MINB, typename K>
cudaError_t cluster_occupancy(K kern, int si, int &ncl) {
    using C = XCfg<G, NG, RT, RG, B>;
    constexpr size_t kMaxSmem = max_smem<MINB>();
    return per_device(g_state<G, NG, RT, RG, B, CL, MINB>[si], ncl, [&](int &v) -> cudaError_t {
        cudaError_t e2 =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
        if (e2 != cudaSuccess) return e2;
        cudaLaunchConfig_t q = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        q.blockDim = dim3(C::THREADS);
        q.gridDim = dim3(CL);
        q.dynamicSmemBytes = kMaxSmem;
        q.attrs = attr;
        q.numAttrs = 1;
        int nc = 0;
        e2 = cudaOccupancyMaxActiveClusters(&nc, kern, &q);
        if (e2 != cudaSuccess) return e2;
        v = nc > 0 ? nc : 1;
        return cudaSuccess;
    });
}

// Clusters of the mode's kernel (without p) that can be resident at once.
template <int G, int NG, int RT, int RG, int B, int CL = 2, int MINB = 1>
cudaError_t resident_clusters(hh_mode mode, int &ncl) {
    switch (mode) {
        case HH_MODE_W:
            return cluster_occupancy<G, NG, RT, RG, B, CL, MINB>(
                split_chain_kernel<HH_MODE_W, G, NG, RT, RG, B, CL, MINB>, 0, ncl);
        case HH_MODE_WT:
            return cluster_occupancy<G, NG, RT, RG, B, CL, MINB>(
                split_chain_kernel<HH_MODE_WT, G, NG, RT, RG, B, CL, MINB>, 1, ncl);
        default:
            return cluster_occupancy<G, NG, RT, RG, B, CL, MINB>(
                split_chain_kernel<HH_MODE_SYM, G, NG, RT, RG, B, CL, MINB>, 2, ncl);
    }
}

// CL CTAs per cluster split the columns (CTA r owns [r*HALF, (r+1)*HALF));
// MINB CTAs per SM bound the registers.  Mode S with P also writes
// p = W^T (sigma .* x) (rows of P, leading dimension ldp, 16-byte aligned).
// high_priority: the launch takes the device's highest scheduling priority
// (for a launch that shares the GPU with one on another stream).
template <int G, int NG, int RT, int RG, int B, int CL = 2, int MINB = 1>
cudaError_t launch(hh_mode mode, const float *X, int64_t ldx, float *Y, int64_t ldy,
                   int64_t batch, int n, const float *V, const float *tau, int64_t ldv, int h,
                   const float *gram, const float *sign, const float *d, int *err,
                   cudaStream_t st, float *P = nullptr, int64_t ldp = 0,
                   bool high_priority = false) {
    using C = XCfg<G, NG, RT, RG, B>;
    if (n < 1 || n > CL * C::HALF || n % 4 || ldv < CL * C::HALF || ldv % 4 ||
        h > max_h<G, NG, RT, RG, B, MINB>())
        return cudaErrorInvalidValue;
    const size_t smem = h > 0 ? (size_t)h * C::HALF * sizeof(float) : 16;
    int prio_least = 0, prio_greatest = 0;
    if (high_priority) {
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
        if (e != cudaSuccess) return e;
    }
    auto run = [&](auto kern, int si) -> cudaError_t {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        attr[1].id = cudaLaunchAttributePriority;
        attr[1].val.priority = prio_greatest;
        cfg.blockDim = dim3(C::THREADS);
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = high_priority ? 2 : 1;
        int ncl = 1;
        cudaError_t e = cluster_occupancy<G, NG, RT, RG, B, CL, MINB>(kern, si, ncl);
        if (e != cudaSuccess) return e;
        const int64_t groups = ((batch + RT - 1) / RT + RG - 1) / RG;  // row-group tiles / RG
        const int grid_cl = (int)(groups < ncl ? groups : ncl);
        cfg.gridDim = dim3(CL * grid_cl);
        cfg.dynamicSmemBytes = smem;
        return cudaLaunchKernelEx(&cfg, kern, X, ldx, Y, ldy, batch, n, V, tau, ldv, h, gram,
                                  sign, d, err, mode == HH_MODE_SYM ? P : nullptr, ldp);
    };
    switch (mode) {
        case HH_MODE_W: return run(split_chain_kernel<HH_MODE_W, G, NG, RT, RG, B, CL, MINB>, 0);
        case HH_MODE_WT: return run(split_chain_kernel<HH_MODE_WT, G, NG, RT, RG, B, CL, MINB>, 1);
        default:
            if (P) return run(split_chain_kernel<HH_MODE_SYM, G, NG, RT, RG, B, CL, MINB, true>, 3);
            return run(split_chain_kernel<HH_MODE_SYM, G, NG, RT, RG, B, CL, MINB>, 2);
    }
}

}  // namespace split
}  // namespace hh
