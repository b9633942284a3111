// Batched persistent launch: many independent reflector chains (§II-A, Eqs.
// (1)-(2) and the symmetric form of Eq. (21)) of uneven n, h and batch size in
// one kernel launch, captured once in a CUDA graph and replayed.
//
// Work list.  Each transform's rows are cut into tiles (ROWS rows of its tile
// shape); runs of tiles form items of roughly equal cost, and items are sorted
// by cost, largest first.  The persistent CTAs take items from an atomic
// counter (the index of the next item is fetched one item ahead) and walk their
// tiles; the next tile's rows are brought into shared memory by the bulk-copy
// engine while the current tile is computed, as in the single-transform staged
// kernel.
//
// Tile shapes.  One kernel holds several (G, NG, RT, B) layouts of 256
// threads: RG = 256 / G row groups of G threads, each thread RT rows x NG
// granules of 4 floats (64 or 128 floats of vector state), COVER = G * NG * 4
// columns, B reflectors per reduction round.  The arithmetic is the
// single-transform kernel's chain (staged::chain, the Gram-corrected blocked
// rounds), instantiated per shape with its partial-cover option: a warp whose
// granule i lies past n neither reads nor computes it (a warp-uniform test),
// so a transform of n columns costs n, not COVER, columns of arithmetic.  The
// kernel runs one CTA of 256 threads per SM with up to 255 registers per
// thread.  Shapes are chosen per (n, h) by the autotuner (hh_tune), which
// times every shape that covers n on synthetic data and keeps the fastest;
// untuned shapes fall back to the nearest tuned h for that n, then to a fixed
// rule.
//
// Resident shape.  A further shape keeps each transform's reflectors in shared
// memory instead of reading them from L2 once per tile: clusters of
// ceil(n / 512) CTAs split the columns as the single-transform column-split
// kernel does, one launch per cluster size, each on a static schedule that
// hands every cluster a contiguous stretch of its tasks (see
// cluster_batch_kernel).  The autotuner times it beside the staged shapes.
// All launches of a batch and mode are captured in one graph.
//
// Streams.  A batch's work counter and task table are shared by its launches;
// a launch on a stream other than the previous launch's first waits for that
// launch (an event), so calls on different streams never overlap on them.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "hh_split.cuh"

namespace hh {
namespace batched {

#ifndef HH_BATCH_FORK
#define HH_BATCH_FORK 1  // the launches of one graph on parallel branches (0: in sequence)
#endif

constexpr int kThreads = 256;
constexpr int kNumShapes = 11;
constexpr int kClusterShape = 10;        // resident reflectors, clusters of CTAs (below)
constexpr int kStageBytes = 128 * 1024;  // >= ROWS * COVER * 4 for every shape
constexpr int kRedFloats = 512;          // >= 2 * RG * (B * RT) * NW for every shape

struct ShapeInfo {
    int G, NG, RT, B;
};
static const ShapeInfo kShape[kNumShapes] = {
    {32, 1, 16, 2},   // 0: COVER  128, 128 rows per tile,  64 floats per thread
    {32, 2, 16, 2},   // 1: COVER  256, 128 rows, 128 floats
    {32, 4, 8, 2},    // 2: COVER  512,  64 rows, 128 floats
    {32, 8, 4, 2},    // 3: COVER 1024,  32 rows, 128 floats
    {32, 8, 4, 4},    // 4: COVER 1024,  32 rows, 128 floats, 4 reflectors per round
    {64, 4, 4, 4},    // 5: COVER 1024,  16 rows,  64 floats, 4 reflectors per round
    {64, 8, 4, 2},    // 6: COVER 2048,  16 rows, 128 floats
    {128, 4, 4, 4},   // 7: COVER 2048,   8 rows,  64 floats, 4 reflectors per round
    {128, 8, 4, 2},   // 8: COVER 4096,   8 rows, 128 floats
    {32, 4, 8, 4},    // 9: COVER  512,  64 rows, 128 floats, 4 reflectors per round
    {32, 4, 8, 4},    // 10: resident reflectors, 512 columns per CTA, clusters of up to
                      //     four CTAs: COVER 2048, 64 rows, h <= 100
};
constexpr int kClusterHalf = 512;    // columns of one CTA of the resident shape
constexpr int kClusterMaxCL = 4;     // CTAs per cluster: n <= 4 * 512
constexpr int kClusterMaxH = 100;    // h * 512 floats <= 200 KiB of shared memory
inline int shape_cover(int s) {
    return s == kClusterShape ? kClusterMaxCL * kClusterHalf : kShape[s].G * kShape[s].NG * 4;
}
inline int shape_rows(int s) { return kShape[s].RT * (kThreads / kShape[s].G); }
constexpr int kMaxN = 4096;

// One transform as the kernel sees it.
struct Task {
    const float *X;
    float *Y;
    int64_t ldx, ldy, rows;
    const float *V, *tau, *gram, *sign, *d;
    int64_t ldv;
    int n, h, shape, rows_per_tile;
};
// A run of ntiles tiles of one task, starting at tile0.
struct Item {
    int64_t tile0;
    int task, ntiles;
};

// Block-wide state of the batched kernel, in shared memory so that the
// per-shape tile functions (compiled separately, see below) reach it without
// pointers: the tile stage, its mbarrier, the reduction buffer, the current and
// next tile (two slots), the abort flag, and the scheduler state used by
// thread 0 (the index of the next item, fetched one item ahead; the current
// item's task, tile and tiles left).
extern __shared__ __align__(128) float b_stage[];
__shared__ __align__(8) uint64_t b_full_bar;
__shared__ __align__(16) float b_red[kRedFloats];
__shared__ int b_task[2];
__shared__ long long b_tile[2];
__shared__ int b_aborted;
__shared__ int b_pend, b_ctask, b_left;
__shared__ long long b_ctile;

// Thread 0: the tile after the current one (or task -1) into slot `out`.
__device__ __forceinline__ void advance(const Item *__restrict__ items, int nitems, int *counter,
                                        int out) {
    int task = -1;
    long long tl = 0;
    if (b_left > 0) {
        tl = ++b_ctile;
        --b_left;
        task = b_ctask;
    } else if (b_pend < nitems) {
        const Item it = items[b_pend];
        b_pend = atomicAdd(counter, 1);
        b_ctask = task = it.task;
        b_ctile = tl = it.tile0;
        b_left = it.ntiles - 1;
    }
    b_task[out] = task;
    b_tile[out] = tl;
}

// Thread 0: bring the rows of tile `tl` of task `task` into the stage.
__device__ __forceinline__ void issue_copy(const Task *__restrict__ tasks, int task, int64_t tl) {
    const Task &tk = tasks[task];
    const int rpt = tk.rows_per_tile;
    const int64_t r0 = tl * rpt;
    const int64_t rest = tk.rows - r0;
    const int nvalid = rest < rpt ? (int)rest : rpt;
    const uint32_t row_bytes = (uint32_t)tk.n * 4u;
    staged::mbar_expect_tx(&b_full_bar, row_bytes * (uint32_t)nvalid);
    const float *src = tk.X + r0 * tk.ldx;
    if (tk.ldx == tk.n) {
        staged::bulk_g2s(b_stage, src, row_bytes * (uint32_t)nvalid, &b_full_bar);
    } else {
        for (int r = 0; r < nvalid; ++r)
            staged::bulk_g2s(b_stage + (size_t)r * tk.n, src + r * tk.ldx, row_bytes, &b_full_bar);
    }
}

// One tile of the task in slot `slot` with shape (G, NG, RT, B): rows from
// the stage into registers, the stage handed to the next tile's copy, the
// chain of `mode`, and the rows stored.  Not inlined, so every shape gets its
// own register allocation.  Returns the reduction-buffer parity.
template <int G, int NG, int RT, int B>
__device__ __noinline__ int tile_body(const Task *__restrict__ tasks, int slot, int mode, int buf) {
    constexpr int RG = kThreads / G;
    using C = staged::SCfg<G, NG, RT, RG, B>;
    constexpr int E2 = C::E2, ROWS = C::ROWS;
    static_assert(ROWS * C::COVER * 4 <= kStageBytes, "stage size");
    static_assert(2 * RG * C::NV * C::NW <= kRedFloats, "reduction buffer");
    const Task &tk = tasks[b_task[slot]];
    const int64_t tile = b_tile[slot];
    const int tid = threadIdx.x;
    const int rg = tid / G;
    const int t = tid - rg * G;
    const int warp = t >> 5, lane = t & 31;
    const int n = tk.n;
    const int64_t rows = tk.rows;
    // granule indices i with this warp's first column (32 * warp + G * i) * 4 < n
    const int n4 = n >> 2;
    int act = 0;
    if (n4 > 32 * warp) {
        act = (n4 - 32 * warp + G - 1) / G;
        if (act > NG) act = NG;
    }
    const int64_t r0 = tile * ROWS;
    float2 x[RT][E2];
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        const int lr = rg * RT + r;
        const bool valid = r0 + lr < rows;
        const float *srow = b_stage + (size_t)lr * n;
#pragma unroll
        for (int i = 0; i < NG; ++i) {
            const int col = (t + G * i) * 4;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < act && valid && col < n) q = *reinterpret_cast<const float4 *>(srow + col);
            x[r][2 * i] = make_float2(q.x, q.y);
            x[r][2 * i + 1] = make_float2(q.z, q.w);
        }
    }
    __syncthreads();  // every thread has its rows: the stage may be refilled
    if (tid == 0 && b_task[slot ^ 1] >= 0 && !*(volatile int *)&b_aborted) {
        staged::fence_proxy_async();
        issue_copy(tasks, b_task[slot ^ 1], b_tile[slot ^ 1]);
    }

    const float *sign = tk.sign;
    if (mode != HH_MODE_W && sign) staged::scale2_part<G, NG, RT, RG, B>(x, sign, t, act);
    for (int half = 0; half < (mode == HH_MODE_SYM ? 2 : 1); ++half) {
        if (half == 1) staged::scale2_part<G, NG, RT, RG, B>(x, tk.d, t, act);
        const bool asc = mode != HH_MODE_W && half == 0;
        staged::chain<G, NG, RT, RG, B, false, true>(x, asc, tk.h, tk.V, tk.ldv, tk.tau, tk.gram,
                                                     t, lane, warp, rg, b_red, buf, nullptr, act);
    }
    if (mode != HH_MODE_WT && sign) staged::scale2_part<G, NG, RT, RG, B>(x, sign, t, act);

    float *Y = tk.Y;
    const int64_t ldy = tk.ldy;
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        const int64_t row = r0 + rg * RT + r;
        if (row >= rows) continue;
        float *yr = Y + row * ldy;
#pragma unroll
        for (int i = 0; i < NG; ++i) {
            if (i >= act) break;
            const int col = (t + G * i) * 4;
            if (col < n)
                __stcs(reinterpret_cast<float4 *>(yr + col),
                       make_float4(x[r][2 * i].x, x[r][2 * i].y, x[r][2 * i + 1].x,
                                   x[r][2 * i + 1].y));
        }
    }
    return buf;
}

// Requirements (checked on the host): every task n % 4 == 0, n <= COVER of its
// shape, X and Y 16-byte aligned with ldx % 4 == 0, V rows zero padded to
// ldv >= round_up(n, 128); *counter == 0 at launch; kStageBytes of dynamic
// shared memory.
__global__ void __launch_bounds__(kThreads, 1)
batched_chain_kernel(const Task *__restrict__ tasks, const Item *__restrict__ items, int nitems,
                     int *__restrict__ counter, int mode, int *__restrict__ err) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        b_aborted = 0;
        staged::mbar_init(&b_full_bar, 1);
        staged::fence_proxy_async();
        b_left = 0;
        b_pend = atomicAdd(counter, 1);
        advance(items, nitems, counter, 0);
        if (b_task[0] >= 0) issue_copy(tasks, b_task[0], b_tile[0]);
    }
    __syncthreads();

    uint32_t phase = 0;
    int buf = 0, slot = 0;
    for (;;) {
        const int task = b_task[slot];
        if (task < 0) break;
        // the next tile, read by all after the barrier in tile_body
        if (tid == 0) advance(items, nitems, counter, slot ^ 1);
        if (!*(volatile int *)&b_aborted && !staged::mbar_wait_bounded(&b_full_bar, phase)) {
            atomicExch(err, (int)HH_ERR_TIMEOUT);
            staged::mbar_wait_bounded(&b_full_bar, phase);  // one more chance for the copy in flight
            *(volatile int *)&b_aborted = 1;
        }
        phase ^= 1;
        switch (tasks[task].shape) {
            case 0: buf = tile_body<32, 1, 16, 2>(tasks, slot, mode, buf); break;
            case 1: buf = tile_body<32, 2, 16, 2>(tasks, slot, mode, buf); break;
            case 2: buf = tile_body<32, 4, 8, 2>(tasks, slot, mode, buf); break;
            case 3: buf = tile_body<32, 8, 4, 2>(tasks, slot, mode, buf); break;
            case 4: buf = tile_body<32, 8, 4, 4>(tasks, slot, mode, buf); break;
            case 5: buf = tile_body<64, 4, 4, 4>(tasks, slot, mode, buf); break;
            case 6: buf = tile_body<64, 8, 4, 2>(tasks, slot, mode, buf); break;
            case 7: buf = tile_body<128, 4, 4, 4>(tasks, slot, mode, buf); break;
            case 8: buf = tile_body<128, 8, 4, 2>(tasks, slot, mode, buf); break;
            default: buf = tile_body<32, 4, 8, 4>(tasks, slot, mode, buf); break;
        }
        slot ^= 1;
    }
}

// ---- resident-reflector tiles (shape kClusterShape) ----
//
// The transforms of this shape run on the column-split kernel's layout
// (split::chain): a cluster of CL = ceil(n / 512) CTAs splits every vector's
// columns, 512 per CTA, and each CTA holds its columns of all h reflectors in
// shared memory while it works on that transform, so no reflector value is
// read from L2 inside the row loop.  One kernel per CL (1..4) takes a static,
// transform-ordered schedule built on the host: cluster c walks items
// cstart[c] .. cstart[c+1]-1, each a run of rows of one task, and loads a
// task's reflectors once, when its first item begins.  Row group rg of every
// CTA of the cluster takes the same tiles of RT rows of an item
// (rg, rg + RG, ...), so the per-round exchange of partial dot products pairs
// up across the cluster exactly as in the single-transform kernel.
constexpr int kCG = 32, kCNG = 4, kCRT = 8, kCRG = kThreads / kCG, kCB = 4;
using CCfg = split::XCfg<kCG, kCNG, kCRT, kCRG, kCB>;
static_assert(CCfg::HALF == kClusterHalf, "resident shape: 512 columns per CTA");
static_assert(CCfg::THREADS == kThreads, "resident shape: 256 threads");
constexpr int kClusterUnit = kCRT * kCRG;  // rows of one pass of the row groups
constexpr int kClusterSmem = kClusterMaxH * kClusterHalf * 4;

// Rows [r0, r1) of task `task`.
struct CItem {
    int task, pad;
    int64_t r0, r1;
};

// Scale the first `act` granules of the held columns (this CTA's, from s) by s.
__device__ __forceinline__ void cscale(float2 (&x)[kCRT][CCfg::E2], const float *__restrict__ s,
                                       int t, int act, int ncols) {
#pragma unroll
    for (int i = 0; i < kCNG; ++i) {
        if (i >= act) break;
        const int col = (t + kCG * i) * 4;
        if (col >= ncols) continue;
        const float4 q = __ldg(reinterpret_cast<const float4 *>(s + col));
        const float2 lo = make_float2(q.x, q.y), hi = make_float2(q.z, q.w);
#pragma unroll
        for (int r = 0; r < kCRT; ++r) {
            x[r][2 * i] = __fmul2_rn(x[r][2 * i], lo);
            x[r][2 * i + 1] = __fmul2_rn(x[r][2 * i + 1], hi);
        }
    }
}

// Requirements (checked on the host): every task of the launch has
// (CL - 1) * 512 < n <= CL * 512, n % 4 == 0, h <= kClusterMaxH, V rows zero
// padded to at least round_up(n, 128) columns, X and Y 16-byte aligned with
// ldx % 4 == 0 and ldy % 4 == 0; items of a cluster in task order; the
// dynamic shared memory holds max h * 512 floats.  Waits are bounded: on
// expiry the status word gets HH_ERR_TIMEOUT, no further reflector copy is
// issued, and the copy in flight gets one more bounded wait before the CTA
// leaves.
template <int MODE, int CL>
__global__ void __launch_bounds__(kThreads, 1)
cluster_batch_kernel(const Task *__restrict__ tasks, const CItem *__restrict__ items,
                     const int *__restrict__ cstart, int *__restrict__ err) {
    constexpr int G = kCG, NG = kCNG, RT = kCRT, RG = kCRG, B = kCB;
    constexpr int E2 = CCfg::E2, NV = CCfg::NV, NW = CCfg::NW, HALF = CCfg::HALF;
    float *vs = b_stage;  // h x HALF: this CTA's columns of the current task's reflectors
    __shared__ __align__(8) uint64_t vbar;
    __shared__ __align__(8) uint64_t rbar[RG][2];
    __shared__ __align__(16) float rslot[RG][2 * CL * NW * NV];
    __shared__ int aborted;

    const int tid = threadIdx.x;
    const int rg = tid / G;
    const int t = tid - rg * G;
    const int warp = t >> 5, lane = t & 31;
    const uint32_t rank = split::cluster_rank();
    const int c0 = (int)rank * HALF;
    const int cid = (int)split::cluster_id();

    if (tid == 0) {
        aborted = 0;
        staged::mbar_init(&vbar, 1);
        for (int g = 0; g < RG; ++g) {
            staged::mbar_init(&rbar[g][0], NW);
            staged::mbar_init(&rbar[g][1], NW);
        }
        split::fence_mbarrier_init();
        staged::fence_proxy_async();
    }
    // every mbarrier of the cluster is initialised before any peer stores into it
    split::cluster_sync();
    split::Exchange<CL> xc;
    xc.round = 0;
    xc.rank = rank;
#pragma unroll
    for (int pc = 0; pc < CL - 1; ++pc) {
        const uint32_t other = (rank + 1u + (uint32_t)pc) % (uint32_t)CL;
        xc.peer_slot[pc] = split::peer_addr(staged::smem_u32(&rslot[rg][0]), other);
        xc.peer_bar[pc] = split::peer_addr(staged::smem_u32(&rbar[rg][0]), other);
    }
    xc.waiting = true;

    uint32_t vphase = 0, last_par = 0;
    int issued = 0, confirmed = 0;  // reflector copies of thread 0, and those seen complete
    int cur = -1;
    const int i1 = cstart[cid + 1];
    for (int it = cstart[cid]; it < i1; ++it) {
        const CItem item = items[it];
        const Task &tk = tasks[item.task];
        const int n = tk.n, h = tk.h;
        const int ncols = n - c0 < HALF ? n - c0 : HALF;  // >= 1 for CL = ceil(n / HALF)
        const int act = (ncols + G * 4 - 1) / (G * 4);   // granules of a thread inside n
        if (item.task != cur) {
            __syncthreads();  // every row group is done with the previous reflectors
            if (h > 0) {
                if (tid == 0 && !*(volatile int *)&aborted) {
                    staged::fence_proxy_async();
                    const uint32_t rowb = (uint32_t)act * G * 16u;
                    staged::mbar_expect_tx(&vbar, rowb * (uint32_t)h);
                    for (int k = 0; k < h; ++k)
                        staged::bulk_g2s(vs + (size_t)k * HALF, tk.V + (size_t)k * tk.ldv + c0, rowb,
                                         &vbar);
                    ++issued;
                    last_par = vphase;
                }
                if (!*(volatile int *)&aborted) {
                    if (split::wait_cluster_bounded(&vbar, vphase)) {
                        if (tid == 0) ++confirmed;
                    } else {
                        atomicExch(err, (int)HH_ERR_TIMEOUT);
                        *(volatile int *)&aborted = 1;
                    }
                }
                vphase ^= 1u;
            }
            cur = item.task;
        }
        const float *X = tk.X;
        float *Y = tk.Y;
        const int64_t ldx = tk.ldx, ldy = tk.ldy, rb = item.r0, re = item.r1;
        const int64_t ntl = (re - rb + RT - 1) / RT;
        for (int64_t tl = rg; tl < ntl; tl += RG) {
            const int64_t r0 = rb + tl * RT;
            // the group's next tile of this item into L2 while this one is computed
            if (t == 0) {
                const int64_t nr0 = r0 + (int64_t)RG * RT;
#pragma unroll
                for (int r = 0; r < RT; ++r)
                    if (nr0 + r < re) split::prefetch_l2(X + (nr0 + r) * ldx + c0, (uint32_t)ncols * 4u);
            }
            float2 x[RT][E2];
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const bool valid = r0 + r < re;
                const float *xr = X + (r0 + r) * ldx + c0;
#pragma unroll
                for (int i = 0; i < NG; ++i) {
                    const int col = (t + G * i) * 4;
                    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (i < act && valid && col < ncols)
                        q = __ldcs(reinterpret_cast<const float4 *>(xr + col));
                    x[r][2 * i] = make_float2(q.x, q.y);
                    x[r][2 * i + 1] = make_float2(q.z, q.w);
                }
            }
            if (MODE != HH_MODE_W && tk.sign) cscale(x, tk.sign + c0, t, act, ncols);
            // W: k = h..1; W^T: k = 1..h; S: k = 1..h, scale by d, k = h..1
            for (int half = 0; half < (MODE == HH_MODE_SYM ? 2 : 1); ++half) {
                if (half == 1) cscale(x, tk.d + c0, t, act, ncols);
                const bool asc = MODE != HH_MODE_W && half == 0;
                split::chain<G, NG, RT, RG, B, CL, true>(x, asc, h, vs, tk.tau, tk.gram, t, lane,
                                                         warp, &rslot[rg][0], &rbar[rg][0], xc,
                                                         err, act);
            }
            if (MODE != HH_MODE_WT && tk.sign) cscale(x, tk.sign + c0, t, act, ncols);
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                if (r0 + r >= re) continue;
                float *yr = Y + (r0 + r) * ldy + c0;
#pragma unroll
                for (int i = 0; i < NG; ++i) {
                    if (i >= act) break;
                    const int col = (t + G * i) * 4;
                    if (col < ncols)
                        __stcs(reinterpret_cast<float4 *>(yr + col),
                               make_float4(x[r][2 * i].x, x[r][2 * i].y, x[r][2 * i + 1].x,
                                           x[r][2 * i + 1].y));
                }
            }
        }
    }
    // a reflector copy that was never seen complete gets one more bounded wait
    if (tid == 0 && issued > confirmed) split::wait_cluster_bounded(&vbar, last_par);
    // no CTA leaves while a peer may still store into its receive slots
    __syncthreads();
    split::cluster_sync();
}

// Fill p[0..count) with values in [-1, 1) from an integer hash of the index
// (synthetic data for the autotuner's timing runs).
__global__ void fill_kernel(float *p, int64_t count, uint32_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + seed;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        p[i] = (float)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
    }
}

// ---- resident CTAs per SM, per device ----
static std::mutex g_attr_mu;
static std::map<int, int> g_per_sm;

static cudaError_t resident_per_sm(int dev, int *per_sm) {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto it = g_per_sm.find(dev);
    if (it != g_per_sm.end()) {
        *per_sm = it->second;
        return cudaSuccess;
    }
    cudaError_t e = cudaFuncSetAttribute(batched_chain_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kStageBytes);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batched_chain_kernel, kThreads,
                                                      kStageBytes);
    if (e != cudaSuccess) return e;
    *per_sm = g_per_sm[dev] = nb > 0 ? nb : 1;
    return cudaSuccess;
}

// ---- resident shape: co-resident clusters per device and cluster size ----
static std::map<std::pair<int, int>, int> g_cluster_slots;

template <int CL>
static cudaError_t cluster_slots_cl(int *ncl) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(cluster_batch_kernel<HH_MODE_W, CL>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kClusterSmem)) ||
        (e = cudaFuncSetAttribute(cluster_batch_kernel<HH_MODE_WT, CL>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kClusterSmem)) ||
        (e = cudaFuncSetAttribute(cluster_batch_kernel<HH_MODE_SYM, CL>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kClusterSmem)))
        return e;
    cudaLaunchConfig_t q = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    q.blockDim = dim3(kThreads);
    q.gridDim = dim3(CL);
    q.dynamicSmemBytes = kClusterSmem;
    q.attrs = attr;
    q.numAttrs = 1;
    int nc = 0;
    e = cudaOccupancyMaxActiveClusters(&nc, cluster_batch_kernel<HH_MODE_SYM, CL>, &q);
    *ncl = nc > 0 ? nc : 1;
    return e;
}

static cudaError_t cluster_slots(int dev, int cl, int *ncl) {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto it = g_cluster_slots.find({dev, cl});
    if (it != g_cluster_slots.end()) {
        *ncl = it->second;
        return cudaSuccess;
    }
    cudaError_t e;
    switch (cl) {
        case 1: e = cluster_slots_cl<1>(ncl); break;
        case 2: e = cluster_slots_cl<2>(ncl); break;
        case 3: e = cluster_slots_cl<3>(ncl); break;
        default: e = cluster_slots_cl<4>(ncl); break;
    }
    if (e == cudaSuccess) g_cluster_slots[{dev, cl}] = *ncl;
    return e;
}

// Relative time of one row on the resident shape: per round of kCB
// reflectors, FMAs over the widest CTA's granules plus the reduction (and the
// exchange between CTAs), and the row's load and store.
static double cluster_row_cost(int n, int h) {
    const int cl = (n + kClusterHalf - 1) / kClusterHalf;
    const int a = cl > 1 ? kCNG : (n + kCG * 4 - 1) / (kCG * 4);
    return (double)((h + kCB - 1) / kCB) * (16.0 * a + (cl > 1 ? 12.0 : 4.0)) + 6.0 * a;
}

// ---- autotuner table: (n, h) -> shape ----
struct TuneEntry {
    int shape = -1;
    float ms[kNumShapes];
};
static std::mutex g_tune_mu;
static std::map<std::pair<int64_t, int64_t>, TuneEntry> g_tune;

static bool shape_fits(int s, int64_t n, int64_t h) {
    return s >= 0 && s < kNumShapes && n <= shape_cover(s) && (s != kClusterShape || h <= kClusterMaxH);
}

// Fixed rule: the smallest cover of n with 128 floats of state per thread
// (64 for n <= 128), two reflectors per round.
static int default_shape(int64_t n) {
    if (n <= 128) return 0;
    if (n <= 256) return 1;
    if (n <= 512) return 2;
    if (n <= 1024) return 3;
    if (n <= 2048) return 6;
    return 8;
}

static int lookup_shape(int64_t n, int64_t h) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find({n, h});
    if (it != g_tune.end() && shape_fits(it->second.shape, n, h)) return it->second.shape;
    // nearest tuned h for the same n (log distance; ties to the smaller h)
    int best = -1;
    double bd = 1e300;
    for (auto &kv : g_tune) {
        if (kv.first.first != n || !shape_fits(kv.second.shape, n, h)) continue;
        const double dist = fabs(log((double)(kv.first.second + 1) / (double)(h + 1)));
        if (dist < bd) {
            bd = dist;
            best = kv.second.shape;
        }
    }
    return best >= 0 ? best : default_shape(n);
}

}  // namespace batched

// One launch of the resident shape: its tasks have (CL-1)*512 < n <= CL*512.
struct CPart {
    int grid = 0, nitems = 0, hmax = 0;  // clusters launched, items, largest h
    batched::CItem *d_items = nullptr;   // items, grouped by cluster in cluster order
    int *d_cstart = nullptr;             // cluster c: items cstart[c] .. cstart[c+1]-1
};

// A batch: the device work list, the task table and one graph per mode.
struct Batch {
    int device = 0, count = 0, grid = 0, nitems = 0;
    std::vector<const Plan *> plans;
    std::vector<int> shapes;
    std::vector<batched::Task> tasks;  // as last uploaded
    bool uploaded = false;
    batched::Task *pinned = nullptr;   // staging for task-table uploads
    cudaEvent_t upload_done = nullptr;
    batched::Task *d_tasks = nullptr;
    batched::Item *d_items = nullptr;
    int *d_counter = nullptr, *d_err = nullptr;
    CPart cpart[batched::kClusterMaxCL];  // resident-shape launches, CL = 1..4
    cudaStream_t capture = nullptr;
#if HH_BATCH_FORK
    // launches of one graph on parallel branches (fork, then one join per launch)
    cudaStream_t side[batched::kClusterMaxCL + 1] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[batched::kClusterMaxCL + 1] = {};
#endif
    cudaGraph_t graph[3] = {nullptr, nullptr, nullptr};
    cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
    // the last launch (its stream and completion event): a launch on another
    // stream waits for it, since both use d_counter and d_tasks
    cudaEvent_t done = nullptr;
    cudaStream_t last_stream = nullptr;
    bool launched = false;
};

static void free_batch(Batch *b) {
    if (!b) return;
    for (int m = 0; m < 3; ++m) {
        if (b->exec[m]) cudaGraphExecDestroy(b->exec[m]);
        if (b->graph[m]) cudaGraphDestroy(b->graph[m]);
    }
    if (b->capture) cudaStreamDestroy(b->capture);
#if HH_BATCH_FORK
    for (int j = 0; j <= batched::kClusterMaxCL; ++j) {
        if (b->side[j]) cudaStreamDestroy(b->side[j]);
        if (b->join_ev[j]) cudaEventDestroy(b->join_ev[j]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
#endif
    for (auto &cp : b->cpart) {
        cudaFree(cp.d_items);
        cudaFree(cp.d_cstart);
    }
    if (b->upload_done) cudaEventDestroy(b->upload_done);
    if (b->done) cudaEventDestroy(b->done);
    cudaFreeHost(b->pinned);
    cudaFree(b->d_tasks);
    cudaFree(b->d_items);
    cudaFree(b->d_counter);
    cudaFree(b->d_err);
    delete b;
}

// Build a batch over the plans with the given rows per task; shapes[i] >= 0
// forces a shape (the autotuner), else the tuned table decides.
static hh_status batch_create(Batch **out, int count, const hh_plan_t *plans, const int64_t *rows,
                              const int *force_shape) {
    using namespace batched;
    *out = nullptr;
    if (count < 0) return fail(HH_ERR_INVALID_ARG, "count %d < 0", count);
    if (count > 0 && (!plans || !rows)) return fail(HH_ERR_INVALID_ARG, "plans or batch is NULL");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    Batch *b = new (std::nothrow) Batch;
    if (!b) return fail(HH_ERR_OOM, "host allocation");
    b->device = dev;
    b->count = count;
    b->plans.resize(count);
    b->shapes.resize(count);
    b->tasks.resize(count);
    // per-tile cost in units proportional to time: 4nh flops plus the 8n bytes of
    // the row at the FP32 ridge (~12 flop per byte)
    std::vector<double> tile_cost(count);
    double total = 0;
    for (int i = 0; i < count; ++i) {
        const Plan *p = reinterpret_cast<const Plan *>(plans[i]);
        hh_status st = check_plan(p);
        if (st) {
            free_batch(b);
            return fail(st, "plan %d: %s", i, hh_last_error());
        }
        if (p->path != HH_PATH_FUSED || p->dtype != HH_F32) {
            free_batch(b);
            return fail(HH_ERR_UNSUPPORTED, "plan %d: the batched launch takes F32 plans only", i);
        }
        if (p->n % 4 != 0 || p->n > kMaxN) {
            free_batch(b);
            return fail(HH_ERR_UNSUPPORTED, "plan %d: n = %lld (needs n %% 4 == 0, n <= %d)", i,
                        (long long)p->n, kMaxN);
        }
        if (rows[i] < 0) {
            free_batch(b);
            return fail(HH_ERR_INVALID_ARG, "batch[%d] = %lld < 0", i, (long long)rows[i]);
        }
        int s = force_shape ? force_shape[i] : -1;
        if (s < 0) s = lookup_shape(p->n, p->h);
        if (!shape_fits(s, p->n, p->h)) {
            free_batch(b);
            return fail(HH_ERR_INVALID_ARG, "plan %d: shape %d does not cover n = %lld, h = %lld",
                        i, s, (long long)p->n, (long long)p->h);
        }
        b->plans[i] = p;
        b->shapes[i] = s;
        Task &t = b->tasks[i];
        t = Task{};
        t.ldx = t.ldy = p->n;
        t.rows = rows[i];
        t.V = (const float *)p->u;
        t.tau = (const float *)p->tau_t;
        t.gram = (const float *)p->gram;
        t.sign = (const float *)p->sign;
        t.d = (const float *)p->d;
        t.ldv = p->ldv;
        t.n = (int)p->n;
        t.h = (int)p->h;
        t.shape = s;
        t.rows_per_tile = shape_rows(s);
        tile_cost[i] = (double)shape_rows(s) * (4.0 * p->n * (double)p->h + 96.0 * p->n);
        const int64_t tiles = (rows[i] + t.rows_per_tile - 1) / t.rows_per_tile;
        if (s != kClusterShape) total += tile_cost[i] * (double)tiles;
    }
    int per_sm = 1, sms = 1;
    if ((e = resident_per_sm(dev, &per_sm)) ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) {
        free_batch(b);
        return cuda_fail(e, "batched kernel attributes");
    }
    const int slots = sms * per_sm;
    // items of about total / (24 * slots) each, at least one tile
    const double target = total / (24.0 * slots);
    std::vector<Item> items;
    std::vector<double> icost;
    for (int i = 0; i < count; ++i) {
        const Task &t = b->tasks[i];
        if (t.shape == kClusterShape) continue;  // scheduled below
        const int64_t tiles = (t.rows + t.rows_per_tile - 1) / t.rows_per_tile;
        int64_t per = (int64_t)(target / tile_cost[i]);
        if (per < 1) per = 1;
        if (per > (1 << 20)) per = 1 << 20;
        for (int64_t t0 = 0; t0 < tiles; t0 += per) {
            const int64_t k = std::min(per, tiles - t0);
            items.push_back(Item{t0, i, (int)k});
            icost.push_back(tile_cost[i] * (double)k);
        }
    }
    if (items.size() > 0x7fffffff) {
        free_batch(b);
        return fail(HH_ERR_UNSUPPORTED, "work list of %zu items", items.size());
    }
    std::vector<int> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return icost[a] > icost[c]; });
    std::vector<Item> sorted(items.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
    b->nitems = (int)sorted.size();
    b->grid = b->nitems < slots ? b->nitems : slots;

    const size_t tbytes = sizeof(Task) * (size_t)(count > 0 ? count : 1);
    const size_t ibytes = sizeof(Item) * (size_t)(b->nitems > 0 ? b->nitems : 1);
    if ((e = dev_malloc(&b->d_tasks, tbytes)) || (e = dev_malloc(&b->d_items, ibytes)) ||
        (e = dev_malloc(&b->d_counter, sizeof(int))) || (e = dev_malloc(&b->d_err, sizeof(int))) ||
        (e = cudaMallocHost(&b->pinned, tbytes)) ||
        (e = cudaEventCreateWithFlags(&b->upload_done, cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) ||
        (e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking)) ||
        (e = cudaMemset(b->d_err, 0, sizeof(int))) ||
        (b->nitems > 0 && (e = cudaMemcpy(b->d_items, sorted.data(), sizeof(Item) * sorted.size(),
                                          cudaMemcpyHostToDevice)))) {
        free_batch(b);
        return cuda_fail(e, "batch allocation");
    }
#if HH_BATCH_FORK
    if ((e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming))) {
        free_batch(b);
        return cuda_fail(e, "batch allocation");
    }
    for (int j = 0; j <= kClusterMaxCL; ++j)
        if ((e = cudaStreamCreateWithFlags(&b->side[j], cudaStreamNonBlocking)) ||
            (e = cudaEventCreateWithFlags(&b->join_ev[j], cudaEventDisableTiming))) {
            free_batch(b);
            return cuda_fail(e, "batch allocation");
        }
#endif
    // Resident-shape tasks: one launch per cluster size CL, each with a static
    // schedule.  The tasks' rows, in task order, are cut into runs of
    // kClusterUnit rows; a run goes to the cluster whose share of the launch's
    // total cost (cluster_row_cost per row) holds the run's midpoint, so each
    // cluster gets a contiguous stretch of the task list and loads each of its
    // tasks' reflectors once.
    for (int cl = 1; cl <= kClusterMaxCL; ++cl) {
        std::vector<int> ids;
        double wsum = 0;
        int64_t units = 0;
        int hmax = 0;
        for (int i = 0; i < count; ++i) {
            const Task &t = b->tasks[i];
            if (t.shape != kClusterShape || t.rows == 0) continue;
            if ((t.n + kClusterHalf - 1) / kClusterHalf != cl) continue;
            ids.push_back(i);
            wsum += cluster_row_cost(t.n, t.h) * (double)t.rows;
            units += (t.rows + kClusterUnit - 1) / kClusterUnit;
            hmax = std::max(hmax, t.h);
        }
        if (ids.empty()) continue;
        int ncl = 1;
        if ((e = cluster_slots(dev, cl, &ncl))) {
            free_batch(b);
            return cuda_fail(e, "resident-shape attributes");
        }
        const int grid = (int)std::min<int64_t>(ncl, units);
        const double share = wsum / grid;
        std::vector<CItem> its;
        std::vector<int> owner;
        double cum = 0;
        for (int i : ids) {
            const Task &t = b->tasks[i];
            const double uc = cluster_row_cost(t.n, t.h);
            for (int64_t r = 0; r < t.rows; r += kClusterUnit) {
                const int64_t r1 = std::min<int64_t>(t.rows, r + kClusterUnit);
                const double mid = cum + 0.5 * uc * (double)(r1 - r);
                const int k = std::min(grid - 1, (int)(mid / share));
                if (!its.empty() && its.back().task == i && owner.back() == k)
                    its.back().r1 = r1;
                else {
                    its.push_back(CItem{i, 0, r, r1});
                    owner.push_back(k);
                }
                cum += uc * (double)(r1 - r);
            }
        }
        // owner is non-decreasing: the items are already grouped by cluster
        std::vector<int> cstart(grid + 1, 0);
        for (int k : owner) ++cstart[k + 1];
        for (int k = 0; k < grid; ++k) cstart[k + 1] += cstart[k];
        CPart &cp = b->cpart[cl - 1];
        cp.grid = grid;
        cp.nitems = (int)its.size();
        cp.hmax = hmax;
        if ((e = dev_malloc(&cp.d_items, sizeof(CItem) * its.size())) ||
            (e = dev_malloc(&cp.d_cstart, sizeof(int) * cstart.size())) ||
            (e = cudaMemcpy(cp.d_items, its.data(), sizeof(CItem) * its.size(),
                            cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(cp.d_cstart, cstart.data(), sizeof(int) * cstart.size(),
                            cudaMemcpyHostToDevice))) {
            free_batch(b);
            return cuda_fail(e, "batch allocation");
        }
    }
    *out = b;
    return HH_OK;
}

// Items of every launch of the batch.
static int64_t batch_items(const Batch *b) {
    int64_t n = b->nitems;
    for (const CPart &cp : b->cpart) n += cp.nitems;
    return n;
}

// One resident-shape launch of CL-CTA clusters on stream s.
template <int CL>
static cudaError_t launch_cluster(const Batch *b, const CPart &cp, int mode, cudaStream_t s) {
    using namespace batched;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kThreads);
    cfg.gridDim = dim3(CL * cp.grid);
    cfg.dynamicSmemBytes = cp.hmax > 0 ? (size_t)cp.hmax * kClusterHalf * 4 : 16;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const Task *tasks = b->d_tasks;
    const CItem *items = cp.d_items;
    const int *cstart = cp.d_cstart;
    switch (mode) {
        case HH_MODE_W:
            return cudaLaunchKernelEx(&cfg, cluster_batch_kernel<HH_MODE_W, CL>, tasks, items,
                                      cstart, b->d_err);
        case HH_MODE_WT:
            return cudaLaunchKernelEx(&cfg, cluster_batch_kernel<HH_MODE_WT, CL>, tasks, items,
                                      cstart, b->d_err);
        default:
            return cudaLaunchKernelEx(&cfg, cluster_batch_kernel<HH_MODE_SYM, CL>, tasks, items,
                                      cstart, b->d_err);
    }
}

// Launch j of the batch (0..kClusterMaxCL-1: the resident shape with
// CL = kClusterMaxCL - j; kClusterMaxCL: the staged shapes) on stream s, if
// it has work.
static cudaError_t launch_part(const Batch *b, int j, int mode, cudaStream_t s) {
    using namespace batched;
    if (j == kClusterMaxCL) {
        if (b->nitems == 0) return cudaSuccess;
        cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
        batched_chain_kernel<<<b->grid, kThreads, kStageBytes, s>>>(b->d_tasks, b->d_items,
                                                                    b->nitems, b->d_counter, mode,
                                                                    b->d_err);
        return cudaGetLastError();
    }
    const int cl = kClusterMaxCL - j;
    const CPart &cp = b->cpart[cl - 1];
    if (cp.nitems == 0) return cudaSuccess;
    switch (cl) {
        case 1: return launch_cluster<1>(b, cp, mode, s);
        case 2: return launch_cluster<2>(b, cp, mode, s);
        case 3: return launch_cluster<3>(b, cp, mode, s);
        default: return launch_cluster<4>(b, cp, mode, s);
    }
}

static hh_status batch_graph(Batch *b, int mode) {
    if (b->exec[mode]) return HH_OK;
    cudaError_t e;
    if ((e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal)))
        return cuda_fail(e, "cudaStreamBeginCapture");
    // the launches in order: resident shape with four, three, two and one CTAs
    // per cluster, then the staged shapes
    cudaError_t le = cudaSuccess;
#if HH_BATCH_FORK
    // on parallel branches of the graph, so that one launch's last CTAs share
    // the GPU with the next launch's first
    le = cudaEventRecord(b->fork_ev, b->capture);
    for (int j = 0; j <= batched::kClusterMaxCL && le == cudaSuccess; ++j) {
        if ((le = cudaStreamWaitEvent(b->side[j], b->fork_ev, 0)) ||
            (le = launch_part(b, j, mode, b->side[j])) ||
            (le = cudaEventRecord(b->join_ev[j], b->side[j])))
            break;
        le = cudaStreamWaitEvent(b->capture, b->join_ev[j], 0);
    }
#else
    for (int j = 0; j <= batched::kClusterMaxCL && le == cudaSuccess; ++j)
        le = launch_part(b, j, mode, b->capture);
#endif
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->capture, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(le != cudaSuccess ? le : e, "batched graph capture");
    }
    cudaGraphExec_t x = nullptr;
    if ((e = cudaGraphInstantiate(&x, g, 0))) {
        cudaGraphDestroy(g);
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    b->graph[mode] = g;
    b->exec[mode] = x;
    return HH_OK;
}

static hh_status batch_apply(Batch *b, int mode, const void *const *X, const int64_t *ldx,
                             void *const *Y, const int64_t *ldy, cudaStream_t s) {
    using batched::Task;
    if (!b) return fail(HH_ERR_INVALID_ARG, "batch is NULL");
    if (mode != HH_MODE_W && mode != HH_MODE_WT && mode != HH_MODE_SYM)
        return fail(HH_ERR_INVALID_ARG, "unknown mode %d", mode);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != b->device)
        return fail(HH_ERR_INVALID_ARG, "batch was created on device %d, current device is %d",
                    b->device, dev);
    if (b->count > 0 && (!X || !Y)) return fail(HH_ERR_INVALID_ARG, "X or Y array is NULL");
    bool changed = !b->uploaded;
    std::vector<Task> next = b->tasks;
    for (int i = 0; i < b->count; ++i) {
        Task &t = next[i];
        if (t.rows == 0) continue;
        if (mode == HH_MODE_SYM && !t.d)
            return fail(HH_ERR_INVALID_ARG, "task %d: apply_sym needs a plan with spectrum d", i);
        const int64_t lx = ldx ? ldx[i] : t.n, ly = ldy ? ldy[i] : t.n;
        if (lx < t.n || ly < t.n || lx % 4 || ly % 4)
            return fail(HH_ERR_INVALID_ARG,
                        "task %d: leading dimensions %lld, %lld (need >= n and a multiple of 4)", i,
                        (long long)lx, (long long)ly);
        if ((uintptr_t)X[i] % 16 || (uintptr_t)Y[i] % 16)
            return fail(HH_ERR_INVALID_ARG, "task %d: X and Y must be 16-byte aligned", i);
        if (X[i] == Y[i] && lx != ly)
            return fail(HH_ERR_INVALID_ARG, "task %d: in-place apply needs ldx == ldy", i);
        if (X[i] != t.X || Y[i] != t.Y) {
            if (!device_ptr(X[i], b->device) || !device_ptr(Y[i], b->device))
                return fail(HH_ERR_INVALID_ARG, "task %d: X or Y is not a device pointer of device %d",
                            i, b->device);
        }
        if (X[i] != t.X || Y[i] != t.Y || lx != t.ldx || ly != t.ldy) changed = true;
        t.X = (const float *)X[i];
        t.Y = (float *)Y[i];
        t.ldx = lx;
        t.ldy = ly;
    }
    if (batch_items(b) == 0) return HH_OK;  // nothing to launch
    hh_status st = batch_graph(b, mode);
    if (st) return st;
    // the previous launch on another stream still owns the counter and the table
    if (b->launched && b->last_stream != s && (e = cudaStreamWaitEvent(s, b->done, 0)))
        return cuda_fail(e, "cross-stream ordering");
    if (changed) {
        // the staging buffer may still feed the previous upload
        if ((e = cudaEventSynchronize(b->upload_done))) return cuda_fail(e, "upload wait");
        memcpy(b->pinned, next.data(), sizeof(Task) * (size_t)b->count);
        if ((e = cudaMemcpyAsync(b->d_tasks, b->pinned, sizeof(Task) * (size_t)b->count,
                                 cudaMemcpyHostToDevice, s)) ||
            (e = cudaEventRecord(b->upload_done, s)))
            return cuda_fail(e, "task table upload");
        b->tasks = next;
        b->uploaded = true;
    }
    if ((e = cudaGraphLaunch(b->exec[mode], s))) return cuda_fail(e, "cudaGraphLaunch");
    if ((e = cudaEventRecord(b->done, s))) return cuda_fail(e, "launch event");
    b->last_stream = s;
    b->launched = true;
    return HH_OK;
}

}  // namespace hh

using namespace hh;

extern "C" {

hh_status hh_batch_create(hh_batch_t *out, int count, const hh_plan_t *plans,
                          const int64_t *batch) {
    if (!out) return fail(HH_ERR_INVALID_ARG, "out is NULL");
    Batch *b = nullptr;
    hh_status st = batch_create(&b, count, plans, batch, nullptr);
    if (st) return st;
    *out = reinterpret_cast<hh_batch_t>(b);
    return HH_OK;
}

hh_status hh_batch_apply(hh_batch_t batch, hh_mode mode, const void *const *X, const int64_t *ldx,
                         void *const *Y, const int64_t *ldy, void *stream) {
    TraceRange trace("hh_batch_apply");
    return batch_apply(reinterpret_cast<Batch *>(batch), (int)mode, X, ldx, Y, ldy,
                       reinterpret_cast<cudaStream_t>(stream));
}

hh_status hh_batch_sync(hh_batch_t batch, void *stream) {
    Batch *b = reinterpret_cast<Batch *>(batch);
    if (!b) return fail(HH_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int word = 0;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(&word, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemsetAsync(b->d_err, 0, sizeof(int), s)) || (e = cudaStreamSynchronize(s)))
        return cuda_fail(e, "hh_batch_sync");
    if (word == HH_ERR_TIMEOUT)
        return fail(HH_ERR_TIMEOUT, "a kernel's bounded wait on its bulk copy expired");
    if (word != 0) return fail(HH_ERR_CUDA, "device status word %d", word);
    return HH_OK;
}

hh_status hh_batch_info(hh_batch_t batch, int64_t *nitems, int *grid, int *shapes) {
    const Batch *b = reinterpret_cast<const Batch *>(batch);
    if (!b) return fail(HH_ERR_INVALID_ARG, "batch is NULL");
    if (nitems) *nitems = batch_items(b);
    if (grid) {
        // CTAs of the largest launch
        int g = b->grid;
        for (int cl = 1; cl <= batched::kClusterMaxCL; ++cl)
            g = std::max(g, cl * b->cpart[cl - 1].grid);
        *grid = g;
    }
    if (shapes)
        for (int i = 0; i < b->count; ++i) shapes[i] = b->shapes[i];
    return HH_OK;
}

hh_status hh_batch_destroy(hh_batch_t batch) {
    Batch *b = reinterpret_cast<Batch *>(batch);
    if (!b) return HH_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != b->device) cudaSetDevice(b->device);
    cudaError_t e = cudaDeviceSynchronize();
    free_batch(b);
    if (cur != b->device) cudaSetDevice(cur);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize (batch destroy)");
    return HH_OK;
}

hh_status hh_batch_shape(int shape, int *G, int *NG, int *RT, int *rows_per_tile, int *cover) {
    using namespace batched;
    if (shape < 0 || shape >= kNumShapes)
        return fail(HH_ERR_INVALID_ARG, "shape %d outside [0, %d)", shape, kNumShapes);
    if (G) *G = kShape[shape].G;
    if (NG) *NG = kShape[shape].NG;
    if (RT) *RT = kShape[shape].RT;
    if (rows_per_tile) *rows_per_tile = shape_rows(shape);
    if (cover) *cover = shape_cover(shape);
    return HH_OK;
}

int hh_batch_num_shapes(void) { return batched::kNumShapes; }

hh_status hh_batch_shape_limits(int shape, int *max_h, int *max_cluster) {
    using namespace batched;
    if (shape < 0 || shape >= kNumShapes)
        return fail(HH_ERR_INVALID_ARG, "shape %d outside [0, %d)", shape, kNumShapes);
    const bool res = shape == kClusterShape;
    if (max_h) *max_h = res ? kClusterMaxH : -1;
    if (max_cluster) *max_cluster = res ? kClusterMaxCL : 0;
    return HH_OK;
}

hh_status hh_tune_set(int64_t n, int64_t h, int shape) {
    using namespace batched;
    if (n < 1 || h < 0) return fail(HH_ERR_INVALID_ARG, "n = %lld, h = %lld", (long long)n, (long long)h);
    if (!shape_fits(shape, n, h))
        return fail(HH_ERR_INVALID_ARG, "shape %d does not cover n = %lld, h = %lld", shape,
                    (long long)n, (long long)h);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneEntry &t = g_tune[{n, h}];
    t.shape = shape;
    for (int s = 0; s < kNumShapes; ++s) t.ms[s] = NAN;
    return HH_OK;
}

hh_status hh_tune_get(int64_t n, int64_t h, int *shape, float *ms) {
    using namespace batched;
    if (n < 1 || h < 0) return fail(HH_ERR_INVALID_ARG, "n = %lld, h = %lld", (long long)n, (long long)h);
    if (shape) *shape = lookup_shape(n, h);
    if (ms) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find({n, h});
        for (int s = 0; s < kNumShapes; ++s) ms[s] = it != g_tune.end() ? it->second.ms[s] : NAN;
    }
    return HH_OK;
}

hh_status hh_tune_clear(void) {
    std::lock_guard<std::mutex> lk(batched::g_tune_mu);
    batched::g_tune.clear();
    return HH_OK;
}

hh_status hh_tune_save(const char *path) {
    if (!path) return fail(HH_ERR_INVALID_ARG, "path is NULL");
    FILE *f = fopen(path, "w");
    if (!f) return fail(HH_ERR_INVALID_ARG, "cannot open %s for writing", path);
    fprintf(f, "# libhh batched tile shapes: n h shape\n");
    {
        std::lock_guard<std::mutex> lk(batched::g_tune_mu);
        for (auto &kv : batched::g_tune)
            fprintf(f, "%lld %lld %d\n", (long long)kv.first.first, (long long)kv.first.second,
                    kv.second.shape);
    }
    const bool ok = fclose(f) == 0;
    return ok ? HH_OK : fail(HH_ERR_INVALID_ARG, "write error on %s", path);
}

hh_status hh_tune_load(const char *path) {
    if (!path) return fail(HH_ERR_INVALID_ARG, "path is NULL");
    FILE *f = fopen(path, "r");
    if (!f) return fail(HH_ERR_INVALID_ARG, "cannot open %s", path);
    char line[256];
    int lineno = 0;
    std::vector<std::pair<std::pair<int64_t, int64_t>, int>> rows;
    while (fgets(line, sizeof line, f)) {
        ++lineno;
        const char *c = line;
        while (*c == ' ' || *c == '\t') ++c;
        if (*c == '#' || *c == '\n' || *c == '\0') continue;
        long long n = 0, h = 0;
        int s = -1;
        char extra = 0;
        if (sscanf(c, "%lld %lld %d %c", &n, &h, &s, &extra) != 3 || n < 1 || h < 0 ||
            !batched::shape_fits(s, n, h)) {
            fclose(f);
            return fail(HH_ERR_INVALID_ARG, "%s:%d: expected 'n h shape' with a shape covering n",
                        path, lineno);
        }
        rows.push_back({{n, h}, s});
    }
    fclose(f);
    for (auto &r : rows) hh_tune_set(r.first.first, r.first.second, r.second);
    return HH_OK;
}

hh_status hh_tune(const int64_t *ns, int nn, const int64_t *hs, int nh, int64_t rows,
                  void *stream) {
    TraceRange trace("hh_tune");
    using namespace batched;
    if (nn < 0 || nh < 0 || (nn > 0 && !ns) || (nh > 0 && !hs))
        return fail(HH_ERR_INVALID_ARG, "ns/hs arrays");
    if (rows < 1) return fail(HH_ERR_INVALID_ARG, "rows = %lld < 1", (long long)rows);
    for (int i = 0; i < nn; ++i)
        if (ns[i] < 4 || ns[i] % 4 || ns[i] > kMaxN)
            return fail(HH_ERR_INVALID_ARG, "n = %lld (needs n %% 4 == 0, 4 <= n <= %d)",
                        (long long)ns[i], kMaxN);
    for (int j = 0; j < nh; ++j)
        if (hs[j] < 0 || hs[j] > 65536) return fail(HH_ERR_INVALID_ARG, "h = %lld", (long long)hs[j]);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int64_t nmax = 0, hmax = 0;
    for (int i = 0; i < nn; ++i) nmax = std::max(nmax, ns[i]);
    for (int j = 0; j < nh; ++j) hmax = std::max(hmax, hs[j]);
    if (nn == 0 || nh == 0) return HH_OK;
    float *U = nullptr, *X = nullptr, *Y = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    hh_status st = HH_OK;
    const size_t vbytes = sizeof(float) * (size_t)std::max<int64_t>(hmax, 1) * nmax;
    const size_t xbytes = sizeof(float) * (size_t)rows * nmax;
    if ((e = dev_malloc(&U, vbytes)) || (e = dev_malloc(&X, xbytes)) || (e = dev_malloc(&Y, xbytes)) ||
        (e = cudaEventCreate(&e0)) || (e = cudaEventCreate(&e1))) {
        st = cuda_fail(e, "tune allocation");
        goto done;
    }
    fill_kernel<<<1024, 256, 0, s>>>(U, (int64_t)(vbytes / 4), 17u);
    fill_kernel<<<1024, 256, 0, s>>>(X, (int64_t)(xbytes / 4), 29u);
    if ((e = cudaGetLastError())) {
        st = cuda_fail(e, "tune fill");
        goto done;
    }
    for (int i = 0; i < nn && !st; ++i) {
        for (int j = 0; j < nh && !st; ++j) {
            const int64_t n = ns[i], h = hs[j];
            hh_plan_t plan = nullptr;
            st = hh_create_ex(&plan, n, h, U, n, nullptr, nullptr, HH_F32, HH_PATH_FUSED, stream);
            if (st) break;
            TuneEntry ent;
            float best = INFINITY;
            for (int sh = 0; sh < kNumShapes && !st; ++sh) {
                ent.ms[sh] = NAN;
                if (!shape_fits(sh, n, h)) continue;
                Batch *b = nullptr;
                st = batch_create(&b, 1, &plan, &rows, &sh);
                if (st) break;
                const void *xp = X;
                void *yp = Y;
                for (int w = 0; w < 2 && !st; ++w)
                    st = batch_apply(b, HH_MODE_W, &xp, nullptr, &yp, nullptr, s);
                const int reps = 5;
                if (!st && (e = cudaEventRecord(e0, s))) st = cuda_fail(e, "event");
                for (int r = 0; r < reps && !st; ++r)
                    st = batch_apply(b, HH_MODE_W, &xp, nullptr, &yp, nullptr, s);
                float ms = 0;
                if (!st && ((e = cudaEventRecord(e1, s)) || (e = cudaEventSynchronize(e1)) ||
                            (e = cudaEventElapsedTime(&ms, e0, e1))))
                    st = cuda_fail(e, "tune timing");
                if (!st) {
                    hh_status bs = hh_batch_sync(reinterpret_cast<hh_batch_t>(b), stream);
                    if (bs) st = bs;
                }
                cudaStreamSynchronize(s);
                free_batch(b);
                if (st) break;
                ent.ms[sh] = ms / reps;
                if (ent.ms[sh] < best) {
                    best = ent.ms[sh];
                    ent.shape = sh;
                }
            }
            cudaStreamSynchronize(s);
            hh_destroy(plan);
            if (!st) {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_tune[{n, h}] = ent;
            }
        }
    }
done:
    cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(U);
    cudaFree(X);
    cudaFree(Y);
    return st;
}

}  // extern "C"
