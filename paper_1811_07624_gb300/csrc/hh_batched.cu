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

#include "hh_staged.cuh"

namespace hh {
namespace batched {

constexpr int kThreads = 256;
constexpr int kNumShapes = 10;
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
};
inline int shape_cover(int s) { return kShape[s].G * kShape[s].NG * 4; }
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

// ---- autotuner table: (n, h) -> shape ----
struct TuneEntry {
    int shape = -1;
    float ms[kNumShapes];
};
static std::mutex g_tune_mu;
static std::map<std::pair<int64_t, int64_t>, TuneEntry> g_tune;

static bool shape_fits(int s, int64_t n) { return s >= 0 && s < kNumShapes && n <= shape_cover(s); }

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
    if (it != g_tune.end() && shape_fits(it->second.shape, n)) return it->second.shape;
    // nearest tuned h for the same n (log distance; ties to the smaller h)
    int best = -1;
    double bd = 1e300;
    for (auto &kv : g_tune) {
        if (kv.first.first != n || !shape_fits(kv.second.shape, n)) continue;
        const double dist = fabs(log((double)(kv.first.second + 1) / (double)(h + 1)));
        if (dist < bd) {
            bd = dist;
            best = kv.second.shape;
        }
    }
    return best >= 0 ? best : default_shape(n);
}

}  // namespace batched

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
    cudaStream_t capture = nullptr;
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
        if (!shape_fits(s, p->n)) {
            free_batch(b);
            return fail(HH_ERR_INVALID_ARG, "plan %d: shape %d does not cover n = %lld", i, s,
                        (long long)p->n);
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
        total += tile_cost[i] * (double)tiles;
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
    *out = b;
    return HH_OK;
}

static hh_status batch_graph(Batch *b, int mode) {
    if (b->exec[mode]) return HH_OK;
    cudaError_t e;
    if ((e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal)))
        return cuda_fail(e, "cudaStreamBeginCapture");
    cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->capture);
    batched::batched_chain_kernel<<<b->grid, batched::kThreads, batched::kStageBytes, b->capture>>>(
        b->d_tasks, b->d_items, b->nitems, b->d_counter, mode, b->d_err);
    cudaError_t le = cudaGetLastError();
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
    if (b->nitems == 0) return HH_OK;  // nothing to launch
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
    if (nitems) *nitems = b->nitems;
    if (grid) *grid = b->grid;
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

hh_status hh_tune_set(int64_t n, int64_t h, int shape) {
    using namespace batched;
    if (n < 1 || h < 0) return fail(HH_ERR_INVALID_ARG, "n = %lld, h = %lld", (long long)n, (long long)h);
    if (!shape_fits(shape, n))
        return fail(HH_ERR_INVALID_ARG, "shape %d does not cover n = %lld", shape, (long long)n);
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
            !batched::shape_fits(s, n)) {
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
                if (!shape_fits(sh, n)) continue;
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
