// Compact-WY apply on the tensor cores (BF16 storage, FP32 accumulation).
//
// A product of reflectors is I minus a low-rank term: for H_1 ... H_m with
// H_k = I - tau_k v_k v_k^T (§II-A, Eq. (2)),
//     H_1 ... H_m = I - V T V^T,   V = [v_1 .. v_m],
// with T upper triangular, T_kk = tau_k, T[0:k, k] = -tau_k T[0:k, 0:k] V[:, 0:k]^T v_k
// (the forward accumulation of Schreiber and Van Loan).  For vectors stored as
// rows, Y = X W^T = X - (X V) T^T V^T = X - (X V) (V T)^T, i.e. two GEMMs:
//     Z = X V          (M = rows, N = m, K = n)
//     Y = X - Z V'^T   (M = rows, N = n, K = m),  V' = V T   (W^T: V' = V T^T).
// The paper's 4nm operations per vector (§II-A) are exactly these two GEMMs.
//
// The chain is cut into panels of at most 256 reflectors (a panel's Z fits in
// tensor memory); W = W_1 ... W_P is applied panel by panel (W: P first), each
// panel one pass over the vectors.  T and V' are computed in FP64 on the GPU
// when the plan is created, from the BF16 reflectors as stored, and V' is
// rounded to BF16 once; tau is FP64 (the normalisation the transform's
// orthogonality rests on).  The sign D of Eq. (1) is applied in the last
// panel's epilogue (W) or folded into the first panel's V and epilogue (W^T).
//
// Kernel: persistent, one CTA per SM over 128-row tiles, warp-specialised (a
// TMA warp, an MMA warp, four epilogue warps), operands in a ring of TMA
// stages (128-byte swizzle), GEMM 2 in 64-column chunks over four tensor-memory
// accumulators so the epilogue of one chunk overlaps the MMAs of the next and
// GEMM 1 of the next tile; details at wy_panel_kernel.  All mbarrier waits are
// bounded.
#include <algorithm>
#include <cstring>
#include <new>

#include "hh_tc.cuh"

namespace hh {

struct WYPlan {
    int PB = 0, P = 0;       // reflectors per panel (multiple of 64, <= 256), panels
    int64_t hpad = 0;        // P * PB
    int64_t n8 = 0;          // row stride of the BF16 reflector copies (n rounded up to 8)
    __nv_bfloat16 *Vb = nullptr;    // hpad x n8, v_k as given (zero rows past h)
    __nv_bfloat16 *Vs = nullptr;    // sign-scaled copy (W^T, first panel), or null
    __nv_bfloat16 *Vp = nullptr;    // P x n x PB: V_p T_p^T (operand of W^T)
    __nv_bfloat16 *Vpp = nullptr;   // P x n x PB: V_p T_p   (operand of W)
    float *sign = nullptr;          // n, or null
    double *V64 = nullptr, *G = nullptr, *T = nullptr;  // create-time work arrays
    CUtensorMap mapV, mapVs, mapVp, mapVpp;  // tensor maps of Vb, Vs, Vp, Vpp
};

namespace wy {

constexpr int kTileM = 128;     // rows per tile (M of both GEMMs)
constexpr int kChunkN = 64;     // output columns per GEMM 2 accumulator
constexpr int kNumAcc = 2;      // GEMM 2 accumulators, tensor-memory columns 384 + 64a
// Tensor-memory columns: Z (FP32, GEMM 1's accumulator) [0, 256), Z as BF16
// (GEMM 2's A operand, two per column) [256, 384), accumulators [384, 512).
constexpr uint32_t kTmemZb = 256, kTmemAcc = 384;
constexpr int kThreads = 224;   // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue, warp 6 TMA
constexpr int kMaxStages = 8;
constexpr uint32_t kEBox = kTileM * kChunkN * 2;  // epilogue box, 128 x 64 BF16 = 16 KB
// Dynamic shared memory: 1 KB alignment slack, the epilogue ring and the
// operand ring; their stage counts are set per plan by the host.
constexpr size_t kSmemBytes = 220 * 1024;

// ---- create-time kernels (FP64) ---------------------------------------------------------

// V64 (hpad x n) and the BF16 copies; tau_k (0 for v_k = 0 and past h); flag bit 0
// for a non-finite entry.
__global__ void __launch_bounds__(256)
wy_convert_kernel(const __nv_bfloat16 *__restrict__ U, int64_t ldu, int64_t n, int64_t h,
                  int64_t n8, const int8_t *__restrict__ sign, double *__restrict__ V64,
                  __nv_bfloat16 *__restrict__ Vb, __nv_bfloat16 *__restrict__ Vs,
                  double *__restrict__ tau, double *__restrict__ vnorm, int *__restrict__ flag) {
    __shared__ double red[256];
    const int64_t k = blockIdx.x;
    double s = 0.0;
    bool finite = true;
    for (int64_t j = threadIdx.x; j < n8; j += 256) {
        double x = 0.0;
        __nv_bfloat16 b = __float2bfloat16(0.f);
        if (k < h && j < n) {
            b = U[k * ldu + j];
            x = (double)__bfloat162float(b);
            finite &= isfinite(x);
            s += x * x;
        }
        if (j < n) V64[k * n + j] = x;
        Vb[k * n8 + j] = b;
        if (Vs) {
            const float sg = (j < n && sign[j] < 0) ? -1.f : 1.f;
            Vs[k * n8 + j] = __float2bfloat16(sg * __bfloat162float(b));
        }
    }
    if (!finite) atomicOr(flag, 1);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        tau[k] = red[0] > 0.0 ? 2.0 / red[0] : 0.0;
        vnorm[k] = sqrt(red[0]);
    }
}

// Gram matrix of each panel: G[p][i][j] = v_{p PB + i} . v_{p PB + j}.
__global__ void __launch_bounds__(128)
wy_gram_kernel(const double *__restrict__ V64, int64_t n, int PB, double *__restrict__ G) {
    __shared__ double red[128];
    const int i = blockIdx.x, j = blockIdx.y, p = blockIdx.z;
    if (j < i) return;
    const double *a = V64 + ((int64_t)p * PB + i) * n, *b = V64 + ((int64_t)p * PB + j) * n;
    double s = 0.0;
    for (int64_t c = threadIdx.x; c < n; c += 128) s += a[c] * b[c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double *g = G + (int64_t)p * PB * PB;
        g[(int64_t)i * PB + j] = red[0];
        g[(int64_t)j * PB + i] = red[0];
    }
}

// T of each panel; thread i computes row i:
//   T[i][i] = tau_i,  T[i][k] = -tau_k sum_{j=i}^{k-1} T[i][j] G[j][k]  (k > i).
__global__ void wy_tfactor_kernel(const double *__restrict__ G, const double *__restrict__ tau,
                                  int PB, double *__restrict__ T) {
    const int p = blockIdx.x, i = threadIdx.x;
    if (i >= PB) return;
    const double *g = G + (int64_t)p * PB * PB;
    const double *tp = tau + (int64_t)p * PB;
    double *t = T + (int64_t)p * PB * PB + (int64_t)i * PB;
    for (int k = 0; k < i; ++k) t[k] = 0.0;
    t[i] = tp[i];
    for (int k = i + 1; k < PB; ++k) {
        double s = 0.0;
        for (int j = i; j < k; ++j) s += t[j] * g[(int64_t)j * PB + k];
        t[k] = -tp[k] * s;
    }
}

// V'_p = V_p T_p^T and V''_p = V_p T_p as n x PB BF16 (row j = column j of V):
//   V'[j][k]  = sum_{l >= k} T[k][l] v_l[j],   V''[j][k] = sum_{l <= k} T[l][k] v_l[j].
__global__ void __launch_bounds__(256)
wy_vprime_kernel(const double *__restrict__ V64, const double *__restrict__ T, int64_t n, int PB,
                 __nv_bfloat16 *__restrict__ Vp, __nv_bfloat16 *__restrict__ Vpp) {
    __shared__ double col[256];
    const int64_t j = blockIdx.x;
    const int p = blockIdx.y, k = threadIdx.x;
    if (k < PB) col[k] = V64[((int64_t)p * PB + k) * n + j];
    __syncthreads();
    if (k >= PB) return;
    const double *t = T + (int64_t)p * PB * PB;
    double a = 0.0, b = 0.0;
    for (int l = k; l < PB; ++l) a += t[(int64_t)k * PB + l] * col[l];
    for (int l = 0; l <= k; ++l) b += t[(int64_t)l * PB + k] * col[l];
    const int64_t o = ((int64_t)p * n + j) * PB + k;
    Vp[o] = __float2bfloat16((float)a);
    Vpp[o] = __float2bfloat16((float)b);
}

// ---- the apply kernel -----------------------------------------------------------------------

struct PanelArgs {
    int64_t tiles;
    int n, PB, panel;
    int stages;         // operand ring stages of 16 KB + PB x 128 B
    int estages;        // epilogue ring stages of 16 KB (128 rows x 64 columns)
    const float *sign;  // applied per the flags, or null
    int sign_out;       // y = sigma .* (x - acc)  (W, last panel)
    int sign_in;        // y = sigma .* x - acc    (W^T, first panel; GEMM 1 uses the scaled V)
    int *err;
};

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Shared state of the persistent panel kernel.
struct Bars {
    uint64_t full[kMaxStages], empty[kMaxStages];    // operand ring
    uint64_t efull[kMaxStages], eempty[kMaxStages];  // epilogue ring (x in, y out)
    uint64_t z_full;                                 // Z in tensor memory written
    uint64_t zs_full, zs_free;                       // Z as BF16 operand in tensor memory
    uint64_t acc_full[kNumAcc], acc_empty[kNumAcc];
    uint64_t drain;                                  // every MMA of the CTA has completed
    uint32_t tbase;
    int aborted;
};

// Persistent, warp-specialised panel kernel: one CTA per SM walks 128-row
// tiles.  Shared memory holds an epilogue ring of 128 x 64 boxes of X (y is
// written over x and stored from there) and an operand ring.  Warp 0 (one
// thread) issues the operand loads by TMA in the order the MMAs consume them:
// GEMM 1 K chunks (an X box and a V box) and GEMM 2 output chunks (V' boxes).
// Warp 6 (one thread) loads the epilogue boxes.  Warp 1 (one thread) issues the
// MMAs: GEMM 1 into Z (FP32, tensor-memory columns [0, 256)); GEMM 2 per
// 64-column chunk, A = Z as BF16 in tensor memory (columns [256, 384)), into
// one of two accumulators (columns 384 + 64a).  GEMM 1 of the next tile is
// interleaved with GEMM 2 of the current one, chunk by chunk.  Warps 2..5 (one
// tensor-memory lane quadrant each, one row per thread) convert Z to BF16 in
// tensor memory, then per chunk compute y = x - acc in the epilogue box; one
// thread stores the box by TMA.  Chunks run from the last column to the first,
// so the X boxes GEMM 1 read last are read again first (more L2 hits).  TMA
// zero-fills loads and clips stores at the tensor's edges (rows past the
// batch, columns past n).
__global__ void __launch_bounds__(kThreads, 1)
wy_panel_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapV,
                const __grid_constant__ CUtensorMap mapVp, const __grid_constant__ CUtensorMap mapY,
                PanelArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int n = a.n, PB = a.PB, NS = a.stages, NE = a.estages;
    unsigned char *ering = smem;
    unsigned char *ring = ering + (size_t)NE * kEBox;
    __shared__ Bars B;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int KC = (n + 63) / 64;
    const int NC = (n + kChunkN - 1) / kChunkN;
    const uint32_t bytesX = kTileM * 128, bytesV = (uint32_t)PB * 128;
    const uint32_t stage_bytes = bytesX + bytesV;
    const int ybase = a.panel * PB;  // first row of this panel in V
    const int vpbase = a.panel * n;  // first row of this panel in V' (P x n rows)

    if (tid == 0) {
        B.aborted = 0;
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&B.full[s], 1);
            tc::mbar_init(&B.empty[s], 1);
        }
        for (int s = 0; s < NE; ++s) {
            tc::mbar_init(&B.efull[s], 1);
            tc::mbar_init(&B.eempty[s], 1);
        }
        tc::mbar_init(&B.z_full, 1);
        tc::mbar_init(&B.zs_full, 4);
        tc::mbar_init(&B.zs_free, 1);
        tc::mbar_init(&B.drain, 1);
        for (int c = 0; c < kNumAcc; ++c) {
            tc::mbar_init(&B.acc_full[c], 1);
            tc::mbar_init(&B.acc_empty[c], 4);
        }
        tc::fence_barrier_init();
        tc::prefetch_tensormap(&mapX);
        tc::prefetch_tensormap(&mapV);
        tc::prefetch_tensormap(&mapVp);
        tc::prefetch_tensormap(&mapY);
    }
    if (warp == 1) tc::tmem_alloc(&B.tbase, 512);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tz = B.tbase;

    // Bounded wait; after a timeout the kernel records HH_ERR_TIMEOUT and stops
    // waiting (its results are then not to be trusted).  The copy warps then
    // stop issuing loads and the MMA warp stops issuing MMAs; before tensor
    // memory is freed, each of them waits (bounded) for what it has in flight.
    auto aborted = [&]() { return *(volatile int *)&B.aborted != 0; };
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (aborted()) return;
        if (!tc::mbar_wait(bar, parity)) {
            atomicExch(a.err, (int)HH_ERR_TIMEOUT);
            *(volatile int *)&B.aborted = 1;
        }
    };
    constexpr uint32_t kNone = 0xffffffffu;

    // Order of the operand ring and of the MMAs, per tile i (tiles of this CTA
    // t_0, t_1, ...): GEMM 1 of t_0 alone; then for each tile, output chunk j
    // of GEMM 2 (tile i) is followed by K chunk j of GEMM 1 of tile i+1 while
    // both remain, then the rest of either.  The next tile's X streams in while
    // this tile's epilogue runs, and the tensor pipe works on both.
    const int64_t first = blockIdx.x, step = gridDim.x;
    const int steps = NC > KC ? NC : KC;
    if (warp == 0) {
        // ---- TMA producer: operand ring ----------------------------------------------------
        if (lane == 0) {
            uint32_t it = 0;
            uint32_t last[kMaxStages];  // load index that last armed each stage
            for (int s = 0; s < kMaxStages; ++s) last[s] = kNone;
            auto load1 = [&](int64_t tile, int kc) {
                const uint32_t s = it % NS;
                wait(&B.empty[s], ((it / NS) & 1) ^ 1);
                if (aborted()) return;
                last[s] = it;
                unsigned char *st = ring + s * stage_bytes;
                tc::mbar_expect_tx(&B.full[s], bytesX + bytesV);
                tc::tma_load_2d(st, &mapX, kc * 64, (int)(tile * kTileM), &B.full[s]);
                tc::tma_load_2d(st + bytesX, &mapV, kc * 64, ybase, &B.full[s]);
                ++it;
            };
            auto load2 = [&](int nc) {
                const uint32_t s = it % NS;
                wait(&B.empty[s], ((it / NS) & 1) ^ 1);
                if (aborted()) return;
                last[s] = it;
                unsigned char *st = ring + s * stage_bytes;
                tc::mbar_expect_tx(&B.full[s], (uint32_t)PB * 128);
                for (int kb = 0; kb < PB / 64; ++kb)
                    tc::tma_load_2d(st + kb * (kChunkN * 128), &mapVp, kb * 64, vpbase + nc * kChunkN,
                                    &B.full[s]);
                ++it;
            };
            if (first < a.tiles)
                for (int kc = 0; kc < KC; ++kc) load1(first, kc);
            for (int64_t tile = first; tile < a.tiles && !aborted(); tile += step) {
                const bool next = tile + step < a.tiles;
                for (int j = 0; j < steps; ++j) {
                    if (j < NC) load2(NC - 1 - j);
                    if (next && j < KC) load1(tile + step, j);
                }
            }
            // the last load of each stage has landed before the CTA ends (a
            // no-op unless the kernel gave up a wait: the MMAs consumed them)
            for (int s = 0; s < NS; ++s)
                if (last[s] != kNone) tc::mbar_wait(&B.full[s], (last[s] / NS) & 1);
        }
    } else if (warp == 6) {
        // ---- TMA producer: epilogue boxes of X ----------------------------------------------
        if (lane == 0) {
            uint32_t ei = 0;
            uint32_t last[kMaxStages];  // load index that last armed each box
            for (int e = 0; e < kMaxStages; ++e) last[e] = kNone;
            for (int64_t tile = first; tile < a.tiles && !aborted(); tile += step)
                for (int j = 0; j < NC; ++j, ++ei) {
                    const uint32_t e = ei % NE;
                    wait(&B.eempty[e], ((ei / NE) & 1) ^ 1);
                    if (aborted()) break;
                    last[e] = ei;
                    tc::mbar_expect_tx(&B.efull[e], kEBox);
                    tc::tma_load_2d(ering + e * kEBox, &mapX, (NC - 1 - j) * kChunkN,
                                    (int)(tile * kTileM), &B.efull[e]);
                }
            for (int e = 0; e < NE; ++e)
                if (last[e] != kNone) tc::mbar_wait(&B.efull[e], (last[e] / NE) & 1);
        }
    } else if (warp == 1) {
        // ---- MMA issuer ---------------------------------------------------------------------
        if (lane == 0) {
            const uint32_t id1 = tc::idesc_bf16(kTileM, PB);
            const uint32_t id2 = tc::idesc_bf16(kTileM, kChunkN);
            uint32_t it = 0, ai = 0, ti = 0;
            auto mma1 = [&](int kc) {
                const uint32_t s = it % NS;
                wait(&B.full[s], (it / NS) & 1);
                if (aborted()) return;
                tc::tc_fence_after();
                const uint32_t sa = tc::smem_u32(ring + s * stage_bytes), sb = sa + bytesX;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    tc::mma_bf16(tz, tc::sdesc_sw128(sa + 32 * k), tc::sdesc_sw128(sb + 32 * k), id1,
                                 (kc | k) != 0);
                tc::mma_commit(&B.empty[s]);
                ++it;
            };
            auto mma2 = [&]() {
                const uint32_t c = ai % kNumAcc;
                wait(&B.acc_empty[c], ((ai / kNumAcc) & 1) ^ 1);
                const uint32_t s = it % NS;
                wait(&B.full[s], (it / NS) & 1);
                if (aborted()) return;
                tc::tc_fence_after();
                const uint32_t sb = tc::smem_u32(ring + s * stage_bytes);
                const uint32_t tacc = tz + kTmemAcc + c * kChunkN;
                for (int k = 0; k < PB / 16; ++k) {
                    const uint32_t offb = (uint32_t)(k >> 2) * (kChunkN * 128) + (uint32_t)(k & 3) * 32;
                    tc::mma_bf16_ts(tacc, tz + kTmemZb + 8 * k, tc::sdesc_sw128(sb + offb), id2, k != 0);
                }
                tc::mma_commit(&B.empty[s]);
                tc::mma_commit(&B.acc_full[c]);
                ++it;
                ++ai;
            };
            if (first < a.tiles) {
                for (int kc = 0; kc < KC; ++kc) mma1(kc);
                tc::mma_commit(&B.z_full);
            }
            for (int64_t tile = first; tile < a.tiles && !aborted(); tile += step, ++ti) {
                const bool next = tile + step < a.tiles;
                wait(&B.zs_full, ti & 1);  // Z of this tile is in BF16 columns; the FP32 ones are free
                tc::tc_fence_after();
                for (int j = 0; j < steps; ++j) {
                    if (j < NC) mma2();
                    if (next && j < KC) mma1(j);
                }
                if (next) tc::mma_commit(&B.z_full);
                tc::mma_commit(&B.zs_free);  // GEMM 2 of this tile has read the BF16 Z
            }
            // every MMA issued by this thread (and its commits) has completed
            // before tensor memory is freed, also after a wait was given up
            if (ti > 0) tc::mbar_wait(&B.zs_free, (ti - 1) & 1);
            tc::mma_commit(&B.drain);
            tc::mbar_wait(&B.drain, 0);
        }
    } else {
        // ---- epilogue: warps 2..5, tensor-memory lane quadrant warp % 4 ----------------------
        const int q = warp & 3;
        const int m = q * 32 + lane;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const bool leader = warp == 2 && lane == 0;  // stores the epilogue boxes
        uint32_t ai = 0, ti = 0, ei = 0;
        for (int64_t tile = blockIdx.x; tile < a.tiles; tile += gridDim.x, ++ti) {
            const int row0 = (int)(tile * kTileM);
            wait(&B.z_full, ti & 1);
            wait(&B.zs_free, (ti & 1) ^ 1);  // GEMM 2 of the previous tile has read the BF16 Z
            tc::tc_fence_after();
            for (int c = 0; c < PB / 32; ++c) {
                uint32_t r[32], w[16];
                tc::tmem_ld32(tz + lane_off + (uint32_t)(c * 32), r);
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    w[i] = pack_bf16(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
                tc::tmem_st16(tz + lane_off + kTmemZb + (uint32_t)(c * 16), w);
            }
            tc::tmem_wait_st();
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&B.zs_full);
            for (int j = 0; j < NC; ++j, ++ai, ++ei) {
                const int nc = NC - 1 - j;
                const uint32_t c = ai % kNumAcc;
                const uint32_t e = ei % NE;
                wait(&B.acc_full[c], (ai / kNumAcc) & 1);
                tc::tc_fence_after();
                uint32_t r[kChunkN];
                tc::tmem_ld32(tz + lane_off + kTmemAcc + c * kChunkN,
                              *reinterpret_cast<uint32_t(*)[32]>(r));
                tc::tmem_ld32(tz + lane_off + kTmemAcc + c * kChunkN + 32,
                              *reinterpret_cast<uint32_t(*)[32]>(r + 32));
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&B.acc_empty[c]);
                wait(&B.efull[e], (ei / NE) & 1);
                // row m of the box: 128 bytes, 16-byte granules permuted by the swizzle
                unsigned char *box = ering + e * kEBox + m * 128;
                const int col0 = nc * kChunkN;
#pragma unroll
                for (int q8 = 0; q8 < kChunkN / 8; ++q8) {
                    uint4 *g = reinterpret_cast<uint4 *>(box + ((q8 ^ (m & 7)) << 4));
                    const uint4 xv = *g;
                    float sg[8] = {1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f};
                    if (a.sign && col0 + 8 * q8 + 8 <= n) {
                        const float4 s0 = *reinterpret_cast<const float4 *>(a.sign + col0 + 8 * q8);
                        const float4 s1 = *reinterpret_cast<const float4 *>(a.sign + col0 + 8 * q8 + 4);
                        sg[0] = s0.x; sg[1] = s0.y; sg[2] = s0.z; sg[3] = s0.w;
                        sg[4] = s1.x; sg[5] = s1.y; sg[6] = s1.z; sg[7] = s1.w;
                    }
                    const uint32_t *xw = reinterpret_cast<const uint32_t *>(&xv);
                    uint4 yv;
                    uint32_t *yw = reinterpret_cast<uint32_t *>(&yv);
#pragma unroll
                    for (int e2 = 0; e2 < 4; ++e2) {
                        __nv_bfloat162 x2 = *reinterpret_cast<const __nv_bfloat162 *>(&xw[e2]);
                        float x0 = __low2float(x2), x1 = __high2float(x2);
                        if (a.sign_in) {
                            x0 *= sg[2 * e2];
                            x1 *= sg[2 * e2 + 1];
                        }
                        float y0 = x0 - __uint_as_float(r[8 * q8 + 2 * e2]);
                        float y1 = x1 - __uint_as_float(r[8 * q8 + 2 * e2 + 1]);
                        if (a.sign_out) {
                            y0 *= sg[2 * e2];
                            y1 *= sg[2 * e2 + 1];
                        }
                        yw[e2] = pack_bf16(y0, y1);
                    }
                    *g = yv;
                }
                tc::fence_proxy_async();           // y visible to the TMA store
                tc::named_barrier(1, 128);         // the four epilogue warps
                if (leader) {
                    tc::tma_store_2d(&mapY, ering + e * kEBox, col0, row0);
                    tc::bulk_commit_group();
                    // the previous box's store has read shared memory: its stage is free
                    tc::bulk_wait_read<1>();
                    if (ei > 0) tc::mbar_arrive(&B.eempty[(ei - 1) % NE]);
                }
            }
        }
        if (leader) tc::bulk_wait<0>();  // every store written before the kernel ends
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 1) tc::tmem_dealloc(B.tbase, 512);
}

}  // namespace wy

// ---- host side --------------------------------------------------------------------------

void wy_free(Plan *p) {
    WYPlan *w = reinterpret_cast<WYPlan *>(p->wy);
    if (!w) return;
    cudaFree(w->Vb);
    cudaFree(w->Vs);
    cudaFree(w->Vp);
    cudaFree(w->Vpp);
    cudaFree(w->sign);
    cudaFree(w->V64);
    cudaFree(w->G);
    cudaFree(w->T);
    delete w;
    p->wy = nullptr;
}

hh_status wy_prepare(Plan *p, const void *U, int64_t ldu, const int8_t *sign, int *flag,
                     cudaStream_t st) {
    const int64_t n = p->n, h = p->h;
    if (n < 64 || n % 8 != 0)
        return fail(HH_ERR_UNSUPPORTED, "compact-WY path: n must be a multiple of 8 and >= 64");
    if (h < 1) return fail(HH_ERR_UNSUPPORTED, "compact-WY path: h must be >= 1");
    WYPlan *w = new (std::nothrow) WYPlan();
    if (!w) return fail(HH_ERR_OOM, "host allocation failed");
    p->wy = w;
    // panels of PB reflectors, PB a multiple of 64 (the K blocks of GEMM 2 and
    // the 32-column tensor-memory loads of Z) and at most 256 (N of GEMM 1);
    // zero reflectors (H = I) pad the last panel
    const int64_t h64 = round_up(h, 64);
    w->P = (int)((h64 + 255) / 256);
    w->PB = (int)round_up((h64 + w->P - 1) / w->P, 64);
    w->hpad = (int64_t)w->P * w->PB;
    w->n8 = round_up(n, 8);
    cudaError_t e;
    const size_t bv = sizeof(__nv_bfloat16) * (size_t)w->hpad * w->n8;
    const size_t bvp = sizeof(__nv_bfloat16) * (size_t)w->P * n * w->PB;
    if ((e = dev_malloc(&w->Vb, bv)) || (sign && (e = dev_malloc(&w->Vs, bv))) ||
        (e = dev_malloc(&w->Vp, bvp)) || (e = dev_malloc(&w->Vpp, bvp)) ||
        (sign && (e = dev_malloc(&w->sign, sizeof(float) * n))) ||
        (e = dev_malloc(&w->V64, sizeof(double) * (size_t)w->hpad * n)) ||
        (e = dev_malloc(&w->G, sizeof(double) * (size_t)w->P * w->PB * w->PB)) ||
        (e = dev_malloc(&w->T, sizeof(double) * (size_t)w->P * w->PB * w->PB)) ||
        (e = cudaFree(p->tau)) || (e = dev_malloc(&p->tau, sizeof(double) * (size_t)w->hpad)) ||
        (e = cudaFree(p->vnorm)) || (e = dev_malloc(&p->vnorm, sizeof(double) * (size_t)w->hpad)))
        return cuda_fail(e, "cudaMalloc (compact-WY plan)");
    wy::wy_convert_kernel<<<(unsigned)w->hpad, 256, 0, st>>>(
        (const __nv_bfloat16 *)U, ldu, n, h, w->n8, sign, w->V64, w->Vb, w->Vs, p->tau, p->vnorm,
        flag);
    wy::wy_gram_kernel<<<dim3(w->PB, w->PB, w->P), 128, 0, st>>>(w->V64, n, w->PB, w->G);
    wy::wy_tfactor_kernel<<<w->P, 256, 0, st>>>(w->G, p->tau, w->PB, w->T);
    wy::wy_vprime_kernel<<<dim3((unsigned)n, w->P), 256, 0, st>>>(w->V64, w->T, n, w->PB, w->Vp,
                                                                  w->Vpp);
    if ((e = cudaGetLastError())) return cuda_fail(e, "compact-WY preparation");
    hh_status s;
    if ((s = encode_map_bf16(&w->mapV, w->Vb, n, w->hpad, w->n8 * 2, 64, w->PB))) return s;
    if (sign && (s = encode_map_bf16(&w->mapVs, w->Vs, n, w->hpad, w->n8 * 2, 64, w->PB))) return s;
    if ((s = encode_map_bf16(&w->mapVp, w->Vp, w->PB, (uint64_t)w->P * n, w->PB * 2, 64,
                             wy::kChunkN)))
        return s;
    if ((s = encode_map_bf16(&w->mapVpp, w->Vpp, w->PB, (uint64_t)w->P * n, w->PB * 2, 64,
                             wy::kChunkN)))
        return s;
    return HH_OK;
}

// Sign as float for the epilogue (converted once; int8 +-1 checked by the caller).
__global__ void wy_sign_kernel(const int8_t *__restrict__ s, int64_t n, float *__restrict__ out,
                               int *__restrict__ flag) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (s[j] != 1 && s[j] != -1) atomicOr(flag, 4);
        out[j] = s[j] < 0 ? -1.f : 1.f;
    }
}

hh_status wy_prepare_sign(Plan *p, const int8_t *sign, int *flag, cudaStream_t st) {
    WYPlan *w = reinterpret_cast<WYPlan *>(p->wy);
    if (!sign) return HH_OK;
    wy_sign_kernel<<<(unsigned)((p->n + 255) / 256), 256, 0, st>>>(sign, p->n, w->sign, flag);
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(e, "compact-WY sign") : HH_OK;
}

void wy_release_workspace(Plan *p) {
    WYPlan *w = reinterpret_cast<WYPlan *>(p->wy);
    if (!w) return;
    cudaFree(w->V64);
    cudaFree(w->G);
    cudaFree(w->T);
    w->V64 = w->G = w->T = nullptr;
}

#ifndef HH_WY_GRID_CAP
#define HH_WY_GRID_CAP 0
#endif

hh_status wy_apply(const Plan *p, hh_mode mode, const void *X, int64_t ldx, void *Y, int64_t ldy,
                   int64_t batch, cudaStream_t st) {
    const WYPlan *w = reinterpret_cast<const WYPlan *>(p->wy);
    if (mode == HH_MODE_SYM)
        return fail(HH_ERR_UNSUPPORTED, "compact-WY path: apply_sym is not built (use W and W^T)");
    if ((uintptr_t)X % 16 || (uintptr_t)Y % 16 || ldx % 8 || ldy % 8)
        return fail(HH_ERR_UNSUPPORTED,
                    "compact-WY path: X and Y need 16-byte aligned rows (ld a multiple of 8)");
    static PerDevice attr;  // the shared-memory opt-in, once per device
    int unused = 0;
    cudaError_t ea = per_device(attr, unused, [](int &) {
        return cudaFuncSetAttribute(wy::wy_panel_kernel,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)wy::kSmemBytes);
    });
    if (ea) return cuda_fail(ea, "compact-WY shared-memory opt-in");
    const int64_t tiles = (batch + wy::kTileM - 1) / wy::kTileM;
    if (tiles * wy::kTileM > 0x7fffffffLL) return fail(HH_ERR_INVALID_ARG, "batch too large");
    int grid = (int)std::min<int64_t>(tiles, p->num_sms > 0 ? p->num_sms : 1);
#if HH_WY_GRID_CAP > 0
    if (w->PB <= 64 && grid > HH_WY_GRID_CAP) grid = HH_WY_GRID_CAP;
#endif
    // shared memory: as many epilogue boxes (up to 4) as leave room for at
    // least three operand stages, then the operand ring
    const size_t stage_bytes = 128 * 128 + (size_t)w->PB * 128;
    const size_t avail = wy::kSmemBytes - 1024;
    int estages = 4;
    while (estages > 1 && avail < estages * (size_t)wy::kEBox + 3 * stage_bytes) --estages;
    const int stages = (int)std::min<size_t>(wy::kMaxStages,
                                             (avail - estages * (size_t)wy::kEBox) / stage_bytes);
    if (stages < 2) return fail(HH_ERR_UNSUPPORTED, "compact-WY path: panel too wide for shared memory");
    for (int i = 0; i < w->P; ++i) {
        // W = W_1 ... W_P: W applies panel P first; W^T applies panel 1 first.
        const int panel = mode == HH_MODE_W ? w->P - 1 - i : i;
        const void *in = i == 0 ? X : Y;
        const int64_t ldin = i == 0 ? ldx : ldy;
        CUtensorMap mapX, mapY;
        hh_status s = encode_map_bf16(&mapX, in, p->n, batch, (uint64_t)ldin * 2, 64, wy::kTileM);
        if (!s) s = encode_map_bf16(&mapY, Y, p->n, batch, (uint64_t)ldy * 2, 64, wy::kTileM);
        if (s) return s;
        wy::PanelArgs a;
        a.tiles = tiles;
        a.estages = estages;
        a.n = (int)p->n;
        a.PB = w->PB;
        a.stages = stages;
        a.panel = panel;
        a.sign = w->sign;
        a.sign_out = mode == HH_MODE_W && i == w->P - 1 && w->sign;
        a.sign_in = mode == HH_MODE_WT && i == 0 && w->sign;
        a.err = p->err;
        const CUtensorMap &mv = a.sign_in ? w->mapVs : w->mapV;
        // W: Y = X - Z (V T)^T; W^T: Y = X - Z (V T^T)^T
        const CUtensorMap &mvp = mode == HH_MODE_W ? w->mapVpp : w->mapVp;
        wy::wy_panel_kernel<<<grid, wy::kThreads, wy::kSmemBytes, st>>>(mapX, mv, mvp, mapY, a);
        cudaError_t e = cudaGetLastError();
        if (e) return cuda_fail(e, "compact-WY launch");
    }
    return HH_OK;
}

}  // namespace hh
