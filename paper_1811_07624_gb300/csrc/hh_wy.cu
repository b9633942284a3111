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
// Kernel, per 128-row tile, one CTA of 4 warps: thread 0 issues the TMA loads
// (128-byte swizzle) and the tcgen05 MMAs; GEMM 1 streams K in chunks of 64
// through a 2-stage ring into tensor memory; the warps move Z (FP32) to shared
// memory as BF16 in the operand layout; GEMM 2 runs over N in chunks of 128
// with two tensor-memory accumulators, so the MMAs of chunk c+1 overlap the
// epilogue of chunk c (y = x - acc, read from tensor memory by the warp that
// owns the row).  All mbarrier waits are bounded.
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

constexpr int kTileM = 128;
constexpr int kChunkN = 128;
constexpr int kThreads = 128;
constexpr size_t kStageBytes = 64 * 1024;  // ring stage: max(A 16 KB + B PB*128 B, PB*256 B)
constexpr size_t kZBytes = 64 * 1024;      // 128 x 256 BF16
constexpr size_t kSmemBytes = 1024 + 2 * kStageBytes + kZBytes;

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
    const __nv_bfloat16 *Xin;   // panel input (epilogue reads x here)
    int64_t ldx;
    __nv_bfloat16 *Y;
    int64_t ldy;
    int64_t batch;
    int n, PB, panel;
    const float *sign;  // applied per the flags, or null
    int sign_out;       // y = sigma .* (x - acc)  (W, last panel)
    int sign_in;        // y = sigma .* x - acc    (W^T, first panel; GEMM 1 uses the scaled V)
    int *err;
};

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

__global__ void __launch_bounds__(kThreads, 1)
wy_panel_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapV,
                const __grid_constant__ CUtensorMap mapVp, PanelArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *stage[2] = {smem, smem + kStageBytes};
    unsigned char *Zs = smem + 2 * kStageBytes;
    __shared__ __align__(8) uint64_t full[2], empty[2], zbar, accbar[2];
    __shared__ uint32_t tbase;
    __shared__ int aborted;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.n, PB = a.PB;
    const int64_t row0 = (int64_t)blockIdx.x * kTileM;
    const int KC = (n + 63) / 64;
    const int NC = (n + kChunkN - 1) / kChunkN;
    const uint32_t bytesA = kTileM * 128, bytesB1 = (uint32_t)PB * 128, bytesB2 = (uint32_t)PB * 256;
    const int ybase = a.panel * PB;  // first row of this panel in V
    const int vpbase = a.panel * n;  // first row of this panel in V' (P x n rows)

    if (warp == 0) tc::tmem_alloc(&tbase, 512);
    if (tid == 0) {
        aborted = 0;
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
            tc::mbar_init(&accbar[s], 1);
        }
        tc::mbar_init(&zbar, 1);
        tc::fence_barrier_init();
        tc::prefetch_tensormap(&mapX);
        tc::prefetch_tensormap(&mapV);
        tc::prefetch_tensormap(&mapVp);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tz = tbase;                 // Z: columns [0, PB)
    const uint32_t tacc[2] = {tbase + 256, tbase + 384};

    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (*(volatile int *)&aborted) return;
        if (!tc::mbar_wait(bar, parity)) {
            atomicExch(a.err, (int)HH_ERR_TIMEOUT);
            tc::mbar_wait(bar, parity);
            *(volatile int *)&aborted = 1;
        }
    };

    // ---- GEMM 1: Z = X_tile V_panel^T over K = n -------------------------------------------
    if (tid == 0) {
        auto load1 = [&](int kc, int s) {
            tc::mbar_expect_tx(&full[s], bytesA + bytesB1);
            tc::tma_load_2d(stage[s], &mapX, kc * 64, (int)row0, &full[s]);
            tc::tma_load_2d(stage[s] + bytesA, &mapV, kc * 64, ybase, &full[s]);
        };
        load1(0, 0);
        if (KC > 1) load1(1, 1);
        const uint32_t id1 = tc::idesc_bf16(kTileM, PB);
        for (int kc = 0; kc < KC; ++kc) {
            const int s = kc & 1;
            wait(&full[s], (uint32_t)((kc >> 1) & 1));
            tc::tc_fence_after();
            const uint32_t sa = tc::smem_u32(stage[s]), sb = sa + bytesA;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                tc::mma_bf16(tz, tc::sdesc_sw128(sa + 32 * k), tc::sdesc_sw128(sb + 32 * k), id1,
                             (kc | k) != 0);
            tc::mma_commit(&empty[s]);
            if (kc + 2 < KC) {
                wait(&empty[s], (uint32_t)((kc >> 1) & 1));
                load1(kc + 2, s);
            }
        }
        tc::mma_commit(&zbar);
    }
    wait(&zbar, 0);
    tc::tc_fence_after();

    // ---- Z (FP32, tensor memory) -> BF16 operand in shared memory ----------------------------
    {
        const int m = warp * 32 + lane;
        for (int c = 0; c < PB / 32; ++c) {
            uint32_t r[32];
            tc::tmem_ld32(tz + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), r);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint4 w;
                w.x = pack_bf16(__uint_as_float(r[8 * q + 0]), __uint_as_float(r[8 * q + 1]));
                w.y = pack_bf16(__uint_as_float(r[8 * q + 2]), __uint_as_float(r[8 * q + 3]));
                w.z = pack_bf16(__uint_as_float(r[8 * q + 4]), __uint_as_float(r[8 * q + 5]));
                w.w = pack_bf16(__uint_as_float(r[8 * q + 6]), __uint_as_float(r[8 * q + 7]));
                *reinterpret_cast<uint4 *>(Zs + tc::sw128_offset(m, c * 32 + 8 * q, kTileM)) = w;
            }
        }
    }
    tc::fence_proxy_async();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();

    // ---- GEMM 2: acc = Z V'^T per chunk of 128 columns; y = x - acc --------------------------
    const uint32_t id2 = tc::idesc_bf16(kTileM, kChunkN);
    auto load2 = [&](int nc, int s) {
        tc::mbar_expect_tx(&full[s], bytesB2);
        for (int kb = 0; kb < PB / 64; ++kb)
            tc::tma_load_2d(stage[s] + kb * (kChunkN * 128), &mapVp, kb * 64, vpbase + nc * kChunkN,
                            &full[s]);
    };
    auto mma2 = [&](int nc) {
        const int s = nc & 1;
        // full[s] phases: GEMM 1 used ceil(KC/2) or floor(KC/2) of them
        const int used = (KC + 1 - s) / 2;
        wait(&full[s], (uint32_t)((used + (nc >> 1)) & 1));
        tc::tc_fence_after();
        const uint32_t sz = tc::smem_u32(Zs), sb = tc::smem_u32(stage[s]);
        for (int k = 0; k < PB / 16; ++k) {
            const uint32_t off = (uint32_t)(k >> 2) * (kTileM * 128) + (uint32_t)(k & 3) * 32;
            const uint32_t offb = (uint32_t)(k >> 2) * (kChunkN * 128) + (uint32_t)(k & 3) * 32;
            tc::mma_bf16(tacc[s], tc::sdesc_sw128(sz + off), tc::sdesc_sw128(sb + offb), id2, k != 0);
        }
        tc::mma_commit(&accbar[s]);
    };
    if (tid == 0) {
        load2(0, 0);
        if (NC > 1) load2(1, 1);
        mma2(0);
    }
    const int m = warp * 32 + lane;
    const int64_t row = row0 + m;
    for (int nc = 0; nc < NC; ++nc) {
        const int s = nc & 1;
        wait(&accbar[s], (uint32_t)((nc >> 1) & 1));
        tc::tc_fence_after();
        if (tid == 0) {
            if (nc + 1 < NC) mma2(nc + 1);  // its accumulator was drained at nc - 1
            if (nc + 2 < NC) load2(nc + 2, s);  // chunk nc's MMAs are done: stage s is free
        }
        for (int c = 0; c < kChunkN / 32; ++c) {
            uint32_t r[32];
            tc::tmem_ld32(tacc[s] + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), r);
            const int col0 = nc * kChunkN + c * 32;
            if (row >= a.batch || col0 >= n) continue;
            const __nv_bfloat16 *xr = a.Xin + row * a.ldx;
            __nv_bfloat16 *yr = a.Y + row * a.ldy;
            if (col0 + 32 <= n) {
                uint4 xv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) xv[q] = *reinterpret_cast<const uint4 *>(xr + col0 + 8 * q);
                uint4 yv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t *xw = reinterpret_cast<const uint32_t *>(&xv[q]);
                    uint32_t *yw = reinterpret_cast<uint32_t *>(&yv[q]);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        __nv_bfloat162 x2 = *reinterpret_cast<const __nv_bfloat162 *>(&xw[e]);
                        float x0 = __low2float(x2), x1 = __high2float(x2);
                        const int cc = col0 + 8 * q + 2 * e;
                        float s0 = 1.f, s1 = 1.f;
                        if (a.sign) {
                            s0 = a.sign[cc];
                            s1 = a.sign[cc + 1];
                        }
                        if (a.sign_in) {
                            x0 *= s0;
                            x1 *= s1;
                        }
                        float y0 = x0 - __uint_as_float(r[8 * q + 2 * e]);
                        float y1 = x1 - __uint_as_float(r[8 * q + 2 * e + 1]);
                        if (a.sign_out) {
                            y0 *= s0;
                            y1 *= s1;
                        }
                        yw[e] = pack_bf16(y0, y1);
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) *reinterpret_cast<uint4 *>(yr + col0 + 8 * q) = yv[q];
            } else {
                for (int e = 0; e < 32 && col0 + e < n; ++e) {
                    const int cc = col0 + e;
                    const float sg = a.sign ? a.sign[cc] : 1.f;
                    float x = __bfloat162float(xr[cc]);
                    if (a.sign_in) x *= sg;
                    float y = x - __uint_as_float(r[e]);
                    if (a.sign_out) y *= sg;
                    yr[cc] = __float2bfloat16(y);
                }
            }
        }
        tc::tc_fence_before();
        __syncthreads();
        tc::tc_fence_after();
    }
    if (warp == 0) tc::tmem_dealloc(tbase, 512);
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
    if ((e = cudaMalloc(&w->Vb, bv)) || (sign && (e = cudaMalloc(&w->Vs, bv))) ||
        (e = cudaMalloc(&w->Vp, bvp)) || (e = cudaMalloc(&w->Vpp, bvp)) ||
        (sign && (e = cudaMalloc(&w->sign, sizeof(float) * n))) ||
        (e = cudaMalloc(&w->V64, sizeof(double) * (size_t)w->hpad * n)) ||
        (e = cudaMalloc(&w->G, sizeof(double) * (size_t)w->P * w->PB * w->PB)) ||
        (e = cudaMalloc(&w->T, sizeof(double) * (size_t)w->P * w->PB * w->PB)) ||
        (e = cudaFree(p->tau)) || (e = cudaMalloc(&p->tau, sizeof(double) * (size_t)w->hpad)) ||
        (e = cudaFree(p->vnorm)) || (e = cudaMalloc(&p->vnorm, sizeof(double) * (size_t)w->hpad)))
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
    if ((s = encode_map_bf16(&w->mapVp, w->Vp, w->PB, (uint64_t)w->P * n, w->PB * 2, 64, 128)))
        return s;
    if ((s = encode_map_bf16(&w->mapVpp, w->Vpp, w->PB, (uint64_t)w->P * n, w->PB * 2, 64, 128)))
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

hh_status wy_apply(const Plan *p, hh_mode mode, const void *X, int64_t ldx, void *Y, int64_t ldy,
                   int64_t batch, cudaStream_t st) {
    const WYPlan *w = reinterpret_cast<const WYPlan *>(p->wy);
    if (mode == HH_MODE_SYM)
        return fail(HH_ERR_UNSUPPORTED, "compact-WY path: apply_sym is not built (use W and W^T)");
    if ((uintptr_t)X % 16 || (uintptr_t)Y % 16 || ldx % 8 || ldy % 8)
        return fail(HH_ERR_UNSUPPORTED,
                    "compact-WY path: X and Y need 16-byte aligned rows (ld a multiple of 8)");
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(wy::wy_panel_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)wy::kSmemBytes);
        if (e) return cuda_fail(e, "compact-WY shared-memory opt-in");
        attr = true;
    }
    const int64_t tiles = (batch + wy::kTileM - 1) / wy::kTileM;
    if (tiles > 0x7fffffffLL) return fail(HH_ERR_INVALID_ARG, "batch too large");
    for (int i = 0; i < w->P; ++i) {
        // W = W_1 ... W_P: W applies panel P first; W^T applies panel 1 first.
        const int panel = mode == HH_MODE_W ? w->P - 1 - i : i;
        const void *in = i == 0 ? X : Y;
        const int64_t ldin = i == 0 ? ldx : ldy;
        CUtensorMap mapX;
        hh_status s = encode_map_bf16(&mapX, in, p->n, batch, (uint64_t)ldin * 2, 64, wy::kTileM);
        if (s) return s;
        wy::PanelArgs a;
        a.Xin = (const __nv_bfloat16 *)in;
        a.ldx = ldin;
        a.Y = (__nv_bfloat16 *)Y;
        a.ldy = ldy;
        a.batch = batch;
        a.n = (int)p->n;
        a.PB = w->PB;
        a.panel = panel;
        a.sign = w->sign;
        a.sign_out = mode == HH_MODE_W && i == w->P - 1 && w->sign;
        a.sign_in = mode == HH_MODE_WT && i == 0 && w->sign;
        a.err = p->err;
        const CUtensorMap &mv = a.sign_in ? w->mapVs : w->mapV;
        // W: Y = X - Z (V T)^T; W^T: Y = X - Z (V T^T)^T
        const CUtensorMap &mvp = mode == HH_MODE_W ? w->mapVpp : w->mapVp;
        wy::wy_panel_kernel<<<(unsigned)tiles, wy::kThreads, wy::kSmemBytes, st>>>(mapX, mv, mvp, a);
        cudaError_t e = cudaGetLastError();
        if (e) return cuda_fail(e, "compact-WY launch");
    }
    return HH_OK;
}

}  // namespace hh
