// F32 instantiations of the fused chain kernels.  Configurations are picked by
// the number of columns n; COVER = G * NG * 4 columns per row group.
#include "hh_split.cuh"

// Measured (G, NG, RT, RG, B) of the staged configurations for n <= 1024,
// n <= 2048 and n <= 4096 (overridable at compile time for tuning runs).  The
// n <= 1024 and n <= 4096 shapes are wide tiles (32 columns x 4 rows per
// thread, up to 255 registers, 8 warps per SM).
#ifndef HH_N1024_G
#define HH_N1024_G 32
#define HH_N1024_NG 8
#define HH_N1024_RT 4
#define HH_N1024_RG 4
#define HH_N1024_B 2
#endif
#ifndef HH_N2048_G
#define HH_N2048_G 128
#define HH_N2048_NG 4
#define HH_N2048_RT 4
#define HH_N2048_RG 1
#define HH_N2048_B 2
#endif
#ifndef HH_N4096_G
#define HH_N4096_G 128
#define HH_N4096_NG 8
#define HH_N4096_RT 4
#define HH_N4096_RG 1
#define HH_N4096_B 2
#endif

// Eight-CTA clusters for 2048 < n <= 4096 beyond the pair's h (1) or the
// staged kernel there (0).
#ifndef HH_SPLIT8
#define HH_SPLIT8 1
#endif

// Column-split cluster kernel for 2048 < n <= 4096 (each CTA of a pair keeps
// its 2048 columns of every reflector in shared memory): (G, NG, RT, RG, B).
// For 512 < n <= 1024 the same kernel runs on single-CTA "clusters" holding
// all of V (configurations in the dispatch below).
#ifndef HH_SPLIT_G
#define HH_SPLIT_G 64
#define HH_SPLIT_NG 8
#define HH_SPLIT_RT 4
#define HH_SPLIT_RG 4
#define HH_SPLIT_B 4
#endif

namespace hh {

// A second stream per device (non-blocking) with a fork and a join event,
// created on first use (so that a call inside stream capture creates
// nothing): a launch runs part of its work on it beside the caller's stream.
// The mutex also keeps one call's event records and waits together.
struct Side {
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
static std::mutex g_side_mu;

static cudaError_t side_for_device(Side *&out) {
    static Side sides[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    Side &sd = sides[dev];
    if (!sd.stream) {
        if ((e = cudaEventCreateWithFlags(&sd.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&sd.join, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithFlags(&sd.stream, cudaStreamNonBlocking)) != cudaSuccess)
            return e;
    }
    out = &sd;
    return cudaSuccess;
}

// The column-split kernels (which can store p inside the mode-S pass) take
// these shapes.
static bool split_shape(int vec_ok, int64_t n, int h, const int *start) {
    if (!(vec_ok && n % 4 == 0 && n <= 8192)) return false;
#ifndef HH_NO_SPLIT
    if (n > 512 && n <= 1024 && !start && h >= 1 && h <= split::max_h<32, 8, 4, 8, 4, 1>())
        return true;
    if (n > 2048 && n <= 4096 && !start &&
        h <= split::max_h<HH_SPLIT_G, HH_SPLIT_NG, HH_SPLIT_RT, HH_SPLIT_RG, HH_SPLIT_B>())
        return true;
#if HH_SPLIT8
    if (n > 2048 && n <= 4096 && !start && h <= split::max_h<32, 4, 8, 8, 4>()) return true;
#endif
#endif
    return false;
}

static cudaError_t dispatch_f32(hh_mode mode, const float *X, int64_t ldx, float *Y, int64_t ldy,
                                int64_t batch, int64_t n, const float *U, const float *tau,
                                int64_t ldv, int h, const float *gram, const float *sign,
                                const float *d, int vec_ok, int *err, int num_sms, cudaStream_t st,
                                const int *start, float *P, int64_t ldp);

// P (mode S only, may be null): also write p = W^T (sigma .* x), inside the
// pass where the split kernels run, else by a W^T pass before it (so that
// Y may alias X).
cudaError_t fused_dispatch_f32(hh_mode mode, const float *X, int64_t ldx, float *Y, int64_t ldy,
                               int64_t batch, int64_t n, const float *U, const float *tau, int64_t ldv, int h,
                               const float *gram, const float *sign, const float *d, int vec_ok,
                               int *err, int num_sms, cudaStream_t st, const int *start, float *P,
                               int64_t ldp) {
    if (mode == HH_MODE_SYM && P && !split_shape(vec_ok, n, h, start)) {
        cudaError_t e = dispatch_f32(HH_MODE_WT, X, ldx, P, ldp, batch, n, U, tau, ldv, h, gram,
                                     sign, d, vec_ok, err, num_sms, st, start, nullptr, 0);
        if (e != cudaSuccess) return e;
        P = nullptr;
    }
    return dispatch_f32(mode, X, ldx, Y, ldy, batch, n, U, tau, ldv, h, gram, sign, d, vec_ok, err,
                        num_sms, st, start, mode == HH_MODE_SYM ? P : nullptr, ldp);
}

static cudaError_t dispatch_f32(hh_mode mode, const float *X, int64_t ldx, float *Y, int64_t ldy,
                                int64_t batch, int64_t n, const float *U, const float *tau,
                                int64_t ldv, int h, const float *gram, const float *sign,
                                const float *d, int vec_ok, int *err, int num_sms, cudaStream_t st,
                                const int *start, float *P, int64_t ldp) {
    using namespace fused;
    const int ni = (int)n;
    // Aligned rows with n % 4 == 0: persistent blocked kernel, tiles prefetched
    // into shared memory by bulk copies.
    if (vec_ok && n % 4 == 0 && n <= 8192) {
#define HH_STAGED(G, NG, RT, RG, B)                                                            \
    staged::launch<G, NG, RT, RG, B>(mode, X, ldx, Y, ldy, batch, ni, U, tau, ldv, h, gram, sign, \
                                     d, err, num_sms, st, start)
        // (G, NG, RT, RG, B): 4 rows per thread where the register budget allows,
        // so each loaded reflector value feeds 8 FMAs; B reflectors per round;
        // 32 columns per thread where n is large enough to fill them.
        if (n <= 128) return HH_STAGED(32, 1, 8, 4, 2);
        if (n <= 256) return HH_STAGED(32, 2, 8, 4, 2);
        if (n <= 512) return HH_STAGED(32, 4, 4, 4, 2);
#ifndef HH_NO_SPLIT
        // 512 < n <= 1024 with h <= 50: every reflector resident in one CTA's
        // shared memory, one warp per row group (no exchange); four reflectors
        // per round from h = 16, two below (measured).
        if (n > 512 && n <= 1024 && !start && h >= 1 &&
            h <= split::max_h<32, 8, 4, 8, 4, 1>()) {
            if (h >= 16)
                return split::launch<32, 8, 4, 8, 4, 1, 1>(mode, X, ldx, Y, ldy, batch, ni, U, tau,
                                                           ldv, h, gram, sign, d, err, st, P, ldp);
            return split::launch<32, 8, 4, 8, 2, 1, 1>(mode, X, ldx, Y, ldy, batch, ni, U, tau, ldv,
                                                       h, gram, sign, d, err, st, P, ldp);
        }
#endif
        if (n <= 1024) return HH_STAGED(HH_N1024_G, HH_N1024_NG, HH_N1024_RT, HH_N1024_RG, HH_N1024_B);
        if (n <= 2048) return HH_STAGED(HH_N2048_G, HH_N2048_NG, HH_N2048_RT, HH_N2048_RG, HH_N2048_B);
#ifndef HH_NO_SPLIT
        if (n > 2048 && n <= 4096 && !start &&
            h <= split::max_h<HH_SPLIT_G, HH_SPLIT_NG, HH_SPLIT_RT, HH_SPLIT_RG, HH_SPLIT_B>())
            return split::launch<HH_SPLIT_G, HH_SPLIT_NG, HH_SPLIT_RT, HH_SPLIT_RG, HH_SPLIT_B>(
                mode, X, ldx, Y, ldy, batch, ni, U, tau, ldv, h, gram, sign, d, err, st, P, ldp);
#if HH_SPLIT8
        // larger h: clusters of eight CTAs, each keeping 512 columns of every
        // reflector (32 threads x 16 columns x 8 rows per row group)
        if (n > 2048 && n <= 4096 && !start && h <= split::max_h<32, 4, 8, 8, 4>()) {
            int ncl = 0;
            cudaError_t e = split::resident_clusters<32, 4, 8, 8, 4, 8, 1>(mode, ncl);
            if (e != cudaSuccess) return e;
            // Eight-CTA clusters cannot fill every SM (a GPC's SMs are not a
            // multiple of eight).  The SMs they leave run the staged kernel on
            // a share of the rows, on a second stream ordered by events; per
            // SM the cluster kernel is about 1.3x as fast.  The cluster launch
            // takes the highest priority so that its CTAs are placed first.
            // (Requests that keep p stay on the cluster kernel.)
            constexpr int64_t kUnit = 64;  // rows of one cluster round: 8 groups x 8 rows
            const int idle = num_sms - 8 * ncl;
            if (!P && idle > 0 && batch >= (int64_t)num_sms * kUnit) {
                const double w8 = 1.3 * 8.0 * ncl, ws = (double)idle;
                const int64_t b1 = (int64_t)((double)batch * w8 / (w8 + ws)) / kUnit * kUnit;
                std::lock_guard<std::mutex> lock(g_side_mu);
                Side *sd = nullptr;
                if ((e = side_for_device(sd)) != cudaSuccess) return e;
                cudaStream_t side = sd->stream;
                e = cudaEventRecord(sd->fork, st);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(side, sd->fork, 0);
                if (e == cudaSuccess)
                    e = split::launch<32, 4, 8, 8, 4, 8, 1>(mode, X, ldx, Y, ldy, b1, ni, U, tau,
                                                            ldv, h, gram, sign, d, err, st,
                                                            nullptr, 0, true);
                if (e == cudaSuccess)
                    e = staged::launch<HH_N4096_G, HH_N4096_NG, HH_N4096_RT, HH_N4096_RG,
                                       HH_N4096_B>(mode, X + b1 * ldx, ldx, Y + b1 * ldy, ldy,
                                                   batch - b1, ni, U, tau, ldv, h, gram, sign, d,
                                                   err, idle, side, nullptr);
                if (e == cudaSuccess) e = cudaEventRecord(sd->join, side);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(st, sd->join, 0);
                return e;
            }
            return split::launch<32, 4, 8, 8, 4, 8, 1>(mode, X, ldx, Y, ldy, batch, ni, U, tau, ldv,
                                                       h, gram, sign, d, err, st, P, ldp);
        }
#endif
#endif
        if (n <= 4096) return HH_STAGED(HH_N4096_G, HH_N4096_NG, HH_N4096_RT, HH_N4096_RG, HH_N4096_B);
        return HH_STAGED(512, 4, 2, 1, 2);
#undef HH_STAGED
    }
#define HH_LAUNCH(G, NG, RT, RG) \
    launch_cfg<float, G, NG, RT, RG>(mode, X, ldx, Y, ldy, batch, ni, U, tau, ldv, h, sign, d, vec_ok, st)
    if (n <= 128) return HH_LAUNCH(32, 1, 4, 8);
    if (n <= 256) return HH_LAUNCH(32, 2, 4, 8);
    if (n <= 512) return HH_LAUNCH(32, 4, 4, 8);
    if (n <= 1024) return HH_LAUNCH(64, 4, 4, 4);
    if (n <= 2048) return HH_LAUNCH(128, 4, 4, 2);
    if (n <= 4096) return HH_LAUNCH(256, 4, 4, 2);
    if (n <= 8192) return HH_LAUNCH(512, 4, 2, 1);
    if (n <= 16384) return HH_LAUNCH(1024, 4, 1, 1);
#undef HH_LAUNCH
    return launch_wide<float>(mode, X, ldx, Y, ldy, batch, n, U, tau, ldv, h, sign, d, st);
}

}  // namespace hh
