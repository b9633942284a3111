// F64 instantiations of the fused chain kernels (COVER = G * NG * 2 columns).
#include "hh_fused.cuh"

namespace hh {

cudaError_t fused_dispatch_f64(hh_mode mode, const double *X, int64_t ldx, double *Y,
                               int64_t ldy, int64_t batch, int64_t n, const double *U,
                               const double *tau, int64_t ldv, int h, const double *sign, const double *d,
                               int vec_ok, cudaStream_t st) {
    using namespace fused;
    const int ni = (int)n;
#define HH_LAUNCH(G, NG, RT, RG) \
    launch_cfg<double, G, NG, RT, RG>(mode, X, ldx, Y, ldy, batch, ni, U, tau, ldv, h, sign, d, vec_ok, st)
    if (n <= 64) return HH_LAUNCH(32, 1, 2, 8);
    if (n <= 128) return HH_LAUNCH(32, 2, 2, 8);
    if (n <= 256) return HH_LAUNCH(32, 4, 2, 8);
    if (n <= 512) return HH_LAUNCH(64, 4, 2, 4);
    if (n <= 1024) return HH_LAUNCH(128, 4, 2, 2);
    if (n <= 2048) return HH_LAUNCH(256, 4, 2, 2);
    if (n <= 4096) return HH_LAUNCH(512, 4, 2, 1);
    if (n <= 8192) return HH_LAUNCH(1024, 4, 1, 1);
#undef HH_LAUNCH
    return launch_wide<double>(mode, X, ldx, Y, ldy, batch, n, U, tau, ldv, h, sign, d, st);
}

}  // namespace hh
