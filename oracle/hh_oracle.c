/*
 * hh_oracle.c -- plain, slow FP64 reference for the Householder-chain
 * transforms of Rusu, "Approximate Eigenvalue Decompositions of Linear
 * Transformations with a Few Householder Reflectors" (arXiv 1811.07624).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code, header
 * or constant with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes (all arithmetic in double, plain loops, one vector at a
 * time; OpenMP only splits the batch across host threads: each vector's
 * arithmetic is sequential and the same for any thread count, and only the
 * batch sums of the backward depend on it, at rounding level):
 *
 *   reflector    H_k = I - tau_k v_k v_k^T,  tau_k = 2 / (v_k^T v_k)
 *                (§II-A, Eq. (2): H_k = I - 2 u_k u_k^T with u_k = v_k/|v_k|),
 *                tau_k = 0 when v_k = 0, i.e. H_k = I (the "u_k = 0" reflector
 *                of Result 1, §II-B);
 *   chain        W = H_1 H_2 ... H_h, so in W x the reflector H_h acts first
 *                (the ordering of Eqs. (23)-(24) and of Result 3, §II-D);
 *   mode 0 (W)   y = sigma .* (W x)               (Eq. (1), D on the left)
 *   mode 1 (WT)  y = W^T (sigma .* x)             (right factor of Eq. (21))
 *   mode 2 (SYM) y = sigma .* W (d .* W^T (sigma .* x))       (Eq. (21))
 *
 * sigma is the +-1 diagonal D of Eq. (1) (NULL means all +1); d is the
 * spectrum s-bar of Eq. (21).
 *
 * Backward: for a scalar loss L with g = dL/dy per vector, the gradients
 * dL/dx, dL/dv_k (v_k as given, unnormalised) and dL/dd, summed over the
 * batch.  The intermediate vectors of the chain are STORED (not recomputed),
 * and the derivative of one reflector is taken directly with respect to v_k
 * from its definition a' = a - tau v (v^T a), tau = 2/(v^T v):
 *   dL/dv = tau^2 (v^T a)(v^T G) v - tau (v^T a) G - tau (v^T G) a,
 *   dL/da = H G,
 * where G = dL/da' and a is the reflector's input.
 *
 * Fast Mahalanobis distance (§IV-C): for pairs (i, j),
 *   d_S(x_i, x_j) = (x_i - x_j)^T Sbar (x_i - x_j)
 *                 = sum_m d_m [W^T (sigma .* (x_i - x_j))]_m^2.
 *
 * Layouts: U holds h reflectors, reflector k at U + k*ldu (n doubles).
 * X, Y and gradients are row-major with the given leading dimensions.
 * Return value 0 on success, -1 on an invalid argument.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_W 0
#define ORACLE_WT 1
#define ORACLE_SYM 2

static double dot(int64_t n, const double *a, const double *b) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += a[j] * b[j];
    return s;
}

/* tau_k = 2 / (v_k^T v_k), 0 for the zero vector (§II-A Eq. (2), §II-B). */
int oracle_tau(int64_t n, int64_t h, const double *U, int64_t ldu, double *tau) {
    if (n < 1 || h < 0 || (h > 0 && (!U || !tau)) || ldu < n) return -1;
    for (int64_t k = 0; k < h; ++k) {
        double nn = dot(n, U + k * ldu, U + k * ldu);
        tau[k] = (nn > 0.0) ? 2.0 / nn : 0.0;
    }
    return 0;
}

/* z <- H_k z = z - tau_k v_k (v_k^T z). */
static void reflect(int64_t n, const double *v, double tau, double *z) {
    if (tau == 0.0) return;
    double c = tau * dot(n, v, z);
    for (int64_t j = 0; j < n; ++j) z[j] -= c * v[j];
}

/* z <- W z: H_h first, H_1 last. */
static void chain_W(int64_t n, int64_t h, const double *U, int64_t ldu,
                    const double *tau, double *z) {
    for (int64_t k = h - 1; k >= 0; --k) reflect(n, U + k * ldu, tau[k], z);
}

/* z <- W^T z = H_h ... H_1 z: H_1 first. */
static void chain_WT(int64_t n, int64_t h, const double *U, int64_t ldu,
                     const double *tau, double *z) {
    for (int64_t k = 0; k < h; ++k) reflect(n, U + k * ldu, tau[k], z);
}

static void apply_sign(int64_t n, const signed char *sigma, double *z) {
    if (!sigma) return;
    for (int64_t j = 0; j < n; ++j) z[j] *= (double)sigma[j];
}

static int set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int oracle_max_threads(void) { return set_threads(0); }

/* Forward apply, modes W / WT / SYM (Eq. (1), Eq. (21)). */
int oracle_apply(int mode, int64_t n, int64_t h, const double *U, int64_t ldu,
                 const signed char *sigma, const double *d, int64_t B,
                 const double *X, int64_t ldx, double *Y, int64_t ldy, int nthreads) {
    if (n < 1 || h < 0 || B < 0 || ldx < n || ldy < n || ldu < n) return -1;
    if (mode < ORACLE_W || mode > ORACLE_SYM) return -1;
    if (mode == ORACLE_SYM && !d) return -1;
    if (B > 0 && (!X || !Y)) return -1;
    double *tau = (double *)malloc(sizeof(double) * (size_t)(h > 0 ? h : 1));
    if (!tau) return -1;
    if (oracle_tau(n, h, U, ldu, tau) != 0) { free(tau); return -1; }
    set_threads(nthreads);
    int bad = 0;
#pragma omp parallel
    {
        double *z = (double *)malloc(sizeof(double) * (size_t)n);
        if (!z) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(static)
        for (int64_t b = 0; b < B; ++b) {
            if (!z) continue;
            memcpy(z, X + b * ldx, sizeof(double) * (size_t)n);
            if (mode == ORACLE_W) {
                chain_W(n, h, U, ldu, tau, z);
                apply_sign(n, sigma, z);
            } else if (mode == ORACLE_WT) {
                apply_sign(n, sigma, z);
                chain_WT(n, h, U, ldu, tau, z);
            } else {
                apply_sign(n, sigma, z);
                chain_WT(n, h, U, ldu, tau, z);
                for (int64_t j = 0; j < n; ++j) z[j] *= d[j];
                chain_W(n, h, U, ldu, tau, z);
                apply_sign(n, sigma, z);
            }
            memcpy(Y + b * ldy, z, sizeof(double) * (size_t)n);
        }
        free(z);
    }
    free(tau);
    return bad ? -1 : 0;
}

/*
 * One reflector's backward step with the stored input a of a' = H a and the
 * incoming gradient G = dL/da'.  Adds dL/dv into gv, overwrites G by dL/da.
 */
static void reflect_backward(int64_t n, const double *v, double tau,
                             const double *a, double *G, double *gv) {
    if (tau == 0.0) return; /* H = I: no dependence on v, G unchanged */
    double va = dot(n, v, a);
    double vg = dot(n, v, G);
    double cv = tau * tau * va * vg;
    for (int64_t j = 0; j < n; ++j) gv[j] += cv * v[j] - tau * va * G[j] - tau * vg * a[j];
    for (int64_t j = 0; j < n; ++j) G[j] -= tau * vg * v[j];
}

/*
 * Backward of the three modes.  X is the forward input; gY the gradient with
 * respect to the output.  gX (B x n, ldg) may be NULL; gU (h x n, row k at
 * gU + k*ldu) and gd (n) are sums over the batch and may be NULL; gd is only
 * meaningful for SYM.  States are stored per vector.
 */
int oracle_backward(int mode, int64_t n, int64_t h, const double *U, int64_t ldu,
                    const signed char *sigma, const double *d, int64_t B,
                    const double *X, int64_t ldx, const double *gY, int64_t ldgy,
                    double *gX, int64_t ldgx, double *gU, double *gd, int nthreads) {
    if (n < 1 || h < 0 || B < 0 || ldx < n || ldgy < n || ldu < n) return -1;
    if (gX && ldgx < n) return -1;
    if (mode < ORACLE_W || mode > ORACLE_SYM) return -1;
    if (mode == ORACLE_SYM && !d) return -1;
    double *tau = (double *)malloc(sizeof(double) * (size_t)(h > 0 ? h : 1));
    if (!tau) return -1;
    if (oracle_tau(n, h, U, ldu, tau) != 0) { free(tau); return -1; }
    int nt = set_threads(nthreads);
    /* per-thread gradient sums, reduced in thread order at the end */
    size_t gu_sz = (size_t)h * (size_t)n, gd_sz = (size_t)n;
    double *gu_all = (double *)calloc((size_t)nt * (gu_sz + gd_sz) + 1, sizeof(double));
    if (!gu_all) { free(tau); return -1; }
    int bad = 0;
#pragma omp parallel num_threads(nt)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *gu_t = gu_all + (size_t)t * (gu_sz + gd_sz);
        double *gd_t = gu_t + gu_sz;
        /* sa: states of the W part, sb: states of the W^T part */
        double *sa = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(h + 1));
        double *sb = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(h + 1));
        double *G = (double *)malloc(sizeof(double) * (size_t)n);
        if (!sa || !sb || !G) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(static)
        for (int64_t b = 0; b < B; ++b) {
            if (!sa || !sb || !G) continue;
            const double *x = X + b * ldx;
            memcpy(G, gY + b * ldgy, sizeof(double) * (size_t)n);
            /* --- forward with stored states --- */
            /* W^T part (modes WT and SYM): sb[k] = input of H_{k+1}, k = 0..h-1; sb[h] = output */
            if (mode != ORACLE_W) {
                memcpy(sb, x, sizeof(double) * (size_t)n);
                apply_sign(n, sigma, sb);
                for (int64_t k = 0; k < h; ++k) {
                    memcpy(sb + (k + 1) * n, sb + k * n, sizeof(double) * (size_t)n);
                    reflect(n, U + k * ldu, tau[k], sb + (k + 1) * n);
                }
            }
            /* W part (modes W and SYM): sa[h] = input, sa[k] = H_{k+1} sa[k+1];
               so sa[k] is the input of H_k (1-based) for k = 1..h, stored at index k. */
            if (mode != ORACLE_WT) {
                double *top = sa + h * n;
                if (mode == ORACLE_W) {
                    memcpy(top, x, sizeof(double) * (size_t)n);
                } else {
                    for (int64_t j = 0; j < n; ++j) top[j] = d[j] * sb[h * n + j];
                }
                for (int64_t k = h - 1; k >= 0; --k) {
                    memcpy(sa + k * n, sa + (k + 1) * n, sizeof(double) * (size_t)n);
                    reflect(n, U + k * ldu, tau[k], sa + k * n);
                }
            }
            /* --- backward --- */
            if (mode != ORACLE_WT) {
                /* y = sigma .* sa[0]; H_{k+1} (0-based k) maps sa[k+1] -> sa[k] */
                apply_sign(n, sigma, G);
                for (int64_t k = 0; k < h; ++k)
                    reflect_backward(n, U + k * ldu, tau[k], sa + (k + 1) * n, G, gu_t + k * n);
                /* G is now dL/d(input of W part) */
                if (mode == ORACLE_SYM) {
                    for (int64_t j = 0; j < n; ++j) {
                        gd_t[j] += sb[h * n + j] * G[j];
                        G[j] *= d[j];
                    }
                }
            }
            if (mode != ORACLE_W) {
                /* H_{k+1} maps sb[k] -> sb[k+1]; walk k = h-1 .. 0 */
                for (int64_t k = h - 1; k >= 0; --k)
                    reflect_backward(n, U + k * ldu, tau[k], sb + k * n, G, gu_t + k * n);
                apply_sign(n, sigma, G);
            }
            if (gX) memcpy(gX + b * ldgx, G, sizeof(double) * (size_t)n);
        }
        free(sa);
        free(sb);
        free(G);
    }
    if (!bad) {
        if (gU)
            for (int64_t k = 0; k < h; ++k)
                for (int64_t j = 0; j < n; ++j) {
                    double s = 0.0;
                    for (int t = 0; t < nt; ++t) s += gu_all[(size_t)t * (gu_sz + gd_sz) + (size_t)k * n + j];
                    gU[k * ldu + j] = s;
                }
        if (gd)
            for (int64_t j = 0; j < n; ++j) {
                double s = 0.0;
                for (int t = 0; t < nt; ++t) s += gu_all[(size_t)t * (gu_sz + gd_sz) + gu_sz + j];
                gd[j] = s;
            }
    }
    free(gu_all);
    free(tau);
    return bad ? -1 : 0;
}

/*
 * Fast Mahalanobis distances (§IV-C): out[p] = sum_m d_m [W^T (sigma .* delta)]_m^2,
 * delta = X[ia[p]] - X[ib[p]].
 */
int oracle_mahalanobis(int64_t n, int64_t h, const double *U, int64_t ldu,
                       const signed char *sigma, const double *d, int64_t npairs,
                       const double *X, int64_t ldx, const int64_t *ia, const int64_t *ib,
                       double *out, int nthreads) {
    if (n < 1 || h < 0 || npairs < 0 || ldx < n || ldu < n || !d) return -1;
    if (npairs > 0 && (!X || !ia || !ib || !out)) return -1;
    double *tau = (double *)malloc(sizeof(double) * (size_t)(h > 0 ? h : 1));
    if (!tau) return -1;
    if (oracle_tau(n, h, U, ldu, tau) != 0) { free(tau); return -1; }
    set_threads(nthreads);
    int bad = 0;
#pragma omp parallel
    {
        double *z = (double *)malloc(sizeof(double) * (size_t)n);
        if (!z) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(static)
        for (int64_t p = 0; p < npairs; ++p) {
            if (!z) continue;
            const double *xa = X + ia[p] * ldx, *xb = X + ib[p] * ldx;
            for (int64_t j = 0; j < n; ++j) z[j] = xa[j] - xb[j];
            apply_sign(n, sigma, z);
            chain_WT(n, h, U, ldu, tau, z);
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) s += d[j] * z[j] * z[j];
            out[p] = s;
        }
        free(z);
    }
    free(tau);
    return bad ? -1 : 0;
}
