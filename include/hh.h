/*
 * hh.h -- C ABI of libhh, GB300 (sm_103a) kernels for products of Householder
 * reflectors, after Rusu, "Approximate Eigenvalue Decompositions of Linear
 * Transformations with a Few Householder Reflectors" (arXiv 1811.07624).
 *
 * The transform.  A plan holds h reflector vectors v_1..v_h of length n.
 * Reflector k is H_k = I - 2 u_k u_k^T with u_k = v_k / |v_k| (§II-A, Eq. (2));
 * a zero v_k means H_k = I (the "u_k = 0" reflector of Result 1, §II-B).  The
 * chain is W = H_1 H_2 ... H_h, so H_h acts first in W x.  The plan may carry
 * a +-1 sign vector sigma (the diagonal D of Eq. (1)) and a spectrum d (the
 * s-bar of Eq. (21)).  Per row x of X the library computes
 *
 *   hh_apply      y = sigma .* (W x)                       (Eq. (1))
 *   hh_apply_T    y = W^T (sigma .* x)                     (right factor of Eq. (21))
 *   hh_apply_sym  y = sigma .* W (d .* W^T (sigma .* x))   (Eq. (21))
 *
 * and the gradients of a scalar loss through each of them (hh_backward), and
 * the fast Mahalanobis distance of §IV-C (hh_mahalanobis).  The paper counts
 * 4nh operations per W x (§II-A) and (8h+1)n per S x (§III-A).
 *
 * Conventions shared by every entry point:
 *  - Pointers named X, Y, U, d, sign, gX, gY, gU, gd, ia, ib, out are DEVICE
 *    pointers (memory of the current CUDA device).  Host pointers are rejected
 *    with HH_ERR_INVALID_ARG where the runtime can tell them apart.  There is
 *    no CPU fallback: every step runs in this library's CUDA kernels.
 *  - Vectors are rows: X is batch x n, row b at X + b*ldx elements, ldx >= n.
 *    Reflectors are rows too: v_k at U + k*ldu elements, ldu >= n.
 *  - Element type is the plan's dtype: HH_F32 (float), HH_F64 (double) or
 *    HH_BF16 (bfloat16 storage of U, X and Y; FP32 accumulation; the
 *    normalisation and the compact-WY T factor are kept in FP64).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Apply, backward and distance calls are asynchronous on it:
 *    argument errors are reported synchronously, kernel results are ready
 *    when the stream is.  hh_create and hh_destroy synchronise `stream`.
 *    An F32 apply with 2048 < n <= 4096 and 25 < h <= 100 on a large batch
 *    runs part of its rows on a second stream of the library's, forked from
 *    and joined back to `stream` by events; that stream and its events are
 *    created by the first such call on a device, which should run outside
 *    stream capture.
 *  - In-place (Y == X, same ld) is allowed for the three apply calls.
 *    Other overlaps between inputs and outputs are undefined.
 *  - A plan is read-only after hh_create, so one plan may be used from
 *    several streams or host threads at once.
 *  - The caller owns X, Y and every gradient and output buffer.  The plan
 *    copies U, d and sign; the caller may free them once hh_create returns.
 *  - On failure an entry point returns a non-zero hh_status, writes nothing it
 *    was asked to write (argument errors) and records a message that
 *    hh_last_error() returns on the same host thread.
 */
#ifndef HH_H_
#define HH_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HH_OK = 0,
    HH_ERR_INVALID_ARG = 1, /* bad size, null or host pointer, misuse */
    HH_ERR_UNSUPPORTED = 2, /* valid request this build has no kernel for */
    HH_ERR_NONFINITE = 3,   /* U or d holds NaN/Inf (checked at create) */
    HH_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    HH_ERR_OOM = 5,         /* device allocation failed */
    HH_ERR_TIMEOUT = 6      /* a bounded device-side wait expired */
} hh_status;

typedef enum { HH_F32 = 0, HH_F64 = 1, HH_BF16 = 2 } hh_dtype;

typedef enum { HH_MODE_W = 0, HH_MODE_WT = 1, HH_MODE_SYM = 2 } hh_mode;

/* Kernel family for the apply calls.  FUSED: one pass, each vector read and
 * written once, reflectors applied one after another on CUDA cores (F32, F64).
 * WY: compact-WY regrouping W = I - V T V^T run as tcgen05 GEMMs (BF16).
 * AUTO picks FUSED for F32/F64 and WY for BF16. */
typedef enum { HH_PATH_AUTO = 0, HH_PATH_FUSED = 1, HH_PATH_WY = 2 } hh_path;

typedef struct hh_plan_s *hh_plan_t;

/*
 * Create a plan for the h reflectors in U (device, dtype elements, reflector k
 * at U + k*ldu) and the optional spectrum d (device, n elements of dtype, or
 * NULL: then hh_apply_sym and hh_mahalanobis fail with HH_ERR_INVALID_ARG).
 * Reflector vectors need not be unit length; they are normalised in FP64
 * (tau_k = 2 / v_k^T v_k, §II-A Eq. (2)).  Requires n >= 1, h >= 0.
 * The paper's regime is h < n/2 (§II-A); larger h is accepted.
 * Returns HH_ERR_NONFINITE if U or d holds a NaN or Inf.
 * Same as hh_create_ex(out, n, h, U, ldu, d, NULL, dtype, HH_PATH_AUTO, NULL).
 */
hh_status hh_create(hh_plan_t *out, int64_t n, int64_t h, const void *U, int64_t ldu,
                    const void *d, hh_dtype dtype);

/*
 * hh_create with a sign vector and an explicit path.  sign: device int8
 * vector of n entries, each +1 or -1, or NULL for all +1 (the diagonal D of
 * Eq. (1)); any other value gives HH_ERR_INVALID_ARG.  The plan's device
 * memory is allocated with cudaMalloc here and freed by hh_destroy.
 */
hh_status hh_create_ex(hh_plan_t *out, int64_t n, int64_t h, const void *U, int64_t ldu,
                       const void *d, const int8_t *sign, hh_dtype dtype, hh_path path,
                       void *stream);

/* Release a plan (NULL is a no-op).  Synchronises the device first. */
hh_status hh_destroy(hh_plan_t plan);

/*
 * Synchronise `stream` and report device-side failures of this plan's earlier
 * calls on it: HH_ERR_TIMEOUT if a kernel gave up a bounded wait (its output
 * is then incomplete), HH_ERR_INVALID_ARG for a pair index out of range
 * (hh_mahalanobis), HH_ERR_NONFINITE for a NaN or Inf given to hh_update,
 * HH_OK otherwise.  Clears the plan's status word.
 */
hh_status hh_sync(hh_plan_t plan, void *stream);

/*
 * New reflector values for an existing F32 or F64 plan (§II-A: tau_k, the
 * stored copies and the Gram band are recomputed in FP64 as at create): U is h
 * rows of n device elements of the plan's dtype at U + k*ldu; d (n elements)
 * must be given exactly when the plan was created with a spectrum, else NULL.
 * The sign is kept.  Stream-ordered on `stream` with no allocation and no
 * host synchronisation, so later calls on the same stream see the new values
 * (for training loops: one plan, updated after each optimiser step).  A NaN or
 * Inf in U or d is reported by the next hh_sync as HH_ERR_NONFINITE.  BF16
 * (compact-WY) plans: HH_ERR_UNSUPPORTED; create a new plan.
 */
hh_status hh_update(hh_plan_t plan, const void *U, int64_t ldu, const void *d, void *stream);

/* Shape and kernel family of a plan.  Any output pointer may be NULL. */
hh_status hh_plan_info(hh_plan_t plan, int64_t *n, int64_t *h, hh_dtype *dtype,
                       hh_path *path);

/*
 * Zero prefixes of the reflectors (§II-D, the remark after Result 3: the
 * reflectors of a partial QR factorization have k - 1 leading zeros, so H_k
 * costs 4(n - k + 1) operations instead of 4n).  At create, and at every
 * hh_update, the plan records the first non-zero column of each v_k; when the
 * zero prefixes hold at least 1/16 of U's entries, F32 applies with n <= 8192
 * on 16-byte aligned rows skip, per round of reflectors, the column blocks
 * that lie before every reflector's first non-zero (exact: the skipped terms
 * are zeros).  mode 1 turns the skipping on, 0 off, -1 back to that automatic
 * choice, -2 leaves it as it is; *enabled (may be NULL) receives the setting
 * now in force.  Other modes: HH_ERR_INVALID_ARG.  Host-side
 * only, no device work; F64 and BF16 plans accept the call and never skip.
 */
hh_status hh_plan_skip_prefix(hh_plan_t plan, int mode, int *enabled);

/*
 * Y = sigma .* (W X) row by row (§II-A, Eq. (1)).  X: batch x n, row stride
 * ldx; Y: batch x n, row stride ldy.  batch == 0 is a no-op.
 */
hh_status hh_apply(hh_plan_t plan, const void *X, int64_t ldx, void *Y, int64_t ldy,
                   int64_t batch, void *stream);

/* Y = W^T (sigma .* X) row by row (the right-hand factor of Eq. (21)). */
hh_status hh_apply_T(hh_plan_t plan, const void *X, int64_t ldx, void *Y, int64_t ldy,
                     int64_t batch, void *stream);

/* Y = sigma .* W (d .* W^T (sigma .* X)) row by row (§III-A, Eq. (21)):
 * the symmetric matrix D W diag(d) W^T D applied in one pass. */
hh_status hh_apply_sym(hh_plan_t plan, const void *X, int64_t ldx, void *Y, int64_t ldy,
                       int64_t batch, void *stream);

/*
 * Gradients of a scalar loss L through hh_apply (mode HH_MODE_W), hh_apply_T
 * (HH_MODE_WT) or hh_apply_sym (HH_MODE_SYM), given gY = dL/dY.
 *   saved: the forward OUTPUT Y for modes W and WT (the intermediate vectors
 *          are recomputed from it by the involution H_k H_k = I, §II-A, so
 *          none are stored); the forward INPUT X for mode SYM.
 *   gX:    dL/dX (batch x n, ldgx), or NULL to skip.
 *   gU:    dL/dv_k for the reflector vectors as passed to hh_create (h rows of
 *          n, row stride n), summed over the batch; or NULL to skip.
 *   gd:    dL/dd (n), summed over the batch, mode SYM only; or NULL.
 * F32 and F64 plans only.  Needs device scratch, allocated per call with
 * cudaMallocAsync on `stream`.
 */
hh_status hh_backward(hh_plan_t plan, hh_mode mode, const void *saved, int64_t lds,
                      const void *gY, int64_t ldgy, void *gX, int64_t ldgx, void *gU,
                      void *gd, int64_t batch, void *stream);

/*
 * hh_apply_sym that also writes p = W^T (sigma .* x) (batch x n, leading
 * dimension ldp), the state between the two halves of Eq. (21), for
 * hh_backward_sym_py.  Where the column-split kernels run (F32, aligned rows,
 * 512 < n <= 1024 with h <= 50, or 2048 < n <= 4096 with h <= 25) p is stored
 * inside the same pass; elsewhere a W^T pass writes it first, so Y may alias
 * X.  P may alias neither X nor Y.  F32 and F64 plans.
 */
hh_status hh_apply_sym_p(hh_plan_t plan, const void *X, int64_t ldx, void *Y, int64_t ldy,
                         void *P, int64_t ldp, int64_t batch, void *stream);

/*
 * hh_backward for mode SYM from p = W^T (sigma .* x) and y = S_bar x as
 * hh_apply_sym_p returned them (Eq. (21)); the input x is not needed.  The
 * adjoint's states are read instead of recomputed (on F32 with aligned rows,
 * n and h multiples of 4 and h <= 64; otherwise x = sigma .* (W p) is formed
 * first, W being orthogonal).  Same gradients and errors as
 * hh_backward(HH_MODE_SYM, x, ...); p and y that are not this plan's for
 * one x give wrong gradients, not an error.
 */
hh_status hh_backward_sym_py(hh_plan_t plan, const void *P, int64_t ldp, const void *y,
                             int64_t ldy, const void *gY, int64_t ldgy, void *gX, int64_t ldgx,
                             void *gU, void *gd, int64_t batch, void *stream);

/*
 * hh_backward for mode SYM given the forward output as well: x (the forward
 * input, batch x n, ldx) and y = S_bar x (batch x n, ldy) as hh_apply_sym of
 * this plan returned it for the same rows (Eq. (21)).  The state
 * q = W (d .* W^T (sigma .* x)) that the adjoint walks from is sigma .* y, so
 * it is read instead of recomputed.  Same gradients, results and errors as
 * hh_backward(HH_MODE_SYM, x, ...); a y that is not this plan's output for x
 * gives wrong gradients, not an error.  F32 and F64 plans (F64 and rows that
 * are not 16-byte aligned take the hh_backward path and do not read y).
 */
hh_status hh_backward_sym_y(hh_plan_t plan, const void *x, int64_t ldx, const void *y,
                            int64_t ldy, const void *gY, int64_t ldgy, void *gX, int64_t ldgx,
                            void *gU, void *gd, int64_t batch, void *stream);

/*
 * hh_backward that allocates nothing.  The paper has no counterpart: this
 * entry point is for callers that cannot let a library allocate device memory
 * on its own schedule, such as code running inside a host (a framework, a
 * serving process, a plugin) that owns all of the device's memory and does
 * not allow cudaMalloc behind its back, or a latency-bound training loop that
 * must not block or fail with out-of-memory part-way through a step.
 *
 * Same arguments, results and errors as hh_backward, but its scratch is a
 * fixed 32 MiB array that is part of the library's device image: every device
 * that loads the library holds it until the process exits.  No cudaMalloc,
 * cudaMallocAsync or cudaFree is called.  One CTA's partial sums take
 * (h + 1) * C * s + 8 h bytes (s the element size, C the kernel's column tile:
 * n rounded up to a power of two, at least 128 for F32 / 64 for F64); the call
 * uses as many CTAs as fit and returns HH_ERR_INVALID_ARG when one does not
 * (for example F32 with n = 4096 and h > 2046).
 *
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress); make that first call before any
 * stream capture.  All calls share the one array and the kernels initialise
 * what they read, but calls whose work overlaps on the GPU (other streams,
 * other host threads) race on it and give wrong gradients: serialise them.
 */
hh_status hh_backward_noalloc(hh_plan_t plan, hh_mode mode, const void *saved, int64_t lds,
                              const void *gY, int64_t ldgy, void *gX, int64_t ldgx, void *gU,
                              void *gd, int64_t batch, void *stream);

/*
 * Fast Mahalanobis distances (§IV-C): for p < npairs,
 *   out[p] = (x_a - x_b)^T S (x_a - x_b) = sum_m d_m [W^T (sigma .* (x_a - x_b))]_m^2
 * with x_a = row ia[p] and x_b = row ib[p] of X (int64 device indices, each
 * in [0, nrows)).  out: npairs elements of the plan's dtype.  Needs d.
 * F32 and F64 plans, n <= 4096.  An index outside [0, nrows) gives NaN for
 * that pair and makes hh_sync report HH_ERR_INVALID_ARG.
 */
hh_status hh_mahalanobis(hh_plan_t plan, const void *X, int64_t ldx, int64_t nrows,
                         const int64_t *ia, const int64_t *ib, int64_t npairs, void *out,
                         void *stream);

/*
 * Gradients of L = sum_p gout[p] * out[p] for the distances of hh_mahalanobis
 * (a metric-learning loss, §IV-C): gU (h rows of n, with respect to the
 * reflector vectors as given) and gd (n), each summed over the pairs, or NULL
 * to skip.  gout: npairs device elements of the plan's dtype (dL/d out[p]).
 * No gradient for X.  An index outside [0, nrows) contributes nothing and
 * makes hh_sync report HH_ERR_INVALID_ARG.  Scratch is allocated per call
 * with cudaMallocAsync on `stream`.
 */
hh_status hh_mahalanobis_backward(hh_plan_t plan, const void *X, int64_t ldx, int64_t nrows,
                                  const int64_t *ia, const int64_t *ib, int64_t npairs,
                                  const void *gout, void *gU, void *gd, void *stream);

/*
 * Batched persistent launch.  Many independent transforms (plans of uneven n
 * and h, each with its own batch of vectors) applied in ONE persistent kernel
 * launch, replayed from a CUDA graph.  The paper applies one transform at a
 * time (§II-A); running many at once is this library's own addition, and so is
 * the tile-shape autotuner below.
 *
 * hh_batch_create: plans[i] (count entries) must be F32 FUSED-path plans of
 * the current device with n % 4 == 0 and n <= 4096 (else HH_ERR_UNSUPPORTED);
 * batch[i] >= 0 is the number of vectors of transform i.  The batch refers to
 * the plans, which must outlive it.  Tile shapes come from the autotuner's
 * table (hh_tune / hh_tune_load / hh_tune_set) as it stands at create time.
 * Allocates the work list and task table on the device; synchronous.
 */
typedef struct hh_batch_s *hh_batch_t;
hh_status hh_batch_create(hh_batch_t *out, int count, const hh_plan_t *plans,
                          const int64_t *batch);

/*
 * Apply every transform of the batch in `mode` (W, WT or SYM as hh_apply,
 * hh_apply_T, hh_apply_sym): Y[i] = op_i(X[i]) for batch[i] rows.  X, Y: host
 * arrays of count device pointers (16-byte aligned, rows of n floats);
 * ldx, ldy: host arrays of count row strides (multiples of 4, >= n), or NULL
 * for n.  X[i] == Y[i] is allowed with equal strides.  The first call per mode
 * captures the launches (one per cluster size of the resident shape, then a
 * counter reset and the staged-shape kernel, each only where it has work) in
 * a CUDA graph; every call replays it on `stream`.  When the pointers or strides differ from the
 * previous call, the task table is first copied to the device on `stream`.
 * Stream-ordered; calls on different streams must not overlap on the GPU
 * (they share the work counter).
 */
hh_status hh_batch_apply(hh_batch_t batch, hh_mode mode, const void *const *X, const int64_t *ldx,
                         void *const *Y, const int64_t *ldy, void *stream);

/* Report (and clear) the batch's device status word, as hh_sync.  Synchronises
 * `stream`. */
hh_status hh_batch_sync(hh_batch_t batch, void *stream);

/* Work items of all the batch's launches, CTAs of its largest launch, and the
 * tile shape of each transform (count ints, or NULL). */
hh_status hh_batch_info(hh_batch_t batch, int64_t *nitems, int *grid, int *shapes);

/* Synchronises the device, then frees the batch.  NULL is a no-op. */
hh_status hh_batch_destroy(hh_batch_t batch);

/* Tile shapes of the batched kernel, 0 .. hh_batch_num_shapes()-1: G threads
 * per row group, NG granules of 4 floats and RT rows per thread, rows per tile,
 * and the largest n the shape covers (G * NG * 4 for a staged shape).
 *
 * Staged shapes stream every tile's rows through shared memory and read the
 * reflectors from L2 once per tile, with work items taken from a shared
 * counter.  The resident shape (hh_batch_shape_limits reports max_cluster > 0)
 * splits each vector's columns over a cluster of ceil(n / (G * NG * 4)) CTAs,
 * up to max_cluster, keeps each CTA's columns of all h <= max_h reflectors of
 * one transform in shared memory, and runs a static, transform-ordered
 * schedule built at hh_batch_create: one launch per cluster size, each
 * cluster loading a transform's reflectors once.  The launches of one batch
 * and mode are captured in the same graph.  Any output pointer of either
 * kind of shape is a plain pointer argument (NULL skips it). */
int hh_batch_num_shapes(void);
hh_status hh_batch_shape(int shape, int *G, int *NG, int *RT, int *rows_per_tile, int *cover);
/* max_h: the largest h the shape takes (-1: no limit); max_cluster: CTAs per
 * cluster of the resident shape (0 for a staged shape).  HH_ERR_INVALID_ARG
 * for a shape outside [0, hh_batch_num_shapes()). */
hh_status hh_batch_shape_limits(int shape, int *max_h, int *max_cluster);

/*
 * Autotuner.  hh_tune times, for every (n, h) in ns x hs, each tile shape that
 * covers n on `rows` synthetic vectors (a batch of one transform, mode W,
 * CUDA events on `stream`, 2 warm-up and 5 timed launches) and records the
 * fastest in a process-wide table.  Needs n % 4 == 0, 4 <= n <= 4096.
 * Synchronises `stream`.  hh_tune_get returns the shape hh_batch_create would
 * use for (n, h): the table entry, else the entry of the nearest h for the same
 * n, else a fixed rule; and the measured milliseconds per shape (hh_batch_num_
 * shapes() floats, NaN where not measured), or NULL.  hh_tune_set pins an
 * entry (HH_ERR_INVALID_ARG where the shape does not take (n, h)).  hh_tune_save / hh_tune_load write / merge the table as text lines
 * "n h shape".  hh_tune_clear empties it.  Host-only except hh_tune.
 */
hh_status hh_tune(const int64_t *ns, int nn, const int64_t *hs, int nh, int64_t rows,
                  void *stream);
hh_status hh_tune_get(int64_t n, int64_t h, int *shape, float *ms);
hh_status hh_tune_set(int64_t n, int64_t h, int shape);
hh_status hh_tune_save(const char *path);
hh_status hh_tune_load(const char *path);
hh_status hh_tune_clear(void);

/*
 * Test hooks for failure handling; the paper has no counterpart.
 *
 * hh_debug_fail_alloc(k): the k-th device allocation the library makes from
 * now on (plans, batches, backward scratch) fails as if the device were out of
 * memory, so that call returns HH_ERR_OOM having freed what it held; k = 0
 * switches the hook off.  Host only; process-wide.
 *
 * hh_debug_wait_timeout(cycles, stream): runs the bounded mbarrier wait that
 * every pipelined kernel uses on a barrier nothing arrives on, with a limit
 * of `cycles` clock cycles (1 .. 4e9), and synchronises `stream`.  Returns
 * HH_ERR_TIMEOUT, the expected outcome: the wait gave up and the kernel ended
 * normally, leaving the context usable.
 */
hh_status hh_debug_fail_alloc(int k);
hh_status hh_debug_wait_timeout(int64_t cycles, void *stream);

/* Message for the last failed call on this host thread ("" if none). */
const char *hh_last_error(void);

/* Library version string. */
const char *hh_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HH_H_ */
