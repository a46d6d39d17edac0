/*
 * lmreg.h -- C ABI of the GB300 (sm_103a) factored Levenberg-Marquardt
 * registration library.
 *
 * The library minimises an LNCC image-similarity loss over a dense 3-D
 * displacement field u, L(u) = L_sim(F, M o (Id + u)) (Section 1, Eq. 1 of
 * Jena, Chaudhari, Gee, "Factored Levenberg-Marquardt for Diffeomorphic Image
 * Registration"), with the per-voxel rank-1 damped step of Eq. tile1
 * (Appendix A), the compositive update of Eq. compositive (Section 2.1), the
 * damping rule of Eq. lambda-update and the rejection rule of Eq. rejection
 * (Section 3.4), on a coarse-to-fine pyramid (Section 2.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Volumes are [D][H][W] (z, y, x) with x fastest, contiguous.
 *  - A displacement field is float32 [3][D][H][W]: component 0 along x (W),
 *    1 along y (H), 2 along z (D), in voxel units; u(p) names the sample
 *    point p + u(p) in voxel index coordinates.
 *  - All data pointers are DEVICE pointers unless a parameter says "host".
 *    The caller owns every pointer it passes; the library never frees them
 *    and keeps no pointer past the call unless stated (lm_init keeps the
 *    fixed/moving image pointers for the context's lifetime).
 *  - Calls are ordered on the CUDA stream given to lm_init.  Entry points
 *    that fill a host struct synchronise that stream before returning.
 *  - Every function returns LM_OK (0) or a negative LM_E* code; nothing
 *    throws across the ABI.  lm_strerror() names a code, lm_last_error()
 *    describes the last failure on the calling thread.
 *  - The loss reported everywhere is r = 1 - LNCC in [0, 1] (the residual of
 *    the squared-loss form (1 - LNCC)^2 of Section 2.2).
 */
#ifndef LMREG_H
#define LMREG_H

#include <stddef.h>

#if defined(__GNUC__)
#define LM_API __attribute__((visibility("default")))
#else
#define LM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define LM_OK            0
#define LM_EINVAL       -1  /* bad argument: null pointer, shape, parameter */
#define LM_ENOMEM       -2  /* device or host allocation failed */
#define LM_ECUDA        -3  /* a CUDA runtime call failed */
#define LM_ENONFINITE   -4  /* a loss or gradient reduction was not finite */
#define LM_ETIMEOUT     -5  /* a bounded device wait ran out */
#define LM_EUNSUPPORTED -6  /* valid request this build does not handle */
#define LM_ESTATE       -7  /* call out of order (e.g. lm_step before reset) */
#define LM_EBOUNDS      -8  /* debug-bounds build: a kernel wrote outside a
                               buffer (lm_debug_check) */
/* LM_ETIMEOUT: the gradient-smoothing kernel waits on its TMA tiles with a
 * bound (2^20 polls or 0.5 s); a wait that runs out voids that evaluation
 * and the call returns LM_ETIMEOUT with the context still usable (the state
 * keeps its last accepted field).
 *
 * Host-side fault injection (read when a context is created; tests only):
 *   LM_FAULT_ALLOC=n    the context's n-th device allocation fails as if
 *                       cudaMalloc had (the create call returns LM_ENOMEM
 *                       and frees what it had allocated);
 *   LM_FAULT_TIMEOUT=1  every evaluation's smoothing kernel first waits on a
 *                       barrier that no copy completes (nothing is in flight),
 *                       so that the bounded wait runs out: evaluations return
 *                       LM_ETIMEOUT.  Neither faults nor hangs the device. */

/* ---- similarity and method (lm_params.loss, lm_params.method) ---------- */
#define LM_LOSS_LNCC     0  /* r = 1 - LNCC (Section 2.2)                    */
#define LM_LOSS_MSE      1  /* r = V^-1 sum (F - M(p + u))^2 (Section 2.2)   */
#define LM_LOSS_MI       2  /* r = log2 B - MI, Parzen MI (Section 2.2)      */
#define LM_METHOD_LM     0  /* factored LM, Eq. tile1 / Eq. tilen            */
#define LM_METHOD_DEMONS 1  /* Demons as per-voxel LM on MSE, Eq. demons     */

/* ---- image storage types ----------------------------------------------- */
#define LM_F32  0  /* float32 images */
#define LM_BF16 1  /* bfloat16 images, sampled and accumulated in float32 */

/* An image volume.  At most (2^31 - 1) / 3 voxels (715,827,882, e.g.
 * 894^3): the kernels index the 3-component fields with 32-bit offsets. */
typedef struct {
    int D, H, W;        /* depth (z), height (y), width (x); each >= 1 */
    int dtype;          /* LM_F32 or LM_BF16 */
    const void *data;   /* device pointer to D*H*W elements, caller-owned */
} lm_volume;

/* Optimiser and loss parameters.  lm_default_params() fills the paper's
 * defaults: lambda0 = 0.006, mu+ = 1.5, mu- = 0.975 (Section 3), rejection
 * off with tau = 1 and 10 retries (Section 3.4). */
typedef struct {
    int    win;         /* LNCC box side k: odd, 3..9.                 [5] */
    float  eps_nr;      /* LNCC numerator stabiliser, >= 0.         [1e-5] */
    float  eps_dr;      /* LNCC denominator stabiliser, > 0.        [1e-5] */
    float  sigma_grad;  /* Gaussian sigma on the gradient, 0..2.       [1] */
    float  sigma_warp;  /* Gaussian sigma on the composed warp, 0..2.  [0] */
    float  step;        /* epsilon of Eq. compositive, voxels, > 0.  [0.5] */
    double lambda0;     /* initial damping, > 0.                   [0.006] */
    double mu_inc;      /* damping increase factor mu+, > 1.         [1.5] */
    double mu_dec;      /* damping decrease factor mu-, in (0, 1). [0.975] */
    double lambda_max;  /* damping cap, >= lambda0, may be +inf.    [+inf] */
    int    reject;      /* 1: Eq. rejection on.                         [0] */
    double tau;         /* rejection tolerance ratio, >= 0.          [1.0] */
    int    max_retries; /* retries after a rejection, 0..32.          [10] */
    int    tile;        /* curvature tile side k, 1..16 (Eq. tilen):    [1]
                           1 = the pointwise step of Eq. tile1; k > 1
                           pools ghat ghat^T as its mean over the
                           non-overlapping k x k x k tiles of the grid
                           (the last tile of an axis cut at the volume
                           edge) and solves (H_tile + lambda I) du =
                           -r ghat per voxel. */
    int    loss;        /* LM_LOSS_LNCC, LM_LOSS_MSE or LM_LOSS_MI. [LNCC]
                           MI: both images are binned over the joint range
                           of F, M and 0 into B = bins bins with cubic
                           B-spline Parzen windows; MI in bits; the
                           residual is r = log2 B - MI (the squared-loss
                           form (log2 B - MI)^2 of Section 2.2). */
    int    method;      /* LM_METHOD_LM or LM_METHOD_DEMONS.           [LM]
                           Demons (Section 2.3) needs LM_LOSS_MSE, tile 1
                           and reject 0.  Each iteration takes, per voxel,
                           du = r n / (|n|^2 + alpha^2 r^2) with the voxel's
                           residual r = F - M(p + u) and n the gradient of
                           M at p + u (Eq. demons), smooths du with the
                           sigma_grad Gaussian, scales it by step and
                           composes it (Eq. compositive; sigma_warp
                           smoothing as for LM).  Every step is kept; the
                           damping fields are unused; the reported loss is
                           the MSE and gmax the largest smoothed update. */
    float  alpha;       /* Demons damping weight, lambda_x = alpha^2 r^2,
                           > 0.                                          [1] */
    int    bins;        /* MI histogram bins B per image, 4..64.       [32] */
} lm_params;

/* Coarse-to-fine schedule: levels run in order, factor[l] in {1, 2, 4}
 * (image size divided by factor[l], rounded down, at least 1),
 * iters[l] >= 0 LM iterations at that level. */
#define LM_MAX_LEVELS 4
typedef struct {
    int nlevels;
    int factor[LM_MAX_LEVELS];
    int iters[LM_MAX_LEVELS];
} lm_schedule;

/* Outcome of one LM iteration. */
typedef struct {
    double loss;        /* loss of the field after the iteration */
    double loss_first;  /* loss of the first trial of the iteration */
    double lambda;      /* damping after the iteration */
    float  gmax;        /* max_p |g(p)| of the field after the iteration */
    int    accepted;    /* 1 = a trial was accepted, 0 = discarded */
    int    retries;     /* rejected trials before the outcome */
    int    evals;       /* loss evaluations spent (retries + 1) */
    int    stopped;     /* 1 = the pair has reached its target loss
                           (lm_batch_set_targets) and no longer iterates */
} lm_step_info;

/* Optimiser scalars of a context (for inspection, teacher forcing and
 * checkpoints).  has_prev = 0 means L_prev is not defined yet. */
typedef struct {
    double loss;        /* L_t */
    double loss_prev;   /* L_{t-1} */
    double lambda;
    float  gmax;
    int    has_prev;
    int    iter;        /* iterations run since lm_reset */
    int    evals;       /* loss evaluations since lm_reset */
    long long kernel_launches; /* kernels this context enqueued since
                                  lm_reset (read-only for lm_set_state) */
} lm_state;

/* One record per finished LM iteration, written on the device by the
 * decision that ends the iteration (Eq. lambda-update, Eq. rejection). */
typedef struct {
    double loss;        /* loss of the field after the iteration */
    double lambda;      /* damping after the iteration */
    float  gmax;        /* max_p |g(p)| of the field after the iteration */
    int    accepted;    /* 1 = a trial was accepted, 0 = discarded */
    int    retries;     /* rejected trials before the outcome */
} lm_log_entry;

/* Records the device keeps per context (a ring: the most recent ones). */
#define LM_LOG_CAP 8192

/* Summary of a registration run. */
typedef struct {
    int    nlevels;
    int    level_dims[LM_MAX_LEVELS][3];    /* D, H, W of each level */
    int    level_iters[LM_MAX_LEVELS];
    int    level_evals[LM_MAX_LEVELS];
    int    level_accepted[LM_MAX_LEVELS];
    double level_loss[LM_MAX_LEVELS];       /* loss at the end of the level */
    double final_loss;
    long long voxel_evals;                  /* sum over levels of V * evals */
    double wall_ms;                         /* host wall time of the call */
} lm_report;

typedef struct lm_ctx lm_ctx;

/* Fill *p with the defaults listed above.  LM_EINVAL if p is NULL. */
LM_API int lm_default_params(lm_params *p);

/* Create a context for one fixed/moving pair of equal shape and dtype: the
 * registration problem of Section 1, Eq. 1 (minimise L_sim(F, M o (Id + u))
 * over the displacement u), with the LM parameters of Section 3 (lambda0,
 * mu+, mu-) and the rejection parameters of Section 3.4 in p.
 * fixed, moving: image descriptors; their device data must stay valid and
 *   unchanged for the context's lifetime.
 * p: parameters (copied); NULL = defaults.
 * cuda_stream: cudaStream_t to order all work on (NULL = default stream).
 * The context allocates its own device scratch (76 bytes per voxel, 100
 * with warp smoothing, plus pyramid levels on first lm_register).  LM_EINVAL on bad shapes or
 * parameters, LM_ENOMEM / LM_ECUDA on allocation failure. */
LM_API int lm_init(lm_ctx **ctx, const lm_volume *fixed, const lm_volume *moving,
            const lm_params *p, void *cuda_stream);

/* Release the context and its scratch.  NULL is ignored. */
LM_API void lm_destroy(lm_ctx *ctx);

/* Evaluate the loss and its smoothed gradient at u without touching the
 * optimiser state: M resampled at Id + u (Section 2.1), the residual r of
 * the squared-loss form of Section 2.2 and its gradient with respect to u,
 * smoothed by the sigma_grad Gaussian (the gradient g that Eq. tile1 takes;
 * Section 3 describes the FireANTs-style smoothed gradient).  This is what
 * every LM iteration evaluates for its trial.  u: device [3][D][H][W].  loss (host, may be
 * NULL), g_out (device [3][D][H][W], may be NULL), gmax (host, may be NULL).
 * Synchronises the stream.  LM_ENONFINITE if the loss is not finite. */
LM_API int lm_eval(lm_ctx *ctx, const float *u, double *loss, float *g_out,
            float *gmax);

/* Start an LM run from the field u (device, in/out for later lm_step
 * calls): evaluates L_0 and g_0 at u, sets lambda = lambda0 (Section 3) and
 * clears the loss history that Eq. lambda-update and Eq. rejection compare
 * against.  Asynchronous. */
LM_API int lm_reset(lm_ctx *ctx, float *u);

/* One LM iteration (Section 2.2 / 3.3) on the field u passed to the last
 * lm_reset: the trial u* = v + u o (Id + v) with v = step * du from
 * Eq. tile1 (Eq. tilen for tile > 1; for Demons v = step * the smoothed
 * update of Eq. demons), its loss, and the damping / rejection decision
 * (Demons keeps every step).  On return u holds u_{t+1}.  info (host, may be NULL): filled after a stream
 * synchronisation; NULL keeps the call asynchronous.  LM_ESTATE if u is not
 * the pointer given to lm_reset. */
LM_API int lm_step(lm_ctx *ctx, float *u, lm_step_info *info);

/* n LM iterations, each exactly the iteration of lm_step (Eq. tile1 or
 * Eq. tilen, Eq. compositive, Eq. lambda-update and Eq. rejection, Sections
 * 2.1-2.2 and 3.4), replayed from a captured CUDA graph; info of the last
 * iteration (host, may be NULL).  u as for lm_step.  Without rejection
 * (p.reject = 0 or max_retries = 0) the call is asynchronous when info is
 * NULL.  With rejection each replay runs one attempt, a retry where the
 * last trial was rejected, and the call synchronises to replay until all
 * n iterations are done. */
LM_API int lm_iterate(lm_ctx *ctx, float *u, int n, lm_step_info *info);

/* Read / overwrite the optimiser scalars (synchronising).  lm_set_state
 * keeps the context's field and gradient, replacing only the scalars. */
LM_API int lm_get_state(lm_ctx *ctx, lm_state *out);
LM_API int lm_set_state(lm_ctx *ctx, const lm_state *in);

/* The context's iteration log since its last lm_reset, oldest first
 * (synchronising).  With out NULL, *n receives the number of records
 * available (at most LM_LOG_CAP); otherwise out (host, caller-owned) holds
 * cap records and receives the most recent min(cap, available) of them,
 * their number in *n.  After lm_register the log is that of the finest
 * level.  LM_EINVAL on a NULL ctx or n, or a negative cap. */
LM_API int lm_get_log(lm_ctx *ctx, lm_log_entry *out, int cap, int *n);

/* Whole coarse-to-fine registration (Section 2.1 pyramid).  u (device,
 * full resolution [3][D][H][W]): in = initial field, out = result.  At each
 * level F and M are Gaussian-blurred (sigma = factor/2) and resampled, the
 * field is carried over with values scaled by the factor ratio, and lambda
 * and the loss history restart.  rep (host, may be NULL) receives a
 * summary.  Synchronises the stream. */
LM_API int lm_register(lm_ctx *ctx, const lm_schedule *s, float *u, lm_report *rep);

/* Checkpoint: the optimiser scalars and the context's gradient of the
 * current field.  lm_state_save with buf NULL writes the needed size to
 * *nbytes; otherwise buf (host) must hold *nbytes bytes.  lm_state_load
 * restores a checkpoint taken from a context of the same shape; the field
 * itself is the caller's u, which must be passed to lm_reset first. */
LM_API int lm_state_save(lm_ctx *ctx, void *buf, size_t *nbytes);
LM_API int lm_state_load(lm_ctx *ctx, const void *buf, size_t nbytes);

/* Measurement aid (the paper times whole steps, Section 3.5; this splits
 * one iteration into its two passes): time the two passes separately.  With
 * the state of the last lm_reset / lm_step on u, launches the trial kernels
 * (pass 2: Eq. tile1 or Eq. tilen + Eq. compositive) n times, then the
 * evaluation kernels (pass 1: resampling, the loss and its gradient,
 * smoothing) n times, each run
 * bracketed by CUDA events on the context's stream, and returns the mean
 * milliseconds per launch in *ms_step and *ms_eval (host).  The optimiser
 * state is not changed.  Synchronises the stream. */
LM_API int lm_time_passes(lm_ctx *ctx, float *u, int n, double *ms_eval,
                          double *ms_step);

/* ---- batches of pairs ------------------------------------------------- */
/* A batch registers npairs independent pairs (shapes may differ, one dtype)
 * with the same parameters.  Every pass of an iteration is one kernel launch
 * over the work of all pairs (CTAs are shared among the pairs in proportion
 * to their voxels), an iteration is one replay of a captured CUDA graph,
 * and each pair keeps its own damping, loss history and rejection state on
 * the device.  Arrays below have npairs entries. */
typedef struct lm_batch lm_batch;

/* fixed[i], moving[i]: image descriptors as for lm_init (data kept for the
 * batch's lifetime).  LM_EINVAL on bad shapes, mixed dtypes or parameters. */
LM_API int lm_batch_init(lm_batch **b, int npairs, const lm_volume *fixed,
                         const lm_volume *moving, const lm_params *p,
                         void *cuda_stream);
LM_API void lm_batch_destroy(lm_batch *b);
/* Loss (host doubles) and gmax (host floats, may be NULL) of each pair at
 * u[i] (device fields); g_out (array of device pointers, may be NULL)
 * receives the smoothed gradients.  Synchronises. */
LM_API int lm_batch_eval(lm_batch *b, const float *const *u,
                         float *const *g_out, double *loss, float *gmax);
/* As lm_reset for every pair (u[i]: device fields, in/out). */
LM_API int lm_batch_reset(lm_batch *b, float *const *u);
/* n LM iterations of every pair (u as given to lm_batch_reset); infos
 * (host, npairs entries, may be NULL) receive each pair's last outcome.
 * Synchronisation as for lm_iterate. */
LM_API int lm_batch_iterate(lm_batch *b, float *const *u, int n,
                            lm_step_info *infos);
/* Autotuner of the evaluation's tile shape and work split (the paper has
 * no counterpart: it serves batches of many pairs of uneven sizes and
 * volumes of any shape).  The LNCC moment kernel has two output tiles per
 * CTA (LM_E1_TILE_32X16: 256 threads, two CTAs per SM; LM_E1_TILE_32X32:
 * 512 threads, one per SM, k <= 7), and the evaluation kernels run a fixed
 * number of CTA waves split among the pairs in proportion to their voxels.
 * This call times reps evaluations at u (device fields, as for
 * lm_batch_eval) for every candidate (tile; E1 waves 1, 2, 4, 8; E2 waves
 * 2, 3, 4, 8, 16 CTAs per SM in total; at least 8 or 1 z slices per
 * z-streaming CTA), then reps trial-field passes for 512, 1024, 2048 or
 * 4096 step-kernel blocks per pair, and keeps the fastest for all later
 * calls (the captured iteration graph is rebuilt).  The trial passes write
 * only the trial slot and the resampling scratch, which the next iteration
 * recomputes, so the optimiser state is unchanged.  lm_register tunes each
 * coarse level's context this way when it first uses it.  Tile and waves change
 * the timing only: the loss is an exact integer sum and every gradient sum
 * has the same order under every choice.  e1_tile, e1_waves, e2_waves,
 * ms_best (host, may be NULL) receive the choice and its time per
 * evaluation.  Synchronises.  LM_EINVAL on NULL b / u or reps < 1. */
#define LM_E1_TILE_32X16 0
#define LM_E1_TILE_32X32 1
LM_API int lm_batch_autotune(lm_batch *b, float *const *u, int reps,
                             int *e1_tile, int *e1_waves, int *e2_waves,
                             double *ms_best);
/* The same for a single-pair context, at its field u (device). */
LM_API int lm_autotune(lm_ctx *ctx, const float *u, int reps, int *e1_tile,
                       int *e1_waves, int *e2_waves, double *ms_best);

/* Carry a displacement field between pyramid levels (Section 2.1), as
 * lm_register does between its levels: the level-b field at voxel p is the
 * level-a field read trilinearly (clamped at the border) at the level-a
 * coordinate of p's centre, (fb p + (fb - 1)/2 - (fa - 1)/2) / fa, times
 * fa / fb (voxel units scale with the level).  src: device [3][Da][Ha][Wa]
 * of a level with factor fa; dst: device [3][Db][Hb][Wb] of factor fb
 * (written).  Asynchronous on cuda_stream.  LM_EINVAL on NULL pointers or
 * non-positive sizes or factors. */
LM_API int lm_field_resample(const float *src, int Da, int Ha, int Wa, int fa,
                             float *dst, int Db, int Hb, int Wb, int fb,
                             void *cuda_stream);

/* Pyramid level of an image (Section 2.1, coarse-to-fine), as lm_register
 * builds it: Gaussian blur with sigma = factor / 2 (taps exp(-j^2 / 2
 * sigma^2), |j| <= ceil(3 sigma), normalised, zero padding), then the
 * level voxel p is the blurred image read trilinearly (zero outside) at the
 * fine coordinate factor p + (factor - 1) / 2.
 *   src: device image [D][H][W] of src->dtype (caller-owned, read);
 *   factor: 2 or 4; the level is [Dl][Hl][Wl] with Dl = max(1, D / factor)
 *   (rounded down) and likewise for H and W;
 *   dst: device, Dl*Hl*Wl elements of src->dtype (written; BF16 levels are
 *   rounded once from the FP32 value);
 *   tmp: device scratch of 2*D*H*W floats (caller-owned, overwritten);
 *   dims (host, may be NULL) receives Dl, Hl, Wl.
 * Asynchronous on cuda_stream.  LM_EINVAL on NULL or host pointers, bad
 * sizes, dtypes or factors. */
LM_API int lm_downsample(const lm_volume *src, int factor, void *dst,
                         float *tmp, int *dims, void *cuda_stream);

/* Per-pair stopping loss.  The paper has no counterpart: it serves batched
 * runs that must bring every pair to a given loss (for instance the final
 * loss of another run) without spending iterations on pairs already there.
 * target: host array of npairs doubles, or NULL to clear every target; a
 * NaN entry means no target for that pair.  After an iteration whose
 * resulting loss is <= target[i], pair i stops: its later iterations are
 * no-ops (its kernels return at once, its field, loss and lambda stay) and
 * its lm_step_info reports stopped = 1, until lm_batch_reset.  Stream
 * ordered (the table update precedes later launches); LM_EINVAL on NULL b. */
LM_API int lm_batch_set_targets(lm_batch *b, const double *target);

/* Coarse-to-fine registration of every pair (as lm_register); reps (host,
 * npairs entries, may be NULL). */
LM_API int lm_batch_register(lm_batch *b, const lm_schedule *s,
                             float *const *u, lm_report *reps);
/* One-shot form: create a batch, register, destroy. */
LM_API int lm_register_batch(int npairs, const lm_volume *fixed,
                             const lm_volume *moving, float *const *u,
                             const lm_params *p, const lm_schedule *s,
                             void *cuda_stream, lm_report *reps);

/* ---- evaluation without allocation ------------------------------------ */
/* The paper has no counterpart: this entry point serves callers that cannot
 * allocate device memory while they evaluate (code inside another
 * framework's memory pool or allocator hooks, real-time loops where the
 * device synchronisation of cudaMalloc / cudaFree is not allowed, processes
 * that gave their free memory to another component).
 *
 * Same result as lm_eval on a fresh context: the loss (r = 1 - LNCC, or
 * the MSE) and its smoothed gradient at u (the smoothed update of
 * Eq. demons for LM_METHOD_DEMONS), without a context and without any
 * allocation.  The MI loss needs per-pair histogram buffers and returns
 * LM_EUNSUPPORTED here.
 * Its scratch is one static device array inside the library, sized for at
 * most LM_NOALLOC_MAX_VOXELS voxels (2^19, e.g. 80^3; about 29 MB, held
 * by every GPU that loads the library until the process exits), counted
 * with rows padded to a multiple of 4 voxels; larger volumes return
 * LM_EINVAL, and so do LNCC volumes whose halo-padded fixed-point layout
 * ((32 ceil(W / 32) + 4w) (32 ceil(H / 32) + 4w) (D + 4w + 2) elements for
 * window k = 2w + 1) exceeds 3 LM_NOALLOC_MAX_VOXELS.
 *   fixed, moving: images as for lm_init; p: parameters (NULL = defaults;
 *   every field is checked as lm_init checks it, and only win, eps_nr,
 *   eps_dr, sigma_grad, loss, method and alpha change the result);
 *   u: device field
 *   [3][D][H][W]; g_out: device [3][D][H][W] (written); loss_out: device
 *   double (written; NaN if the loss or gradient is not finite; may be
 *   NULL); gmax_out: device float (may be NULL); cuda_stream: the stream.
 *   Every non-NULL pointer must be device (or managed) memory; a host
 *   pointer returns LM_EINVAL before anything is launched.
 * Asynchronous on cuda_stream.  The first call on a device looks up the
 * array's device address and prepares the kernels (no allocation); make
 * that first call before any stream capture.  Every call shares the one
 * array, so calls whose work overlaps on the GPU (different streams, or
 * host threads without ordering) race and corrupt each other's results;
 * order them on one stream.  The array keeps the last call's contents;
 * every call overwrites all of the scratch it reads. */
#define LM_NOALLOC_MAX_VOXELS (1 << 19)
LM_API int lm_eval_noalloc(const lm_volume *fixed, const lm_volume *moving,
                           const lm_params *p, const float *u, float *g_out,
                           double *loss_out, float *gmax_out,
                           void *cuda_stream);

/* Debug-bounds build (compiled with -DLM_DEBUG_BOUNDS, the library
 * liblmreg_dbg.so): every device buffer a context allocates sits between
 * two 64 KiB guard bands of 0xFF bytes (NaN as a float, -1 as an integer),
 * so that a kernel reading past a buffer reads NaN or -1 and one writing
 * past it changes a band.  lm_debug_check synchronises and returns LM_OK
 * if every band of the context (and of its pyramid levels) is intact, else
 * LM_EBOUNDS with the buffer and byte in lm_last_error().  The release
 * build returns LM_EUNSUPPORTED.  The caller's own buffers (F, M, u,
 * g_out) are the caller's to guard. */
LM_API int lm_debug_check(lm_ctx *ctx);
LM_API int lm_batch_debug_check(lm_batch *b);

/* Static message for an LM_E* code. */
LM_API const char *lm_strerror(int code);

/* Message describing the last failure on the calling thread ("" if none). */
LM_API const char *lm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LMREG_H */
