/*
 * pinv.h - C ABI of the GB300 Pinv-Recon library (explicit Tikhonov-regularised
 * pseudoinverse MRI reconstruction, arXiv 2410.06129).
 *
 * The forward model is data = Encode x image (Eq. 1) with
 *     Encode[(c, m), n] = s_c(r_n) * exp(-i 2 pi (k_m . r_n + df_n t_m))
 * (Fourier term Eq. 2; coil-sensitivity and B0 off-resonance factors of
 * Section 3.3, multiplied as in the composite encoding of Section 3.3).
 * A plan holds one trajectory/coil/B0 configuration. Building it forms
 *     G = Encode^H Encode + lambda I                      (Eq. 6)
 *     G = L L^H                                           (Eq. 8)
 *     Recon = (L^-1)^H L^-1 Encode^H                      (Eq. 8)
 * and applying it computes image = Recon x data for a batch of frames (Eq. 3),
 * or, for factor-only plans, image = G^-1 (sum_c Encode_c^H data_c)
 * (Section 3.3, last paragraph).
 *
 * Conventions
 *   - Complex numbers are interleaved (re, im). c64 = 2 x float, c128 = 2 x double.
 *   - Voxels lie on a Cartesian grid: voxel with grid index (ix, iy, iz) sits at
 *     r = ((i - dims/2) / dims) * fov per dimension; the flat grid index is
 *     (iz * dims[1] + iy) * dims[0] + ix (x fastest). A plan reconstructs either
 *     the whole grid or an explicit voxel list (mask / over-discretised subset).
 *   - k is in cycles per unit length of fov (cycles/FOV when fov = 1).
 *   - lambda is the diagonal load itself (the paper writes it lambda^2).
 *   - Data batches are [F][C][M_k] (frame-major, coil, sample); images [F][N].
 *
 * Ownership and errors
 *   - Host arrays in pinv_plan_desc are copied during pinv_plan_create; the
 *     caller keeps ownership and may free them when it returns.
 *   - Device buffers passed to pinv_apply belong to the caller and must stay
 *     valid until the work enqueued on the given stream has completed.
 *   - Streams are cudaStream_t values passed as void*; NULL is the legacy
 *     default stream.
 *   - Every call returns a pinv_status and never aborts. pinv_last_error()
 *     returns a thread-local message for the last failing call on that thread.
 *   - Errors found on the device (a non-positive Cholesky pivot, a bounded
 *     wait that gave up) are recorded in the plan's device status word and
 *     returned by pinv_plan_sync().
 *   - A plan may be used from one host thread at a time.
 *
 * Device memory
 *   - Plans, their apply scratch and the build's temporaries take device memory
 *     from one pool per device owned by the library. The pool keeps memory that
 *     plans give back, so creating or building a plan again maps none. When the
 *     last plan is destroyed it is trimmed to 8 GiB (environment PINV_POOL_KEEP_MB:
 *     another size in MiB, 0 returns everything), so a program that creates and
 *     destroys plans of up to that size one after another maps nothing again.
 *     The device's default stream-ordered pool and the caller's allocator are not
 *     touched.
 */
#ifndef PINV_H
#define PINV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PINV_OK = 0,
    PINV_ERR_INVALID_ARG = 1,  /* bad descriptor or argument */
    PINV_ERR_OOM = 2,          /* device allocation failed */
    PINV_ERR_BUDGET = 3,       /* would exceed a memory budget (serving) */
    PINV_ERR_NOT_PD = 4,       /* G not positive definite; info = failing pivot */
    PINV_ERR_NOT_BUILT = 5,    /* apply/export before a successful build */
    PINV_ERR_TIMEOUT = 6,      /* a bounded device wait gave up */
    PINV_ERR_CUDA = 7,         /* CUDA runtime error (message has details) */
    PINV_ERR_INTERNAL = 8,
    PINV_ERR_UNSUPPORTED = 9   /* valid request this build does not implement */
} pinv_status;

typedef enum {
    PINV_FP64 = 0,          /* every stage in FP64 (SIMT DFMA) */
    PINV_MIXED_BF16X3 = 1,  /* tensor-core stages in split BF16, 2 slices / 3 products,
                               FP32 accumulation, FP64 panels, FP64-residual refinement */
    PINV_MIXED_BF16X6 = 2   /* as above with 3 slices / 6 products */
} pinv_precision;

typedef enum {
    PINV_LAMBDA_ABS = 0,            /* lambda used as given */
    PINV_LAMBDA_REL_MEAN_DIAG = 1   /* lambda * trace(E^H E) / N (mean diagonal of E^H E) */
} pinv_lambda_mode;

typedef enum { PINV_C64 = 0, PINV_C128 = 1 } pinv_dtype;

typedef enum {
    PINV_RECON_AUTO = -1,   /* explicit Recon if it fits the plan's footprint rule */
    PINV_RECON_NONE = 0,    /* factor-only: keep L and G^-1, apply via E^H data */
    PINV_RECON_STORE = 1    /* form and keep Recon = E^+ */
} pinv_recon_mode;

typedef struct {
    int ndim;                     /* 1, 2 or 3 */
    int dims[3];                  /* grid size per dimension (unused entries 1) */
    double fov[3];                /* field of view per dimension (unused entries 1.0) */
    const int64_t* voxel_index;   /* optional [N] flat grid indices; NULL = whole grid */
    int64_t n_vox;                /* N (must be prod(dims) when voxel_index is NULL) */
    int64_t n_samples;            /* M_k, samples per coil */
    const double* traj;           /* [M_k][ndim] k-space positions */
    int n_coils;                  /* C >= 1 */
    const double* coil_maps;      /* [C][N] complex128, or NULL when C == 1 (s = 1) */
    const double* b0_hz;          /* optional [N] off-resonance in Hz */
    const double* times;          /* [M_k] sample times in s; required iff b0_hz != NULL */
    double lambda;                /* diagonal load, see lambda_mode */
    int lambda_mode;              /* pinv_lambda_mode */
    int precision;                /* pinv_precision */
    int recon_mode;               /* pinv_recon_mode */
    int refine_max_iters;         /* refinement steps per apply (0 = none) */
    double refine_tol;            /* stop when ||r|| / ||E^H d|| <= tol (0 = run all steps) */
    int refine_residual;          /* mixed plans: pinv_residual arithmetic of the residual */
    int lean;                     /* 1: G / L (and the FP64 W of mixed plans whose residual is not
                                     FP64) exist only during pinv_build; the plan then keeps only
                                     what its apply reads (80 -> 32 bytes per N^2 entry for a mixed
                                     TOEPLITZ plan, which also drops its double-float exact Gram).
                                     Exports of L, W, G^-1 (mixed) and the exact Gram, maps and
                                     batches are then unavailable. 0: keep them. */
} pinv_plan_desc;

/* How the refinement forms the normal-equation residual r = E^H (d - E x) - lambda x.
 * DOUBLE_FLOAT and FP64 generate E twice per step (2 N M F complex MACs).
 * TOEPLITZ uses the identity r = E^H d - G x with the exact Gram G: without B0
 * and with voxels on the grid, (A^H A)[n][n'] depends only on the grid offset
 * between n and n' (Eq. 2), so G is formed in FP64 from a (2n_x-1)(2n_y-1)(2n_z-1)
 * table and the coil products at build time and stored as double-float
 * [N][N] (16 N^2 bytes) plus fixed-point digit tiles (24 N^2 bytes); each
 * apply forms E^H d once and each step costs N^2 F complex MACs. G x runs
 * exactly on the tensor cores (integer digit products); E^H d too with 16 or
 * more frames, otherwise in double-float. Plans with b0_hz reject TOEPLITZ. */
typedef enum {
    PINV_RESIDUAL_DOUBLE_FLOAT = 0, /* r in double-float (hi + lo floats, ~44 bits) on the FP32 units */
    PINV_RESIDUAL_FP64 = 1,         /* r in FP64 (DFMA); FP64 plans always use this */
    PINV_RESIDUAL_TOEPLITZ = 2      /* r = E^H d - G x, exact G from the Toeplitz table, double-float */
} pinv_residual;

typedef struct {
    int64_t n_vox, n_samples, n_rows;   /* N, M_k, M = C * M_k */
    int n_coils, precision, has_recon;
    double lambda_abs;                  /* diagonal load actually used */
    double min_pivot, max_pivot;        /* min / max of diag(L) (real, positive) */
    size_t bytes_device;                /* device memory held by the plan */
    size_t bytes_recon;                 /* of which Recon (E^+) */
    double ms_tables, ms_gram, ms_chol, ms_inverse, ms_recon;  /* last build, CUDA events */
    int info;                           /* failing pivot index (PINV_ERR_NOT_PD), else -1 */
    int last_refine_iters;              /* refinement steps taken by the last apply */
    double last_refine_resid;           /* ||r|| / ||E^H d|| after the last apply's refinement */
    double ms_gram_kernel;              /* of ms_gram: the tensor-core (mixed) or FP64 Gram kernels alone */
    /* The lambda / condition check (Section 2.1: the condition number of the
     * inversion; Section 2.2: the load lambda bounds every eigenvalue of G below
     * by lambda). Each build estimates kappa_1(G) = ||G||_1 ||G^-1||_1: ||G||_1
     * exactly (from G before the Cholesky, or from the exact Gram of TOEPLITZ
     * plans), ||G^-1||_1 by Hager's method (Higham's complex variant, at most
     * five rounds and an alternating-sign vector) with solves through the
     * factor. Mixed plans refine the two final candidates y once against G and
     * then certify them against G itself (||y||_1 / ||G y||_1, G y by the
     * refinement's residual operator), so the estimate is a lower bound of
     * kappa_1(G) up to the rounding of the sums
     * (mixed plans without the TOEPLITZ residual read ||G||_1 from the
     * split-precision Gram, so it carries that Gram's rounding).
     * Hager's estimates are usually within a factor of 3. NaN when G was not
     * positive definite. Runs on the build's stream without host synchronisation. */
    double kappa_est;                   /* estimate of kappa_1(G) */
    double norm1_g;                     /* ||G||_1 */
    double ms_cond;                     /* time of the condition estimate in the last build */
    /* With the refinement's stopping rule (refine_tol > 0) the last apply's
     * residual r = E^H (d - E x) - lambda x is that of the images returned, and
     * since every eigenvalue of G is at least lambda (Section 2.2),
     * ||x - x*|| / ||x|| <= ||r|| / (lambda ||x||) for the exact solution x* of
     * each frame: the largest of these certified bounds over the frames (0
     * without the stopping rule). The rule checks each residual before its
     * correction, so an image already within refine_tol is returned unchanged. */
    double last_refine_bound;
} pinv_plan_info_t;

typedef struct pinv_plan pinv_plan;

/* Library version as 10000 * major + 100 * minor + patch. */
int pinv_version(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (all plans, all threads). Lets callers count the library's launches in a
 * timed region. */
unsigned long long pinv_kernel_launches(void);

/* 1 if the current device runs this build's tensor-core (tcgen05, sm_103a)
 * kernels, which mixed-precision plans need; 0 otherwise. */
int pinv_tc_available(void);

/* Thread-local message describing the last error on this thread ("" if none). */
const char* pinv_last_error(void);

/*
 * Failure handling. Every wait of the tensor-core kernels' pipelines (for a
 * stage's operands, for an MMA group, for its drain) is bounded; past the bound
 * the CTA stops taking work, waits for the MMAs and copies it has issued, frees
 * its tensor memory and records the wait's site, and the build (or batch) then
 * reports PINV_ERR_TIMEOUT from pinv_plan_sync while later work still runs.
 * This sets that bound in SM clock cycles for builds started after the call,
 * process-wide (0: the default, about 2 s). A small value makes real waits run
 * out, which exercises that path; the waits of the clean-up itself keep the
 * default bound. Applies keep the default. Errors: INVALID_ARG for a negative
 * value. The paper has no counterpart: this is a test hook of this library.
 */
pinv_status pinv_set_wait_limit(int64_t cycles);

/*
 * Validate the descriptor, copy its arrays to the device on `stream` and
 * compute lambda. Builds nothing yet. Errors: INVALID_ARG (bad sizes, missing
 * times with b0_hz, C > 1 without coil maps, voxel index out of range),
 * OOM, CUDA. On success *out owns device memory until pinv_plan_destroy.
 */
pinv_status pinv_plan_create(const pinv_plan_desc* desc, void* stream, pinv_plan** out);

/*
 * Enqueue the build on `stream`: phase tables, Gram G = E^H E + lambda I
 * (E generated on the fly, coils folded in as the Hadamard product of the
 * coil-independent Gram with sum_c conj(s_c) s_c^T), blocked Cholesky G = L L^H,
 * G^-1 = (L^-1)^H L^-1, and (unless factor-only) Recon = G^-1 E^H (Eq. 6, 8).
 * Asynchronous: call pinv_plan_sync to learn whether G was positive definite.
 */
pinv_status pinv_build(pinv_plan* plan, void* stream);

/*
 * Wait for all work the plan enqueued, read its device status word and
 * return it: OK, NOT_PD (info = failing pivot), TIMEOUT or CUDA.
 */
pinv_status pinv_plan_sync(pinv_plan* plan);

/*
 * image = Recon x data for n_frames frames (Eq. 3), or G^-1 E^H data for
 * factor-only plans (Section 3.3). d_data: device [F][C][M_k], d_image:
 * device [F][N], both of `dtype` (pinv_dtype). Mixed-precision plans refine
 * each frame with FP64 residuals r = E^H (d - E x) - lambda x up to
 * refine_max_iters times. n_frames == 0 is a no-op. With the stopping rule
 * (refine_tol > 0) a residual or image that is not finite (NaN or Inf in the
 * data) ends the call with PINV_ERR_INVALID_ARG naming the frame. Uses plan-owned
 * scratch sized on first use; concurrent applies of one plan must be
 * serialised on one stream.
 */
pinv_status pinv_apply(pinv_plan* plan, const void* d_data, void* d_image, int64_t n_frames,
                       int dtype, void* stream);

/* Matrices a plan can export (device copies into caller buffers). */
typedef enum {
    PINV_EXPORT_GRAM = 0,    /* [N][N] c128: lower triangle of G (upper left untouched) */
    PINV_EXPORT_CHOL = 1,    /* [N][N] c128: lower triangle of L */
    PINV_EXPORT_GINV = 2,    /* [N][N] c128: G^-1, full */
    PINV_EXPORT_RECON = 3,   /* [N][C*M_k]: Recon = E^+, c128 (FP64 plans) or c64 (mixed) */
    PINV_EXPORT_LINV = 4,    /* [N][N] c128: W = L^-1 (mixed plans; UNSUPPORTED for FP64 plans) */
    PINV_EXPORT_GRAM_EXACT = 5 /* [N][N] c128: the exact Gram of TOEPLITZ-residual plans, full */
} pinv_export_what;

/*
 * Copy an internal matrix into the caller's device buffer `dst` of `bytes`
 * bytes, on `stream`. INVALID_ARG if bytes is too small, NOT_BUILT before a
 * build, UNSUPPORTED for RECON on factor-only plans. The Gram is kept only
 * until the Cholesky overwrites it unless the plan was built after
 * pinv_plan_keep_gram(plan, 1).
 */
pinv_status pinv_plan_export(const pinv_plan* plan, int what, void* dst, size_t bytes, void* stream);

/* Keep a copy of G (before factorisation) for export and diagnostics. */
pinv_status pinv_plan_keep_gram(pinv_plan* plan, int keep);

/* Sizes, lambda, pivots and per-stage timings of the last build. */
pinv_status pinv_plan_info(const pinv_plan* plan, pinv_plan_info_t* out);

/* Free the plan and its device memory (synchronises the device). The memory goes
 * back to the library's pool, which is trimmed to its kept size (8 GiB, or
 * PINV_POOL_KEEP_MB) when the last plan is destroyed. NULL is a no-op. */
void pinv_plan_destroy(pinv_plan* plan);

/* ------------------------------------------------------------------------
 * Batches. Many slices, time series or trajectories of uneven size, each its
 * own plan, built and applied together. The build runs every plan's
 * tensor-core Gram as one persistent launch, every plan's Recon as two more
 * (T = W E^H, then W^H T; Eq. 8), and the per-plan Cholesky and triangular
 * inverse concurrently on per-plan streams in between. The apply runs every
 * plan's apply concurrently. With PINV_BATCH_GRAPH the build sequence is
 * captured into a CUDA graph on the second pinv_batch_build call and replayed
 * from then on; the apply sequence is captured on first use and again
 * whenever its buffers, frame counts or dtype change. Graph capture needs a
 * created stream (not the legacy default stream); applies of plans with a
 * refinement stopping rule (refine_tol > 0) read the host and run uncaptured.
 * Results are bit-identical to pinv_build / pinv_apply on each plan.
 * The plans stay owned by the caller and must outlive the batch; while in a
 * batch they should not be built or applied on their own concurrently.
 * ---------------------------------------------------------------------- */
typedef struct pinv_batch pinv_batch;
#define PINV_BATCH_GRAPH 1

/* Group n_plans plans of one precision (all FP64, or all mixed with the same
 * slice count). Allocates the batch's tensor-core intermediates (W E^H and W^T
 * for explicit-Recon plans: 8 N (M + N) bytes per plan). */
pinv_status pinv_batch_create(pinv_plan* const* plans, int n_plans, int flags, pinv_batch** out);

/* Build every plan (asynchronous on `stream`; errors via pinv_batch_sync). */
pinv_status pinv_batch_build(pinv_batch* batch, void* cuda_stream);

/* image_i = Recon_i x data_i (+ refinement) for every plan i: d_data[i] is
 * [n_frames[i]][C_i][M_k,i] and d_image[i] is [n_frames[i]][N_i], device
 * buffers of `dtype` owned by the caller. */
pinv_status pinv_batch_apply(pinv_batch* batch, const void* const* d_data, void* const* d_image,
                             const int64_t* n_frames, int dtype, void* cuda_stream);

/* Wait for the batch's last build; returns the first plan's failure (its
 * index in *failed_plan, -1 if none) or a batched-launch timeout. */
pinv_status pinv_batch_sync(pinv_batch* batch, int* failed_plan);

/* Free the batch (not its plans). NULL is a no-op. */
void pinv_batch_destroy(pinv_batch* batch);

/* ------------------------------------------------------------------------
 * Serving loop. Recon is built from the trajectory and encoding physics
 * before data arrive and each acquisition then needs only image = Recon x data
 * (Section 4.5, Section 5). A server keeps the factored plans of registered
 * encodings resident in device memory under a byte budget and serves
 * reconstruction requests as they arrive (continuous batching):
 *   - requests are admitted in arrival order into up to max_slots slots, each
 *     with its own stream and scratch, so work of different requests and of
 *     plan builds overlaps on the device;
 *   - a request whose plan is not resident builds it first on a separate build
 *     stream. Room is made in tiers, least recently used first: idle plans
 *     drop their Recon (they keep serving from their factors, x = W^H W E^H d
 *     plus refinement), then idle plans are evicted; a plan whose Recon does
 *     not fit is built factor-only. A plan that cannot fit even factor-only
 *     fails its request with PINV_ERR_BUDGET, and a plan whose Gram is not
 *     positive definite fails its requests with PINV_ERR_NOT_PD; other
 *     requests are unaffected;
 *   - a request's image is computed exactly as pinv_apply would compute it on
 *     the plan in its current form (with or without Recon), whatever else is
 *     in flight.
 * One worker thread per server issues all CUDA work; the calls below only
 * queue, poll or wait and are safe from any host thread. Registered plans run
 * their refinement with a fixed number of steps (refine_tol is ignored) so the
 * worker never blocks on a host read.
 * ---------------------------------------------------------------------- */
typedef struct pinv_server pinv_server;

/* Completion callback, called on the server's worker thread just before the
 * request counts as finished; it must not call the server's wait functions. */
typedef void (*pinv_done_cb)(uint64_t ticket, pinv_status status, void* user);

typedef struct {
    uint64_t completed, failed, builds, evictions;
    double frames;                    /* frames reconstructed by completed requests */
    double p50_ms, p99_ms, mean_ms, max_ms;  /* enqueue -> completion latency */
    double span_s;                    /* first enqueue to last completion */
    size_t resident_bytes;            /* device bytes held by resident plans */
    int resident_plans, queued;
    uint64_t recon_drops;             /* Recons dropped to make room (plans kept their factors) */
} pinv_server_stats_t;

/* Create a server on the current device. hbm_budget_bytes bounds the bytes of
 * resident plans; max_slots (1..64) bounds the requests in flight. */
pinv_status pinv_server_create(size_t hbm_budget_bytes, int max_slots, pinv_server** out);

/* Register an encoding (descriptor arrays are copied); no device work yet. */
pinv_status pinv_serve_register(pinv_server* server, const pinv_plan_desc* desc, int* plan_id);

/* Queue image = Recon x data for n_frames frames of device buffers d_data
 * [F][C][M_k] and d_image [F][N] of `dtype`; the buffers must stay valid until
 * the request finishes. Returns at once with a ticket. */
pinv_status pinv_serve_enqueue(pinv_server* server, int plan_id, const void* d_data, void* d_image,
                               int64_t n_frames, int dtype, pinv_done_cb cb, void* user, uint64_t* ticket);

/* Non-blocking: *done = 1 and *result = its status once the request finished. */
pinv_status pinv_serve_poll(pinv_server* server, uint64_t ticket, int* done, pinv_status* result);

/* Block until the request finished (PINV_ERR_TIMEOUT after timeout_s seconds). */
pinv_status pinv_serve_wait(pinv_server* server, uint64_t ticket, double timeout_s, pinv_status* result);

/* Merging (off until set): a request dispatched to a slot takes with it the
 * requests of the same plan and element type queued behind it, while their
 * frames together stay within max_frames (0 turns merging off). Their frames are
 * gathered into the slot's scratch, reconstructed by one apply and scattered to
 * each request's image; each request still completes and is counted on its own,
 * and its image is the one a standalone apply of its frames gives (up to the
 * order of sums in kernels whose split depends on the frame count). Merging is
 * not done while host faults (PINV_FAULT) are set. */
pinv_status pinv_server_set_merge(pinv_server* server, int64_t max_frames);

/* Times of a finished request, in milliseconds after the server was created:
 * times_ms[0] enqueue and [1] completion as the worker saw it (host clock);
 * [2] start and [3] end of its device work, read from timing events on its
 * slot's stream (device clock, from an event recorded at creation; the start
 * is when the stream reached the request, after any plan build it waited for;
 * both -1 for a request that failed or had no frames). Two requests whose
 * device intervals intersect ran on the device at the same time.
 * PINV_ERR_INVALID_ARG for an unknown or unfinished ticket. */
pinv_status pinv_serve_times(pinv_server* server, uint64_t ticket, double* times_ms);

/* Counters and latency percentiles of the requests completed so far. */
pinv_status pinv_server_stats(pinv_server* server, pinv_server_stats_t* out);

/* Finish queued requests, stop the worker and free every resident plan. */
void pinv_server_destroy(pinv_server* server);

/* Launch-shape autotuner. The apply-side kernels (Recon x data, the
 * double-float residual and E^H d, the FP32 correction) offer several tile
 * shapes per size class; the first launch of a class times each candidate on
 * its stream and keeps the fastest (PINV_AUTOTUNE=0 in the environment turns
 * this off). Candidates differ in speed only: every output is summed in the
 * same order. Writes a one-line summary of the choices made so far into buf
 * (NUL-terminated, truncated to bytes) and returns its full length. */
size_t pinv_autotune_report(char* buf, size_t bytes);

/* Per-voxel image-quality maps (Section 2.5), written to d_out [N] (device
 * float64) on `stream`:
 *   PINV_MAP_SRF   the SRF map, diag(Recon x Encode) (Eq. 9) = 1 - lambda diag(G^-1);
 *   PINV_MAP_NOISE the noise map, diag(Recon Psi Recon^H) (Eq. 10). With psi == NULL
 *                  the data noise is white (Psi = I) and the map is
 *                  diag(G^-1) - lambda diag(G^-2). Otherwise psi is a host
 *                  [C][C] complex128 coil noise covariance applied to every
 *                  sample (Psi = psi (x) I), and the map is formed from the
 *                  stored Recon (PINV_ERR_UNSUPPORTED for factor-only plans).
 * FP64 plans use their FP64 G^-1. Mixed plans with the TOEPLITZ residual refine
 * G^-1 with refine_max_iters double-float steps (temporary memory about
 * 56 N^2 bytes); other mixed plans use W^H W from their split-precision factor
 * (its error, up to kappa(G) times the split rounding, carries into the map).
 * Coil-covariance maps carry the precision of the stored Recon. */
typedef enum { PINV_MAP_SRF = 0, PINV_MAP_NOISE = 1 } pinv_map_what;
pinv_status pinv_plan_map(pinv_plan* plan, int what, const double* psi, double* d_out, void* cuda_stream);

/* Eigenvalue decomposition of the Gram matrix (Section 2.1: the eigenvalues of
 * E^H E are the squared singular values of Encode, and their spectrum shows the
 * conditioning): E^H E + lambda I = P diag(mu + lambda) P^H, by parallel cyclic
 * Jacobi in FP64 on the plan's kept Gram (pinv_plan_keep_gram before the build;
 * a mixed plan's Gram carries its split-precision rounding).
 *   d_mu  [N] doubles, device: eigenvalues of E^H E (lambda removed), decreasing.
 *   d_P   [N][N] c128, device, row-major, column i the eigenvector of mu[i];
 *         may be NULL: eigenvalues only, by Householder reduction to a real
 *         symmetric tridiagonal and bisection instead (sweeps_out = 0).
 *   sweeps_out  Jacobi sweeps taken (may be NULL).
 * Synchronises with the device once per sweep. Sweeps stop at an off-diagonal
 * Frobenius norm of 4 N eps of the whole, or once a sweep no longer halves it
 * below 1e-10. UNSUPPORTED without a kept Gram, or for eigenvectors with N > 8192;
 * PINV_ERR_INTERNAL if 30 sweeps do not converge (the outputs are still written). */
pinv_status pinv_plan_eig(pinv_plan* plan, double* d_mu, void* d_P, int* sweeps_out, void* cuda_stream);

/* Truncated eigen (tSVD) reconstruction (Section 2.1): image = P_r diag(1 / (mu_r
 * + lam)) P_r^H E^H data, r the fewest leading eigenvalues holding the fraction
 * `energy` of the sum of mu (in (0, 1]; 1 keeps all), lam >= 0 an optional
 * Tikhonov loading combined with the truncation. d_mu / d_P from pinv_plan_eig;
 * data [F][C][M_k] and image [F][N] as pinv_apply (dtype PINV_C64 or PINV_C128).
 * rank_out / kappa_out (may be NULL; if given the call waits for the device):
 * r and the condition number sqrt(mu[0] / mu[r-1]) of the truncated problem. */
pinv_status pinv_tsvd_apply(pinv_plan* plan, const double* d_mu, const void* d_P, double energy, double lam,
                            const void* d_data, void* d_image, int64_t n_frames, int dtype, int* rank_out,
                            double* kappa_out, void* cuda_stream);

/* Size of the fixed device scratch array behind pinv_apply_noalloc (64 MiB). */
#define PINV_NOALLOC_SCRATCH_BYTES (64u << 20)

/*
 * Same result as pinv_apply, for callers that cannot allocate device memory
 * when they reconstruct. Examples are a scanner's real-time loop running
 * under a fixed, pre-reserved memory budget, or an application whose device
 * memory belongs to another allocator that must not be bypassed. A cudaMalloc
 * there can also stall the device while it synchronises and break the loop's
 * latency. The paper has no counterpart; this is an interface for such
 * callers.
 *
 * pinv_apply grows plan-owned scratch on first use. This call instead takes
 * its scratch from one file-scope device array of PINV_NOALLOC_SCRATCH_BYTES.
 * That array exists once on every GPU that loads the library and is held until
 * the process exits. The call allocates nothing: no cudaMalloc, cudaFree or
 * allocating library routine.
 *
 * Scratch needed, rounded per buffer to 256 B:
 *   16 F M   when dtype is c64 and the plan is FP64, factor-only or refined;
 *   16 F N   when dtype is c64;
 *   16 F M   when refining, or for mixed factor-only plans;
 *   16 F N   when refining, or for factor-only plans;
 *    8 F M   for mixed plans with Recon and c128 data;
 *    8 F N   for mixed plans with Recon, or refined with the double-float residual;
 *   24 F     when the refinement's stopping rule (refine_tol > 0) is on;
 * plus the partial sums and digit tiles of the tensor-core products, and for
 * plans with B0 that hold the exact-product digit tables, 16 F C N for the
 * coil-weighted images (the call computes the exact total).
 * A call that needs more fails with PINV_ERR_INVALID_ARG and a message giving
 * the size; split the frames over several calls.
 *
 * The first call on a device resolves the array's device address there (once
 * per device, with that device current). Make that first call before any
 * stream capture. Every call shares the array, and it keeps the last call's
 * contents; nothing in it needs to start at zero, since each buffer is fully
 * written before it is read. Calls whose GPU work overlaps (other streams or
 * host threads) race on the array. Arguments and errors are otherwise those of
 * pinv_apply.
 */
pinv_status pinv_apply_noalloc(pinv_plan* plan, const void* d_data, void* d_image, int64_t n_frames,
                               int dtype, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PINV_H */
