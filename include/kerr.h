/*
 * kerr.h -- C ABI of libkerr: batched integration of null and time-like
 * geodesics of the Kerr metric in Cartesian Kerr-Schild coordinates on an
 * NVIDIA GB300 (sm_103a).
 *
 * Method: Chan, Medeiros, Ozel & Psaltis, "GRay2" (arXiv:1706.07062).
 *   - metric g_ab = eta_ab + f l_a l_b, M = 1               (Sec. 2.1, eq. def:CKS, eq. CKSr)
 *   - right-hand side in the optimised split-metric form    (Sec. 2.1, eqs. opt0 and opti)
 *   - classic 4th-order Runge-Kutta stepping                (Sec. 3)
 *   - termination near the horizon or beyond the start radius (Sec. 4)
 * Step-size control (step doubling), surface clipping, the FP32+Kahan
 * precision scheme and the persistent work queue are this library's own
 * additions; their exact rules are stated at kerr_opts below.
 *
 * Conventions shared by every entry point
 *   Units      G = c = M = 1.  State of a geodesic: x^mu = (t, x, y, z) and
 *              k^mu = dx^mu/dlambda = (k^t, k^x, k^y, k^z).
 *   Layout     Structure of arrays.  A "[4][n] plane" argument is 4*n doubles,
 *              component mu of geodesic i at index mu*n + i.  status and steps
 *              are n int32; diag is a [4][n] float plane (E, L_z, Q, u^2).
 *   Memory     Every pointer may be host memory (pageable or pinned) or device
 *              memory of the current device; the library tells them apart with
 *              cudaPointerGetAttributes.  With any host pointer the call
 *              returns only after the stream is synchronised: host buffers are
 *              staged through library-owned device buffers, except that the
 *              end points and diagnostics (x_out, k_out, diag) of the trace
 *              calls are written by the kernels straight into page-locked
 *              (pinned) host buffers.  With device pointers only, the call is
 *              asynchronous on `stream`.  Inputs are never modified.  The
 *              caller owns all inputs and outputs; the context owns its
 *              scratch (work-queue counter, statistics, staging buffers,
 *              CUDA graphs) and frees it in kerr_destroy.
 *   Streams    `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   Errors     0 on success, a negative KERR_E* code otherwise; the message
 *              is in kerr_last_error() (thread-local).  On a negative return
 *              the output buffers are unspecified.  Per-geodesic outcomes are
 *              reported in status[], never as a return code.
 *   n == 0     A no-op that returns 0.
 */
#ifndef KERR_H
#define KERR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KERR_OK 0
#define KERR_EINVAL (-1)   /* bad argument (spin, sizes, options, NULL pointer) */
#define KERR_ENOMEM (-2)   /* device or host allocation failed                  */
#define KERR_ECUDA (-3)    /* a CUDA runtime call failed                        */

/* Per-geodesic outcome written to status[]. */
#define KERR_ESCAPED 1     /* r > r_escape while moving outward (x^i k^i > 0)  */
#define KERR_CAPTURED 2    /* r < 1.01 r_h, r_h = 1 + sqrt(1 - a^2)             */
#define KERR_ENDTIME 3     /* t crossed opts.t_end                              */
#define KERR_MAXSTEPS 4    /* opts.max_steps attempted steps without an event  */
#define KERR_TIMEOUT 5     /* opts.budget_ns ran out; state is where it stopped */
#define KERR_NONFINITE 6   /* the state became (or started) NaN or infinite    */
#define KERR_INVALID_IC 7  /* no real k^t / u^t solves the norm condition       */

/* Arithmetic of the integration. */
#define KERR_FP64 0        /* every step in FP64                                */
#define KERR_FP32_KAHAN 1  /* FP32 steps with compensated (Kahan) state update; */
                           /* FP64 for set-up, diagnostics and steps that start */
                           /* inside opts.fp64_zone * r_h                       */

/* Arithmetic of FP32-path steps inside opts.fp64_zone * r_h. */
#define KERR_ZONE_FP64 0   /* IEEE FP64 (1/64 of the FP32 rate on GB300)         */
#define KERR_ZONE_F32X2 1  /* float-float on the FP32 pipe: unevaluated sums of  */
                           /* two floats, ~48-bit significand                    */

typedef struct kerr_ctx kerr_ctx;

/* Integration options.  Fill with kerr_opts_default() and change fields.
 *
 * Step control (adaptive, tol > 0).  Each attempt of length h takes one RK4
 * step of h and two of h/2 from the same state (11 right-hand sides, the
 * first shared).  With delta = (y_half - y_full)/15 the error is
 *   err = max over i in {x, y, z, k^t, k^x, k^y, k^z} of
 *         |delta_i| / (tol * (1 + max(|y_i|, |y_half_i|)))
 * (t is left out: it never enters the right-hand side).  err <= 1 accepts
 * y_half; either way h is multiplied by clamp(0.9 err^(-1/5), 0.2, 5), by 5 if
 * err == 0 and by 0.2 if err is not finite.
 *
 * Termination, tested after each accepted step in this order:
 *   captured  r < 1.01 r_h;
 *   escaped   r > r_esc and x^i k^i > 0, where r_esc = r_escape if > 0, the
 *             geodesic's start radius if == 0, and +infinity if < 0;
 *   end time  t - t_end changed sign from its initial value (t_end finite).
 * The crossing step is then clipped onto the surface: the step as a function
 * of its length (two RK4 half steps from the last accepted state) is solved
 * for the surface by Illinois regula falsi, to |r - r_stop| <= 1e-12 r_stop on
 * the FP64 path, 2e-6 r_stop for FP32 steps and 1e-10 r_stop for the FP64 (or
 * float-float) zone steps of the FP32+Kahan path, whose end points are only
 * good to ~1e-6 anyway (for t the same factors times max(1, |t_end|), except
 * FP32 steps: 2e-6 times max(1, the step's change of t)), or clip_maxit
 * iterations.  A geodesic that starts inside 1.01 r_h is
 * captured with no step; one that reaches max_steps attempts is MAXSTEPS. */
typedef struct {
    int32_t prec;          /* KERR_FP64 or KERR_FP32_KAHAN                       */
    int32_t renorm_every;  /* > 0: every n accepted steps re-solve k^t (FP64) so */
                           /* that g_ab k^a k^b keeps its initial value, on the  */
                           /* root nearest the current k^t; 0: off               */
    double tol;            /* error tolerance, > 0                               */
    double h0;             /* first trial step in lambda, > 0                    */
    int64_t max_steps;     /* cap on attempted steps per geodesic, >= 0          */
    double r_escape;       /* see above                                          */
    double t_end;          /* +-INFINITY or NaN: no end-time event               */
    double fp64_zone;      /* FP32 path: steps that start at r < fp64_zone * r_h */
                           /* run in FP64; 0 = never                             */
    int32_t clip_maxit;    /* iterations of the surface root-find, >= 1          */
    int32_t variant;       /* kernel launch configuration: -1 = autotuned (or    */
                           /* the default before tuning), else an index < the    */
                           /* value of kerr_num_variants()                       */
    uint64_t budget_ns;    /* wall-time budget of each launch on the device; 0 = */
                           /* none.  Geodesics unfinished when it runs out get   */
                           /* KERR_TIMEOUT and the state reached so far          */
    int32_t zone_prec;     /* FP32 path, arithmetic of the steps inside the     */
                           /* zone: KERR_ZONE_FP64 or KERR_ZONE_F32X2            */
    int32_t zone_variant;  /* launch shape of the zone phase: -1 = default, else */
                           /* an index < kerr_num_zone_variants()                */
    int32_t zone_quantum;  /* FP32 path, zone phase: every this many iterations */
                           /* of a warp (staggered over the warps), geodesics    */
                           /* that took at least half as many attempts since     */
                           /* they got their lane give it to ones that wait for  */
                           /* a lane and go to the back of the queue (processor  */
                           /* sharing; results do not depend on it); 0 = each    */
                           /* geodesic keeps its lane to the end; >= 0           */
} kerr_opts;

/* One pinhole-free parallel-ray camera (the paper's image-plane rays,
 * Sec. 4; its geometry follows this library's reading):
 *   observer direction n = (sin incl, 0, cos incl); image axes
 *   e_alpha = (0, 1, 0), e_beta = (-cos incl, 0, sin incl); pixel (p, q)
 *   has alpha = -w + (p + 1/2) 2w/nx, beta = -w + (q + 1/2) 2w/ny and flat
 *   index q*nx + p; the ray starts at t = 0, x = r_obs n + alpha e_alpha +
 *   beta e_beta, with spatial k = -n and k^t < 0 from g_ab k^a k^b = 0
 *   (past-directed: the ray is traced backward from the observer).        */
typedef struct {
    double a;              /* spin of this image's black hole, |a| <= 1          */
    double incl;           /* inclination in radians                             */
    double r_obs;          /* observer distance, > 1.01 r_h                      */
    double half_width;     /* w, > 0                                             */
    int32_t nx, ny;        /* pixels, > 0                                        */
} kerr_camera;

/* Counters of the last trace call on a context (read after the stream is
 * synchronised). */
typedef struct {
    int64_t geodesics;        /* geodesics handled                               */
    int64_t attempts;         /* attempted steps, all precisions                 */
    int64_t accepted;         /* accepted steps                                  */
    int64_t rhs_fp32;         /* right-hand sides evaluated in FP32              */
    int64_t rhs_fp64;         /* right-hand sides evaluated in FP64              */
    int64_t attempts_fp64;    /* attempted steps taken in FP64                   */
    int64_t deferred;         /* FP32 path: geodesics handed to the FP64-zone    */
                              /* phase (second launch of the same call)          */
    int64_t status_count[8];  /* geodesics per status code                       */
    float kernel_ms;          /* device time of the whole integration launch     */
    int32_t variant;          /* launch configuration used                       */
    float phase_ms[4];        /* FP32 path: set-up, FP32 stepping, FP64-zone     */
                              /* phase, finishing; FP64 path: [1] = stepping     */
    int64_t requeued;         /* FP32 path: zone-phase geodesics that gave their */
                              /* lane to a waiting one (see zone_quantum)        */
    int64_t queue_errors;     /* zone-phase queue hand-overs that timed out (the */
                              /* geodesic is then lost); 0 unless the library is */
                              /* faulty                                          */
    int64_t rhs_fp32_zone_phase;      /* FP32 path: of rhs_fp32, those evaluated */
    int64_t attempts_fp32_zone_phase; /* (and FP32 attempts taken) by the zone   */
                                      /* phase for geodesics outside the zone    */
    int64_t clips;            /* end points clipped onto an event surface        */
    int64_t clip_rhs;         /* right-hand sides evaluated by those clips       */
} kerr_stats;

/* Fills *opts with: prec FP32_KAHAN, tol 1e-6, h0 1, max_steps 1e6,
 * r_escape 0, t_end +inf, fp64_zone 1.5, renorm_every 0, clip_maxit 40,
 * variant -1, budget_ns 0, zone_prec KERR_ZONE_FP64, zone_variant -1,
 * zone_quantum 32 (measured best of 8..64 on the 1024x1024 image). */
void kerr_opts_default(kerr_opts *opts);

/* Creates a context for black-hole spin a (|a| <= 1, else KERR_EINVAL) on the
 * current CUDA device.  The spin applies to kerr_trace_rays and
 * kerr_trace_particles; cameras carry their own. */
int kerr_init(double a, kerr_ctx **out);

/* Frees the context and everything it owns; NULL is a no-op.  Waits for the
 * context's work to finish. */
int kerr_destroy(kerr_ctx *ctx);

/* Integrates n geodesics from the given states (any causal type; nothing is
 * renormalised at the start).  x0, k0: [4][n] planes.  Outputs: end states
 * x_out, k_out ([4][n]), status[n], steps[n] (attempted steps), and diag
 * ([4][n] floats: E = -p_t, L_z = x p_y - y p_x, Carter's Q, u^2 = g_ab k^a k^b
 * at the end state, FP64-computed) unless diag is NULL.  Sec. 2.1 (eqs.
 * opt0/opti), Sec. 3 (RK4), Sec. 4 (termination).
 *
 * cross (NULL = not recorded): [5][n] floats, the first two equatorial
 * crossings along the integration and a redshift there -- r1, phi1, r2,
 * phi2, g1 -- with NaN where absent.  A crossing is an accepted step (or
 * clipped end step) across z = 0, located on z = 0 by the same root-find as
 * the clipping; r is the KS radius, phi = atan2(y, x) - atan2(a, r) the KS
 * azimuth in (-pi, pi], and g1 = 1 / (u^t (1 - Omega xi)) the redshift of a
 * prograde Keplerian emitter at r1 (Omega = 1/(r^{3/2} + a), xi = L_z/E of
 * the start state), NaN inside the ISCO.  (Labels for the surrogate; the
 * paper has none.) */
int kerr_trace_rays(kerr_ctx *ctx, const double *x0, const double *k0, int64_t n,
                    const kerr_opts *opts, double *x_out, double *k_out, int32_t *status,
                    int32_t *steps, float *diag, float *cross, void *stream);

/* Integrates every ray of ncam cameras (Sec. 4: backward null geodesics from
 * an image plane at large distance); the initial states are built on the
 * device in FP64.  Rays are numbered camera by camera, row-major inside a
 * camera; outputs as for kerr_trace_rays with n = sum of nx*ny.  With
 * opts->r_escape == 0 each ray escapes at its own start radius. */
int kerr_trace_camera(kerr_ctx *ctx, const kerr_camera *cams, int32_t ncam,
                      const kerr_opts *opts, double *x_out, double *k_out, int32_t *status,
                      int32_t *steps, float *diag, float *cross, void *stream);

/* Integrates the pixels index[0 .. n-1] (device memory, flat indices q*nx + p
 * in [0, nx*ny)) of one camera; outputs as for kerr_trace_rays, entry i for
 * pixel index[i].  The same rays as kerr_trace_camera, for any subset and
 * order: a share of one image per process when an image is split across
 * GPUs (the only exchange is the host-side concatenation of the outputs). */
int kerr_trace_camera_pixels(kerr_ctx *ctx, const kerr_camera *cam, const int64_t *index,
                             int64_t n, const kerr_opts *opts, double *x_out, double *k_out,
                             int32_t *status, int32_t *steps, float *diag, float *cross,
                             void *stream);

/* Integrates n massive particles (Sec. 3.2: time-like geodesics with the same
 * integrator).  x0: [4][n] plane of start events; v0: [3][n] plane of
 * coordinate velocities dx^i/dt.  u^t is solved in FP64 from g_ab u^a u^b = -1
 * with u^i = u^t v^i; a velocity that is not time-like gives KERR_INVALID_IC
 * (end state = start event, k = 0).  t_end: n end times, one per particle,
 * or NULL to use opts->t_end for all.  Outputs as for kerr_trace_rays (k_out
 * holds u^mu). */
int kerr_trace_particles(kerr_ctx *ctx, const double *x0, const double *v0, const double *t_end,
                         int64_t n, const kerr_opts *opts, double *x_out, double *k_out,
                         int32_t *status, int32_t *steps, float *diag, float *cross,
                         void *stream);

/* Copies the counters of the last trace call into *out (synchronises the
 * context's stream first). */
int kerr_get_stats(kerr_ctx *ctx, kerr_stats *out);

/* Number of kernel launch configurations (block size x register cap). */
int kerr_num_variants(void);

/* Describes variant v: threads per block and minimum resident blocks per SM
 * (which sets the register cap). */
int kerr_variant_info(int v, int32_t *block, int32_t *min_blocks);

/* The same plus the geodesics each thread advances (1, or 2: the FP32
 * stepping phase runs two geodesics per thread on packed f32x2 instructions;
 * such variants are FP32-only, and KERR_FP64 calls reject them) and how the
 * FP32 steps evaluate their right-hand sides (0 inline, 1 one out-of-line
 * copy).  Any output pointer may be NULL.  KERR_EINVAL for v out of range. */
int kerr_variant_shape(int v, int32_t *block, int32_t *min_blocks, int32_t *rays_per_thread,
                       int32_t *rhs_mode);

/* Launch shapes of the FP32 path's zone phase (threads per block, blocks per
 * SM); fewer threads than deferred geodesics lets lanes refill.  Variant 7
 * (the default) is variant 3 whose tail -- once at most half as many zone
 * geodesics remain as the launch has lanes -- keeps at most 16 geodesics per
 * warp and pairs each with an idle lane: the helper computes the full RK4
 * step while the owner computes the half steps (the same arithmetic: results
 * bit-identical to variant 3).  Variant 8 is variant 4 (right-hand sides of
 * the full step and the first half step evaluated in interleaved pairs) with
 * the same two-lane tail, bit-identical to variant 4. */
int kerr_num_zone_variants(void);
int kerr_zone_variant_info(int v, int32_t *block, int32_t *blocks_per_sm);

/* Autotuning (the counterpart of the paper's run-time tuning of the OpenCL
 * work-group size for each image size, Sec. 4).  The search space is the
 * stepping variants -- threads per block x register cap (the minimum
 * resident blocks per SM, which caps registers at 65536 / (block x blocks))
 * x geodesics per thread (1, or 2 on packed f32x2 instructions, FP32 only) x
 * right-hand-side mode -- and, for the FP32+Kahan path with an FP64 zone, the
 * zone-phase launch shapes.  Coordinate search: every stepping variant with
 * the default zone shape, then every zone shape with the best stepping
 * variant; each candidate is traced once untimed (graph capture, buffers) and
 * then timed (device time of the whole call, minimum over repetitions) on a
 * sample of the workload.  The choice is kept by the context for its later
 * calls with variant == -1 / zone_variant == -1 in that precision.
 *
 * cache_path (NULL = no cache): a text file of lines
 *   <gpu>\t<workload key>\t<variant>\t<zone variant>\t<ms>\n
 * where <gpu> is the device name with its SM count ("NVIDIA GB300 (152
 * SMs)") and the key describes the workload's shape and options, including
 * the precision (kerr_tune_key_cameras / kerr_tune_key_particles).  When the
 * file holds the (gpu, key) pair (the last matching line wins) nothing is
 * timed and the stored choice is applied (out->from_cache = 1); otherwise the
 * result is appended. */
typedef struct {
    int32_t variant;       /* chosen stepping variant                           */
    int32_t zone_variant;  /* chosen zone-phase variant, -1 without a zone phase */
    float ms;              /* device time of the chosen configuration (sample)  */
    int32_t from_cache;    /* 1: read from the cache file, nothing was timed    */
    int32_t timed;         /* configurations timed                              */
} kerr_tuning;

/* Tunes on `sample` rays of the camera list: each camera at a resolution
 * lowered in proportion to its share of the rays, over the same field of
 * view, so the sample has the batch's mix of images. */
int kerr_autotune_cameras(kerr_ctx *ctx, const kerr_camera *cams, int32_t ncam,
                          const kerr_opts *opts, int64_t sample, const char *cache_path,
                          kerr_tuning *out, void *stream);

/* Tunes on every (n / sample)-th of n particles (inputs as for
 * kerr_trace_particles, host or device memory; pass shortened end times to
 * tune a long run on a shorter one). */
int kerr_autotune_particles(kerr_ctx *ctx, const double *x0, const double *v0,
                            const double *t_end, int64_t n, const kerr_opts *opts, int64_t sample,
                            const char *cache_path, kerr_tuning *out, void *stream);

/* Workload keys of the cache (host only): the camera list's size, a hash of
 * its geometry (spins, inclinations, distances, widths, pixel counts) and the
 * options that change the work (precision, tol, zone radius and arithmetic,
 * renormalisation); for particles their number, max_steps and the same
 * options.  KERR_EINVAL if `cap` bytes do not hold the key. */
int kerr_tune_key_cameras(const kerr_camera *cams, int32_t ncam, const kerr_opts *opts, char *buf,
                          int32_t cap);
int kerr_tune_key_particles(int64_t n, const kerr_opts *opts, char *buf, int32_t cap);

/* The cache file itself (host only; no GPU needed): lookup returns KERR_OK
 * and fills *out when (gpu, key) is present, 1 when it is not (or the file
 * does not exist), KERR_EINVAL for a malformed file; store appends one line
 * (KERR_EINVAL for empty fields or fields holding a tab or newline). */
int kerr_tune_cache_lookup(const char *path, const char *gpu, const char *key, kerr_tuning *out);
int kerr_tune_cache_store(const char *path, const char *gpu, const char *key,
                          const kerr_tuning *t);

/* The single-camera form: tunes on `sample` rays of cams[0] (no cache) and
 * writes the chosen stepping variant to *best (the zone shape is chosen and
 * kept too). */
int kerr_autotune(kerr_ctx *ctx, const kerr_camera *cam, const kerr_opts *opts,
                  int64_t sample, int32_t *best, void *stream);

/* Allocation-free camera tracing.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- real-time
 * hosts that must not call cudaMalloc/cudaFree once running (both may
 * synchronise the device and have unbounded latency), or hosts whose device
 * memory is owned and budgeted by another framework's pool.
 *
 * Same computation and outputs as kerr_trace_camera (either precision, the
 * same argument checks), with no context: each camera carries its spin.  All
 * scratch lives in one file-scope device array of KERR_STATIC_SCRATCH_BYTES
 * that every GPU that loads the library holds until the process exits.
 * Limits: at most KERR_STATIC_MAX_GEODESICS rays and KERR_STATIC_MAX_CAMERAS
 * cameras per call (KERR_EINVAL beyond); outputs must be device memory
 * (KERR_EINVAL otherwise, since host buffers would need staging).  The
 * array's zone buffer holds one entry per geodesic, as the allocating entry
 * point's does.
 *
 * The first call on a device is the set-up: it looks up the array's device
 * address (cudaGetSymbolAddress) with that device current and caches it, and
 * the CUDA runtime loads the library's kernels on their first use (lazy
 * module loading) and places the array in device memory then -- driver
 * allocations that may synchronise the device.  Make that first call, in each
 * precision that will be used, during start-up and before any stream
 * capture; later calls allocate nothing.  The call is asynchronous on
 * `stream`.  Every call shares the array and leaves its contents there (the
 * counters are cleared at the start of each call), so calls that overlap on
 * the GPU -- on other streams or from other host threads -- race and must be
 * serialised by the caller.  Counters of the call are not reported
 * (kerr_get_stats needs a context). */
#define KERR_STATIC_MAX_GEODESICS 131072
#define KERR_STATIC_MAX_CAMERAS 64
#define KERR_STATIC_SCRATCH_BYTES 28315392
int kerr_trace_camera_static(const kerr_camera *cams, int32_t ncam, const kerr_opts *opts,
                             double *x_out, double *k_out, int32_t *status, int32_t *steps,
                             float *diag, float *cross, void *stream);

/* Host-writable abort flag of the context (a stop request with no
 * counterpart in the paper; the host side of its failure detection).  *flag
 * receives the address of an int32 in mapped pinned host memory, allocated
 * by the first call and owned by the context (freed by kerr_destroy).  While
 * it holds a non-zero value, every launch of this context's trace calls --
 * including one already running -- stops within a few dozen steps: lanes
 * poll the flag, warp by warp, every 32 iterations (the same place as the
 * budget_ns check); unfinished geodesics end with KERR_TIMEOUT and the state
 * reached, which kerr_trace_rays accepts to resume them.  No wait is
 * involved: a kernel that sees the flag finishes its current steps and
 * returns.  Write 0 to re-arm.  KERR_ENOMEM / KERR_ECUDA if the mapped
 * allocation fails. */
int kerr_abort_flag(kerr_ctx *ctx, int32_t **flag);

/* Allocation-failure injection for tests (host-side only; nothing on the GPU
 * faults): the n-th device allocation the library makes from now on (n >= 1)
 * reports cudaErrorMemoryAllocation without allocating, so the call that
 * needed it returns KERR_ENOMEM and leaves its context usable; n = 0
 * disarms.  Process-wide.  KERR_EINVAL for n < 0. */
int kerr_debug_fail_alloc(int32_t n);

/* Integrates rays from n image-plane points, each with its own camera:
 * points[4 * i + 0..3] = (alpha, beta, spin a, inclination) as in
 * kerr_camera (pixel (alpha, beta) of a camera at r_obs with that spin and
 * inclination).  Outputs as for kerr_trace_rays.  Used to generate the
 * surrogate's training rays, whose spins and inclinations vary per ray. */
int kerr_trace_points(kerr_ctx *ctx, const double *points, int64_t n, double r_obs,
                      const kerr_opts *opts, double *x_out, double *k_out, int32_t *status,
                      int32_t *steps, float *diag, float *cross, void *stream);

/* ------------------------------------------------------------------------ */
/* Learned surrogate (the paper has none): an MLP                            */
/*   (alpha/s, beta/s, a, cos i) -> 4 x 256 (SiLU) -> 8 outputs             */
/* (s = KERR_SURR_INPUT_SCALE) predicting the capture logit, the first two    */
/* equatorial crossings as (log-radius, cos phi, sin phi) and the redshift:   */
/*   out = (logit, (ln r1 - 2)/2, cos phi1, sin phi1, (ln r2 - 2)/2,          */
/*          cos phi2, sin phi2, g1 - 1).                                     */
/* Weights are BF16 in the products, FP32 master copies are trained; every    */
/* matrix product runs on the tensor cores with FP32 accumulation.           */
/* Parameters are one FP32 vector: for layer l = 0..4, W_l [out][in] then     */
/* b_l [out] with padded widths in = 16, 256, 256, 256, 256 and out = 256,    */
/* 256, 256, 256, 64 (only 4 inputs and 8 outputs are live; the padding must  */
/* be zero).  All pointers of the surrogate calls are device memory except    */
/* where "host" is stated.                                                    */
/* ------------------------------------------------------------------------ */
#define KERR_SURR_INPUT_SCALE 25.0f
#define KERR_SURR_OUTPUTS 8
typedef struct kerr_surrogate kerr_surrogate;

/* Number of floats in the parameter vector. */
int64_t kerr_surrogate_num_params(void);

/* Creates a surrogate on the current device from host parameters `init`
 * (kerr_surrogate_num_params() floats; initial values are the caller's --
 * e.g. seeded random numbers). */
int kerr_surrogate_create(const float *init, kerr_surrogate **out);
int kerr_surrogate_destroy(kerr_surrogate *s);

/* Copies the FP32 parameters (or the last computed gradient) to host. */
int kerr_surrogate_get_params(kerr_surrogate *s, float *host_out);
int kerr_surrogate_get_grad(kerr_surrogate *s, float *host_out);

/* Parameter files (host code only; no GPU needed): a 96-byte little-endian
 * header -- magic "KERRSURR", version 1, header size, number of parameters,
 * layer count, the padded input and output widths of the five layers, the
 * live input and output widths, KERR_SURR_INPUT_SCALE, an FNV-1a checksum of
 * the parameter bytes, 12 reserved zero bytes -- followed by the
 * kerr_surrogate_num_params() FP32 parameters in the order described above.
 * kerr_params_write writes n == kerr_surrogate_num_params() host floats;
 * kerr_params_read checks every header field, the length and the checksum
 * (KERR_EINVAL naming what differs) before filling `params`.  Save/load
 * move a surrogate's FP32 master parameters through such a file (load
 * creates a new surrogate on the current device; optimizer moments are not
 * stored). */
int kerr_params_write(const char *path, const float *params, int64_t n);
int kerr_params_read(const char *path, float *params, int64_t n);
int kerr_surrogate_save(kerr_surrogate *s, const char *path);
int kerr_surrogate_load(const char *path, kerr_surrogate **out);

/* Network inputs and training targets from points (device, [n][4] doubles as
 * for kerr_trace_points): in [n][4] = (alpha/s, beta/s, a, cos i); the rays
 * are integrated (opts) with crossing labels, and targets [n][8] / masks
 * [n][8] are filled in the output encoding above (mask 0 where a crossing or
 * g1 is absent; the logit target is 1 for captured rays). */
int kerr_surrogate_targets(kerr_ctx *ctx, const double *points, int64_t n, double r_obs,
                           const kerr_opts *opts, float *in, float *targets, float *mask,
                           void *stream);

/* Forward pass: out [n][8] from in [n][4] (device buffers), on the fused
 * tensor-core kernel: all five layers per 128-row tile, tcgen05 MMAs with
 * the accumulator in tensor memory, weights staged by bulk TMA copies.
 * Synchronises `stream`; KERR_ECUDA if the kernel's pipeline timed out. */
int kerr_surrogate_forward(kerr_surrogate *s, const float *in, int64_t n, float *out,
                           void *stream);

/* The same forward on a chosen implementation: KERR_SURR_FWD_TENSOR_CORE
 * (as kerr_surrogate_forward) or KERR_SURR_FWD_GEMM (the layer-by-layer
 * tcgen05 GEMM kernels of the training path, one launch per layer).  Both
 * compute bf16 operands with fp32 accumulation; results differ by
 * accumulation order only.  Both synchronise `stream` and return KERR_ECUDA
 * if a tensor-core pipeline wait timed out. */
#define KERR_SURR_FWD_TENSOR_CORE 0
#define KERR_SURR_FWD_GEMM 1
int kerr_surrogate_forward_impl(kerr_surrogate *s, const float *in, int64_t n, float *out,
                                int32_t impl, void *stream);

/* Loss and gradient of one batch (kept in the surrogate; read it with
 * kerr_surrogate_get_grad).  Loss = mean over rows of
 *   softplus(o0) - y0 o0  +  sum_{j=1..7} m_j (o_j - y_j)^2.
 * *loss (host) receives the value; the call synchronises `stream`. */
int kerr_surrogate_grad(kerr_surrogate *s, const float *in, const float *targets,
                        const float *mask, int64_t n, float *loss, void *stream);

/* Training implementations.  KERR_SURR_TRAIN_FUSED (the default of
 * kerr_surrogate_grad and kerr_surrogate_train): three kernels per step --
 * one CTA per 128-row tile runs the five forward layers, the loss and the four
 * backward layers through the hidden weights with every activation in shared
 * memory and every accumulator in tensor memory; one launch contracts the
 * stored activations and gradients over the batch into all weight and bias
 * gradients; one launch applies Adam and refreshes the bf16 weights.
 * KERR_SURR_TRAIN_GEMM: the layer-by-layer tcgen05 GEMMs (about twenty
 * launches per step).  Both use bf16 operands with fp32 accumulation, bias
 * and SiLU in fp32, bf16 activations and backward signals; their gradients
 * differ by accumulation order only. */
#define KERR_SURR_TRAIN_FUSED 0
#define KERR_SURR_TRAIN_GEMM 1
int kerr_surrogate_grad_impl(kerr_surrogate *s, const float *in, const float *targets,
                             const float *mask, int64_t n, float *loss, int32_t impl,
                             void *stream);

/* Trains with Adam (beta1 0.9, beta2 0.999, eps 1e-8) on n rows for `epochs`
 * passes in order, `batch` rows per step, learning rate lr decayed by cosine
 * to lr/20 over all steps.  loss_per_epoch (host, `epochs` floats, or NULL)
 * receives the mean batch loss of each epoch.  The steps run on a private
 * stream ordered after `stream`, replayed from a CUDA graph captured by the
 * call (the per-step batch offset, schedule and bias corrections are read on
 * the device).  Synchronises `stream`; KERR_ECUDA if a launch failed or a
 * tensor-core pipeline wait timed out. */
int kerr_surrogate_train(kerr_surrogate *s, const float *in, const float *targets,
                         const float *mask, int64_t n, int32_t epochs, int32_t batch, float lr,
                         float *loss_per_epoch, void *stream);
/* kerr_surrogate_train on a chosen implementation (KERR_SURR_TRAIN_*). */
int kerr_surrogate_train_impl(kerr_surrogate *s, const float *in, const float *targets,
                              const float *mask, int64_t n, int32_t epochs, int32_t batch,
                              float lr, float *loss_per_epoch, int32_t impl, void *stream);

/* Renders a camera with the surrogate: the network predicts every pixel; a
 * pixel falls back to the integrator (opts, with crossing labels) when its
 * capture probability lies in [p_lo, p_hi] or its image-plane distance to the
 * Bardeen critical curve of (cam->a, cam->incl) is below crit_dist.
 * out [6][n] planes (n = nx ny): capture probability, r1, phi1, r2, phi2, g1
 * (integrator pixels: probability 0 or 1 and the integrator's labels;
 * network pixels: decoded predictions, NaN where the network's own capture
 * probability is >= 0.5 for the crossing planes).  fallback[n] (uint8, or
 * NULL) marks integrator pixels; *n_fallback (host, or NULL) their count.
 * Synchronises `stream`. */
int kerr_surrogate_render(kerr_ctx *ctx, kerr_surrogate *s, const kerr_camera *cam,
                          const kerr_opts *opts, float p_lo, float p_hi, float crit_dist,
                          float *out, uint8_t *fallback, int64_t *n_fallback, void *stream);

/* Integrates n geodesics in the coordinate time t (Sec. 2.2, eq. geo_t):
 * state (x, y, z, v^x, v^y, v^z) with v = dx/dt, right-hand side
 * dv^i/dt = A^i(u) - v^i A^t(u) for u = (1, v), A the affine acceleration of
 * eqs. opt0/opti (the same function eq. geo_t writes in split-metric form).
 * Works for null and time-like geodesics alike.  x0: [4][n] start events
 * (t0, x, y, z), v0: [3][n] coordinate velocities; each geodesic runs from
 * its t0 to t_end[i] (t_end may be NULL: opts.t_end for all), forward or
 * backward in t.  Step control as for kerr_trace_rays on the six components;
 * a trial step never passes the end time, so the last step lands on it
 * exactly (no clipping needed).  Statuses: KERR_ENDTIME (t = t_end),
 * KERR_CAPTURED (r < 1.01 r_h after a step), KERR_ESCAPED (r > r_esc while
 * moving outward in the direction of integration), KERR_MAXSTEPS,
 * KERR_NONFINITE.  Outputs: x_out [4][n] end events, v_out [3][n], status[n],
 * steps[n] (attempts).  opts: prec KERR_FP64, or KERR_FP32_KAHAN (FP32
 * arithmetic with compensated state updates everywhere: this entry point has
 * no FP64 zone), tol, h0, max_steps, r_escape, t_end.  All buffers device
 * memory (KERR_EINVAL otherwise); asynchronous on `stream`; statistics in
 * kerr_get_stats. */
int kerr_trace_coordtime(kerr_ctx *ctx, const double *x0, const double *v0,
                         const double *t_end, int64_t n, const kerr_opts *opts, double *x_out,
                         double *v_out, int32_t *status, int32_t *steps, void *stream);

/* kerr_trace_rays on the FP64 path (opts->prec must be KERR_FP64) that also
 * stores the solution: for geodesic i, records (lambda, t, x, y, z, k^t, k^x,
 * k^y, k^z) of the start state and after every accepted step (the last one
 * on the termination surface) into traj[i][0 .. cap-1][9] (device memory,
 * n * cap * 9 doubles; lambda counted from 0), with the number stored in
 * traj_count[i] (device; recording stops at cap).  Other arguments and
 * outputs as kerr_trace_rays (no diagnostics or crossings). */
int kerr_trace_rays_dense(kerr_ctx *ctx, const double *x0, const double *k0, int64_t n,
                          const kerr_opts *opts, int32_t cap, double *traj, int32_t *traj_count,
                          double *x_out, double *k_out, int32_t *status, int32_t *steps,
                          void *stream);

/* Root finding on a stored solution (Sec. 2.2, the second way of matching a
 * target time): for each geodesic, the first stored step across which t
 * passes t_target[i]; on it the state is the cubic Hermite interpolant of
 * both ends and their derivatives (dx/dlambda = k, dk/dlambda from eqs.
 * opt0/opti at spin a), and t(lambda) = t_target[i] is solved on it by a
 * bracketed Newton iteration (|t - t_target| <= 1e-13 (1 + |t_target|)).
 * Outputs (device): y_out [8][n] = (t, x, y, z, k^t, k^x, k^y, k^z),
 * lam_out [n], found [n] (1, or 0 with NaN outputs when the stored part of
 * the solution does not reach the target).  Asynchronous on `stream`. */
int kerr_dense_find_time(double a, const double *traj, int32_t cap, const int32_t *traj_count,
                         int64_t n, const double *t_target, double *y_out, double *lam_out,
                         int32_t *found, void *stream);

/* Paper-mode integration (Sec. 3, the timing setting of Sec. 4.2 and
 * Tables 2-3): every geodesic of `state` takes exactly nsteps classic RK4
 * steps of length h in place, with the right-hand side of eqs. opt0/opti,
 * no error control and no termination test (a geodesic that reaches the
 * singularity turns non-finite and keeps costing the same).  state: device
 * memory, n states (t, x, y, z, k^t, k^x, k^y, k^z) of float (fp64 =
 * KERR_FIXED_FP32: plain FP32 arithmetic, one geodesic per thread;
 * KERR_FIXED_FP32X2: the same FP32 steps for two geodesics per thread on
 * packed f32x2 instructions, equal to the one-per-thread results up to the
 * compiler's fusing of multiply-adds) or double (KERR_FIXED_FP64), in layout
 * KERR_LAYOUT_SOA ([8][n]) or KERR_LAYOUT_AOS ([n][8], 16-byte aligned).
 * Spin a, |a| <= 1.  Asynchronous on `stream`.  KERR_EINVAL for bad
 * arguments or host memory; n == 0 or nsteps == 0 is a no-op. */
#define KERR_LAYOUT_SOA 0
#define KERR_LAYOUT_AOS 1
#define KERR_FIXED_FP32 0
#define KERR_FIXED_FP64 1
#define KERR_FIXED_FP32X2 2
int kerr_rk4_fixed(double a, int32_t fp64, int32_t layout, void *state, int64_t n,
                   int32_t nsteps, double h, void *stream);

/* Paper mode in Boyer-Lindquist coordinates (eq. 1; the BL rows of the
 * paper's Tables 2-3, whose BL equations it does not print).  This library's
 * reading: the Hamiltonian form H = N / (2 Sigma) of the BL geodesic
 * equations, state (t, r, theta, phi, p_t, p_r, p_theta, p_phi) with covariant
 * momenta (p_t and p_phi stay constant).  Same arguments and behaviour as
 * kerr_rk4_fixed (KERR_FIXED_FP32 or KERR_FIXED_FP64 only); |a| < 1. */
int kerr_rk4_fixed_bl(double a, int32_t fp64, int32_t layout, void *state, int64_t n,
                      int32_t nsteps, double h, void *stream);

/* BL start states of a camera's rays for kerr_rk4_fixed_bl (this library's
 * reading of a distant observer at (r_obs, theta = incl, phi = 0, t = 0):
 * E = 1, L = -alpha sin(incl), Q = beta^2 + cos^2(incl) (alpha^2 - a^2),
 * p_theta = sign(beta) sqrt(Theta), p_r < 0 from H = 0), nx * ny states into
 * device `state` (float or double, SoA or AoS as for kerr_rk4_fixed).
 * |a| < 1, 0 < incl < pi, r_obs > 2.  Asynchronous on `stream`. */
int kerr_bl_camera_states(const kerr_camera *cam, int32_t fp64, int32_t layout, void *state,
                          void *stream);

/* Check of the integrator's FP64 reciprocal, reciprocal square root and
 * square root (Newton-refined hardware approximations, see the FP64 steps;
 * this library's own primitives, with no counterpart in the paper): for
 * device x[n] writes device out[3][n] = 1/x, 1/sqrt(x), sqrt(x) as the
 * integrator computes them (for finite x > 0; sqrt(0) = 0, and NaN or a
 * negative x gives NaN).  Asynchronous on `stream`.  KERR_EINVAL for
 * n < 0 or NULL buffers with n > 0; n == 0 is a no-op. */
int kerr_check_fp64_math(const double *x, int64_t n, double *out, void *stream);

/* Arithmetic peak of this GPU's FP32 or FP64 pipe (a measurement aid with no
 * counterpart in the paper: the integrator is bound by these pipes, and its
 * roofline fraction is taken against the rate this kernel reaches).  Launches
 * SMs x blocks_per_sm blocks of 256 threads, each thread running 8 independent
 * fused multiply-add chains for 16 x rounds steps: kind KERR_PEAK_FP32 (fma.f32),
 * KERR_PEAK_FP64 (fma.f64) or KERR_PEAK_FP32X2 (packed fma.f32x2, two per
 * instruction).  *flops (host, or NULL) receives the FLOPs the launch performs
 * (2 per fused multiply-add); the caller times the launch on `stream`.  sink:
 * device memory of at least SMs x blocks_per_sm x 256 floats (never written in
 * practice; it keeps the chains from being optimised away).  KERR_EINVAL for
 * an unknown kind, rounds < 1 or blocks_per_sm outside 1..8. */
#define KERR_PEAK_FP32 0
#define KERR_PEAK_FP64 1
#define KERR_PEAK_FP32X2 2
int kerr_fma_chain(int32_t kind, int64_t rounds, int32_t blocks_per_sm, float *sink,
                   double *flops, void *stream);

/* Message of the last failed call on this thread ("" if none). */
const char *kerr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* KERR_H */
