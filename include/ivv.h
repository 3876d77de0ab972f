/*
 * ivv.h -- C ABI of the GB300 isogeometric volume ray integrator.
 *
 * Renders multi-block trivariate B-spline volumes (geometry phi, scalar rho on
 * a common parameter domain P, Eq. 1 of Fuchs & Hjelmervik, "Interactive
 * Isogeometric Volume Visualization with Pixel-Accurate Geometry", TVCG 2015)
 * with the paper's three per-frame stages (§4):
 *   1. intersections of every pixel ray with the 6 boundary surfaces of every
 *      block (§4.1),
 *   2. per-pixel depth-sorted fragment lists and blockwise entry/exit pairing
 *      (§4.2, Alg. 2),
 *   3. for each entry/exit pair, the pulled-back view-ray ODE p' = W(p),
 *      J_phi(p) W = V(phi(p)) (§5.2, Eqs. 10-15), integrated by an embedded
 *      Runge-Kutta pair with error control, with the transfer function and
 *      front-to-back compositing with supersampling (§3.2.1, Alg. 1).
 *
 * Conventions shared by every entry point:
 *   - No function aborts, traps or prints.  Errors are returned as an
 *     ivv_status; ivv_last_error() gives a thread-local message.
 *   - Input arrays are copied at call time; the caller keeps ownership.
 *   - Device pointers are plain CUDA device addresses (e.g. a torch tensor's
 *     data_ptr()).  Streams are cudaStream_t passed as void*; NULL is the
 *     legacy default stream.  Work is enqueued asynchronously on that stream;
 *     only ivv_get_stats and the *_to_host entry point synchronise.
 *   - A volume handle may be used from one host thread at a time.
 *   - Images are float32 RGBA, row-major [height][width][4], row 0 at the
 *     top; colour is the accumulated C_dst of Alg. 1 (background 0), A is the
 *     accumulated opacity alpha_dst.
 */
#ifndef IVV_H
#define IVV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IVV_OK = 0,
  IVV_ERR_INVALID_ARG = 1,     /* bad pointer, size, knot vector, mode ...      */
  IVV_ERR_CUDA = 2,            /* a CUDA runtime call failed                     */
  IVV_ERR_OOM = 3,             /* device allocation failed                       */
  IVV_ERR_ABUF_OVERFLOW = 4,   /* a pixel had more fragments/pairs than stored   */
  IVV_ERR_NONCONVERGED = 5,    /* an iteration hit its cap (reported by stats)   */
  IVV_ERR_DEGENERATE = 6,      /* det J <= 0 inside a block (assumption 4, §5)   */
  IVV_ERR_UNSUPPORTED = 7,     /* e.g. degree > 3                                */
  IVV_ERR_WORKSPACE = 8        /* caller workspace too small or misaligned       */
} ivv_status;

/* Scalar field rho (§1, §6.1): */
enum {
  IVV_SCALAR_CP = 0,        /* rho from the scalar control points              */
  IVV_SCALAR_DETJ = 1,      /* rho = det J_phi, derived per sample              */
  IVV_SCALAR_QUALITY = 2,   /* rho = det J_phi / ||J_phi||_F  (Eq. 23)          */
  IVV_SCALAR_VONMISES = 3   /* rho = von Mises value of the strain of the
                               displacement u (§6.2, Eq. 24), per sample      */
};

/* Arithmetic of the ray stages: */
enum {
  IVV_PREC_FP32 = 0,    /* all kernels FP32                                       */
  IVV_PREC_MIXED = 1,   /* FP32, plus FP64 Newton residual for grazing hits and
                           an FP64 3x3 solve where |det J| < tau_det             */
  IVV_PREC_FP64 = 2     /* all kernels FP64                                       */
};

enum {
  IVV_FLAG_STATS = 1,    /* instrumented kernels: fill ivv_stats counters       */
  IVV_FLAG_TIMING = 2    /* record CUDA events between the stages of the render */
};

/* Stages timed with IVV_FLAG_TIMING (indices into ivv_get_stage_times). */
enum {
  IVV_STAGE_PROJECT = 0,     /* face patch screen boxes                         */
  IVV_STAGE_INTERSECT = 1,   /* ray/face intersections into fragment lists §4.1 */
  IVV_STAGE_PAIR = 2,        /* depth sort and Alg. 2 pairing §4.2              */
  IVV_STAGE_INTEGRATE = 3,   /* ODE integration and compositing §5.2, §3.2.1    */
  IVV_N_STAGES = 4
};

typedef struct ivv_volume ivv_volume;     /* opaque, library-owned */

/* One volume block (Eq. 1): a tensor-product B-spline of degrees degree[d]
 * with n_cp[d] control points per direction d (0=u, 1=v, 2=w).
 * knots[d]: n_cp[d] + degree[d] + 1 non-decreasing values, clamped (first and
 *   last degree[d]+1 equal); they are normalised to [0,1] (the paper clamps
 *   to [0,1]^3, §5.1 and §5.4).
 * geom_cp: [n_cp[2]][n_cp[1]][n_cp[0]][3] doubles, u fastest.
 * scalar_cp: [n_cp[2]][n_cp[1]][n_cp[0]] doubles; required for IVV_SCALAR_CP,
 *   ignored otherwise.
 * disp_cp: [n_cp[2]][n_cp[1]][n_cp[0]][3] doubles, the control points of the
 *   displacement field u: P -> R^3 of a structural analysis (§6.2) on the
 *   block's knots and degrees; required for IVV_SCALAR_VONMISES, ignored
 *   otherwise.  Per sample the library forms J_u J_phi^-1 (the Jacobian of
 *   u o phi^-1, whose transpose solves the paper's J_phi^T X = J_u^T), the
 *   strain tensor sigma = its symmetric part, and
 *   rho = sqrt(((s11-s22)^2 + (s22-s33)^2 + (s33-s11)^2
 *               + 6 (s12^2 + s23^2 + s31^2)) / 2).
 *   Batches (ivv_batch_create) do not take IVV_SCALAR_VONMISES volumes. */
typedef struct {
  int degree[3];
  int n_cp[3];
  const double* knots[3];
  const double* geom_cp;
  const double* scalar_cp;
  const double* disp_cp;
} ivv_block_desc;

/* Pinhole (ortho = 0) or orthographic (ortho = 1) camera.  The ray of pixel
 * (x, y) of a W x H image passes through ndc = ((x+.5)/W*2-1, 1-(y+.5)/H*2):
 * perspective: o = eye, d = normalize(f + ndc_x tan(fovy/2) (W/H) r
 *                                      + ndc_y tan(fovy/2) u);
 * orthographic: d = f, o = eye + ndc_x (h/2)(W/H) r + ndc_y (h/2) u,
 * with f = normalize(target - eye), r = normalize(f x up), u = r x f. */
typedef struct {
  int ortho;
  double eye[3], target[3], up[3];
  double fovy_deg;
  double ortho_height;
} ivv_camera;

/* Render parameters.  Pass NULL for the defaults in brackets.
 * rk_tol       absolute local error bound (inf-norm, parameter space) of the
 *              embedded Bogacki-Shampine 3(2) pair [1e-5]
 * ds           sample distance along the ray in G arc length; <= 0 selects
 *              diag/128, diag = diagonal of the control-point bounding box
 *              (§3.2.1; samples s_j = j ds, last interval partial)
 * supersample_k sub-samples per interval of the linearly interpolated scalar
 *              (§3.2.1 supersampling) [4]
 * c            weight of the perpendicular field V_perp (Eq. 10) [1]
 * early_alpha  stop a pixel once alpha_dst >= early_alpha [1 - 1e-4]
 * use_mlp_guess IVV_GUESS_* initial guess [0].  RF method: the Newton start
 *              of every sample.  Both methods: IVV_GUESS_MLP starts the
 *              stage-2 Newton solves that have no chord context -- entries
 *              on the near plane and entries moved off a singular face
 *              (§5.4) -- from the block's trained network (tensor-core
 *              inference on the list of those entries), falling back to the
 *              plain starts when Newton from it fails.  IVV_GUESS_CHORD is
 *              for the RF method only.
 * precision    IVV_PREC_* [FP32]
 * flags        IVV_FLAG_* [0]
 * x0, y0, full_width, full_height
 *              render the window [x0, x0+width) x [y0, y0+height) of a
 *              full_width x full_height image (0 = the window is the image)
 * method       IVV_METHOD_* [ODE]; RF runs in FP32 or MIXED precision, reads
 *              back the sample count (one stream synchronisation) and keeps
 *              its sample buffers (44 bytes per sample) in library memory
 * rf_tol       RF stopping rule: ||phi(p) - g|| <= rf_tol times the half width
 *              of the pixel at the sample's depth (the paper stops at the
 *              pixel frustum, rf_tol = 1) [0.05]
 * rk_method    IVV_RK_* integrator of the ODE method [IVV_RK_BS32]; the
 *              fixed-step family (§5.2-5.3) takes one step per sample interval
 *              (rk_tol unused) and runs in FP32 or MIXED precision
 * near_clip    > 0: near plane at this distance from the eye along the view
 *              direction (§5.5): intersections in front of it are dropped
 *              and a block whose nearest remaining intersection is an exit
 *              (the plane cuts through the block) is entered on the plane [0]
 *              (its parameter point by Newton from the exit point, or from
 *              the learned guess)
 * n_cut_planes, cut_planes
 *              up to IVV_MAX_CUT_PLANES cutting planes (§5.5), plane k as
 *              (n_x, n_y, n_z, w): the part of the volume with n.g + w > 0 is
 *              cut away, i.e. every entry/exit segment of a ray is shortened
 *              to n.g + w <= 0 [none].  An end point that moves onto a plane
 *              gets its parameter point by Newton (§5.1) from the chord of
 *              the segment; an entry on the near plane that does not invert
 *              inside its block drops its segment. */
typedef struct {
  double rk_tol;
  double ds;
  int supersample_k;
  double c;
  double early_alpha;
  int use_mlp_guess;
  int precision;
  int flags;
  int x0, y0, full_width, full_height;
  int method;
  double rf_tol;
  int rk_method;
  double near_clip;
  int n_cut_planes;
  double cut_planes[4][4];
} ivv_render_params;

#define IVV_MAX_CUT_PLANES 4

/* Integrators of the ODE method (rk_method): */
enum {
  IVV_RK_BS32 = 0,      /* embedded Bogacki-Shampine 3(2), error control, dense output */
  IVV_RK_EULER = 1,     /* fixed step: explicit Euler (the paper's RK1)         */
  IVV_RK_MIDPOINT = 2,  /* fixed step: explicit midpoint (RK2)                  */
  IVV_RK_KUTTA3 = 3,    /* fixed step: Kutta's third-order method (RK3)         */
  IVV_RK_RK4 = 4,       /* fixed step: classic fourth-order Runge-Kutta (RK4)   */
  IVV_RK_RK4_38 = 5,    /* fixed step: Kutta's 3/8 rule (RK4 3/8)               */
  IVV_RK_FEHLBERG5 = 6, /* fixed step: Fehlberg's pair, fifth-order weights (RKF) */
  IVV_RK_IMPLICIT_EULER = 7  /* fixed step: implicit Euler (IRK1), Newton with the
                                exact Jacobian of §5.2 (spline Hessian); use with
                                a large c (the paper's c = 100) */
};

/* Preimage methods of stage 3 (§5): */
enum {
  IVV_METHOD_ODE = 0,   /* pulled-back view-ray ODE, embedded RK (§5.2)         */
  IVV_METHOD_RF = 1     /* per-sample Newton root finding (§5.1), all samples in
                           parallel from an initial guess chosen by use_mlp_guess */
};

/* Initial guesses of the RF method (use_mlp_guess): */
enum {
  IVV_GUESS_CENTER = 0, /* parameter centre (1/2, 1/2, 1/2) of the block         */
  IVV_GUESS_MLP = 1,    /* the block's trained network (ivv_train_guess)         */
  IVV_GUESS_CHORD = 2   /* p_in + (s / L)(p_out - p_in) along the pair            */
};

/* Counters of the last instrumented render (IVV_FLAG_STATS) plus overflow
 * and cap counters of every render since the last ivv_reset_stats. */
typedef struct {
  unsigned long long rays;          /* pixels with >= 1 entry/exit pair        */
  unsigned long long pairs;         /* entry/exit pairs integrated             */
  unsigned long long fragments;     /* stored ray/face intersections           */
  unsigned long long samples;       /* scalar samples s_j composited           */
  unsigned long long rk_steps;      /* accepted RK steps                       */
  unsigned long long rk_rejects;    /* rejected RK steps                       */
  unsigned long long rhs_evals;     /* evaluations of W(p) in the integrator   */
  unsigned long long isect_newton;  /* Newton iterations of ray/face solves    */
  unsigned long long isect_tests;   /* ray/face pairs that passed the hull test */
  unsigned long long fp64_solves;   /* FP64 fallbacks (mixed precision)        */
  unsigned long long abuf_overflow; /* fragments dropped (list full)           */
  unsigned long long pair_overflow; /* pairs dropped (list full)               */
  unsigned long long unmatched;     /* records left unpaired by Alg. 2          */
  unsigned long long step_cap;      /* pairs that hit the RK step cap          */
  unsigned long long rf_newton_iters; /* RF: Newton iterations over all samples */
  unsigned long long rf_unconverged;  /* RF: samples that missed the tolerance  */
  unsigned long long isect_items;   /* (pixel, patch) candidates after the box tests */
  unsigned long long isect_split;   /* candidates that needed the subdivision search */
  unsigned long long rho_evals;     /* samples whose scalar was evaluated on its own (shading pass) */
  unsigned long long entry_shrinks; /* entries with a singular Jacobian moved into the block (§5.4, Eq. 22) */
  unsigned long long entry_newton;  /* Newton iterations of the stage-2 fix-up solves (§5.4, §5.5) */
  unsigned long long async_timeouts; /* bounded waits for tensor-core work that gave up (a device fault) */
  double max_delta_p;               /* max pixel-accuracy error Delta P (Eq. 5) */
} ivv_stats;

/* Build a volume from n_blocks blocks (§4: multi-block models): validate,
 * normalise knots, Bezier-extract every block by knot insertion, elevate all
 * blocks to a common degree P in {2, 3}, extract the 6 boundary faces of
 * every block as Bezier face patches with outward orientation, check
 * det J > 0 at sample points (§5 assumption 4), and upload to the device on
 * `stream` (synchronised before return).  Returns IVV_ERR_DEGENERATE if
 * det J <= 0 is found, IVV_ERR_UNSUPPORTED for degrees > 3. */
ivv_status ivv_create_volume(const ivv_block_desc* blocks, int n_blocks, int scalar_mode,
                             void* stream, ivv_volume** out);

/* Piecewise-linear transfer function (§3.1, Eq. 4): n_knots (2..256) knots
 * r[i] ascending with r[0] = 0 and r[n-1] = 1; rgba [n][4]: emitted colour
 * C_src and extinction weight A in [0,1].  Per sample, with
 * x = clamp((rho - lo) / (hi - lo), 0, 1): alpha_src = 1 - exp(-sigma A xi),
 * so Alg. 1's T = (1 - alpha_src)^(ds_i / xi) = exp(-sigma A ds_i).
 * lo >= hi (or NaN) selects the default range: min/max of the scalar control
 * points, or of the derived scalar over a 64^3 grid of sample points of every
 * block.  Host arrays, copied. */
ivv_status ivv_set_transfer_function(ivv_volume* vol, int n_knots, const float* r, const float* rgba,
                                     float sigma, float lo, float hi);

/* The scalar range in use (after ivv_set_transfer_function). */
ivv_status ivv_get_scalar_range(const ivv_volume* vol, double* lo, double* hi);

/* Bytes of device workspace ivv_render needs for a width x height window at
 * the given precision (fragment lists, pair lists, queues, counters).
 * Windows are limited to 2^27 pixels (IVV_ERR_INVALID_ARG beyond). */
ivv_status ivv_workspace_size(const ivv_volume* vol, int width, int height, int precision,
                              size_t* bytes);

/* Render a width x height window (at most 2^27 pixels) into out_rgba
 * (device, caller-owned, [height][width][4] float32).  workspace: device
 * buffer of at least ivv_workspace_size bytes, 256-byte aligned; NULL makes
 * the library use a buffer it owns (grown with cudaMalloc outside of any
 * stream capture).  The FP32 / MIXED ODE method also keeps a sample buffer
 * per volume (16 bytes per sample, grown with cudaMalloc).  All work is
 * enqueued on `stream` and nothing is synchronised, except that a window
 * whose sample bound exceeds 4 GiB (e.g. 3840x2160 at ds = diag/128) reads
 * its sample total back once (synchronising `stream`; under a stream
 * capture such a window takes the fused integrator instead). */
ivv_status ivv_render(ivv_volume* vol, const ivv_camera* cam, const ivv_render_params* params,
                      int width, int height, float* out_rgba, void* workspace,
                      size_t workspace_bytes, void* stream);

/* Render a small window without allocating device memory.  For callers that
 * cannot call cudaMalloc at render time: real-time or plug-in hosts whose
 * memory is owned by a pool or budget of their own, and threads that must not
 * risk the implicit device synchronisation an allocation may cause.  The paper has no
 * counterpart; this is a deployment variant of ivv_render.
 * The per-frame workspace lives in a file-scope device array of 12 MiB
 * (IVV_NOALLOC_SCRATCH_BYTES), enough for a 64 x 64 window at any precision
 * with up to 16384 face patches; every GPU that loads the library keeps that
 * array until the process exits.  Larger windows return IVV_ERR_WORKSPACE
 * with the required size in ivv_last_error(); use ivv_render for them.
 * Only the ODE method is rendered here (every rk_method and precision, with
 * the fused integrators, which need no sample buffer); the RF method sizes
 * its sample buffers from a read-back and returns IVV_ERR_UNSUPPORTED.
 * The volume (created earlier) and out_rgba (device, caller-owned,
 * [height][width][4] float32) are the caller's.  Every call looks up the
 * array's address in the current device's context (cudaGetSymbolAddress);
 * the first call on a device may load the library's device code.  All calls
 * share the one array, whose contents
 * persist between calls (everything a frame needs zeroed is cleared by the
 * frame itself), so calls that overlap on the GPU -- on different streams or
 * from different threads -- race: serialise them. */
#define IVV_NOALLOC_SCRATCH_BYTES (12u << 20)
ivv_status ivv_render_noalloc(ivv_volume* vol, const ivv_camera* cam, const ivv_render_params* params,
                              int width, int height, float* out_rgba, void* stream);

/* As ivv_render, but out_rgba_host is host memory (pinned for full speed);
 * the image is rendered into library-owned device memory, copied back with
 * cudaMemcpyAsync on `stream`, and the stream is synchronised. */
ivv_status ivv_render_to_host(ivv_volume* vol, const ivv_camera* cam, const ivv_render_params* params,
                              int width, int height, float* out_rgba_host, void* stream);

/* As ivv_render_to_host, without waiting: the frame is rendered on `stream`
 * into one of two library-owned device images (used in turn) and copied to
 * out_rgba_host (pinned host memory, [height][width][4] float32) on a
 * library stream once the render is done, so the copy of one frame runs
 * while the next one renders.  out_rgba_host must not be read or reused
 * before ivv_render_to_host_wait returns; a frame's image is rendered only
 * after the copy that last used the same device image has finished.  Errors
 * as ivv_render (IVV_ERR_WORKSPACE: growing an image inside a stream
 * capture). */
ivv_status ivv_render_to_host_async(ivv_volume* vol, const ivv_camera* cam, const ivv_render_params* params,
                                    int width, int height, float* out_rgba_host, void* stream);

/* Blocks until every copy queued by ivv_render_to_host_async on this volume
 * has reached the host. */
ivv_status ivv_render_to_host_wait(ivv_volume* vol);

/* Stages 1-2 only (§4.1, §4.2): the per-pixel entry/exit pairs in
 * front-to-back order.  Device outputs, caller-owned:
 *   pair_count [height*width] int32,
 *   pairs      [max_pairs][height*width][8] float32 per pixel and slot:
 *              (p_in.u, p_in.v, p_in.w, t_in, p_out.u, p_out.v, p_out.w, t_out)
 *              (FP32 and MIXED; FP64 precision is rejected here),
 *   pair_block [max_pairs][height*width] int32.
 * max_pairs must be >= 1; pairs beyond it are dropped and counted. */
ivv_status ivv_render_pairs(ivv_volume* vol, const ivv_camera* cam, const ivv_render_params* params,
                            int width, int height, int max_pairs, int* pair_count, float* pairs,
                            int* pair_block, void* workspace, size_t workspace_bytes, void* stream);

/* Spline evaluation on the device (Eq. 1 with the Bezier-extracted blocks):
 * p [n][3] device float32 parameter points of one block; outputs (device,
 * any may be NULL): phi [n][3], jac [n][3][3] (jac[r][c] = d phi_r/d p_c),
 * rho [n] (per the volume's scalar mode). */
ivv_status ivv_eval_points(ivv_volume* vol, int block, int n, const float* p, float* phi,
                           float* jac, float* rho, void* stream);

/* Host-only FP64 evaluation of the library's own representation of a
 * volume description (Bezier elements after knot insertion and degree
 * elevation, Eq. 1): no device is used.  p [n][3] parameter points of block
 * `block` in [0,1]^3; outputs (any may be NULL): phi [n][3], jac [n][3][3],
 * rho [n] per scalar_mode.  Runs the whole host preparation, so it validates
 * a description exactly as ivv_create_volume would. */
ivv_status ivv_host_eval(const ivv_block_desc* blocks, int n_blocks, int scalar_mode, int block, int n,
                         const double* p, double* phi, double* jac, double* rho);

/* Host execution of the stage 1-2 code that ivv_render runs on the device
 * (face boxes, ray/patch roots, fragments, depth sort and Alg. 2), for a
 * width x height window: inspection and CPU testing of a volume description;
 * ivv_render never uses it.  Host outputs, caller-owned, same layout as
 * ivv_render_pairs but double: pair_count [height*width],
 * pairs [max_pairs][height*width][8], pair_block [max_pairs][height*width]. */
ivv_status ivv_host_render_pairs(const ivv_block_desc* blocks, int n_blocks, int scalar_mode,
                                 const ivv_camera* cam, const ivv_render_params* params, int width,
                                 int height, int max_pairs, int* pair_count, double* pairs,
                                 int* pair_block);

/* Milliseconds of each stage of the last render made with IVV_FLAG_TIMING
 * (ms[IVV_N_STAGES], CUDA events on the render stream); synchronises that
 * stream.  Returns IVV_ERR_INVALID_ARG if no timed render was made. */
ivv_status ivv_get_stage_times(ivv_volume* vol, float* ms);

/* ---------------------------------------------------------------------------
 * Learned initial guess of the inverse geometry map (not in the paper).
 * Per block, a 3-64-64-3 perceptron (ReLU) maps g_hat = (g - c) * inv_h (per
 * axis), the world point normalised to the block's control-point box
 * [-1,1]^3, to a parameter guess p_hat.  Parameters are one flat float vector of IVV_GUESS_PARAMS
 * values: W1 [64][3], b1 [64], W2 [64][64], b2 [64], W3 [3][64], b3 [3].
 * ------------------------------------------------------------------------- */
#define IVV_GUESS_PARAMS 4611

typedef struct {
  int samples_per_block;   /* forward-map samples per block [1 << 20]        */
  int epochs;              /* passes over the samples [8]                     */
  int batch;               /* mini-batch size, multiple of 128 [4096]         */
  float lr;                /* Adam learning rate, cosine-decayed to lr/10 [3e-3] */
  unsigned long long seed; /* sample and initialisation seed [1]              */
} ivv_guess_train_params;

/* Train every block's network on the device: samples p uniform in [0,1]^3
 * (counter-based hash of (seed, block, index)), targets from g = phi(p)
 * evaluated by the library's spline kernels; Adam on the mean squared error.
 * final_loss (host, [n_blocks], may be NULL) receives each block's mean loss
 * over its first 65536 samples after training.  Allocates its sample buffers
 * (samples_per_block * 32 bytes) for the duration of the call; synchronises
 * `stream`. */
ivv_status ivv_train_guess(ivv_volume* vol, const ivv_guess_train_params* params, float* final_loss,
                           void* stream);

/* Tensor-core inference (FP16 weights, FP32 accumulation): g [n][4] device
 * floats (x, y, z, ignored) of points in the blocks block_of [n] (device
 * int32); p_out [n][4] device floats (p_hat, 0).  Needs trained or set
 * weights (IVV_ERR_INVALID_ARG otherwise). */
ivv_status ivv_guess_points(ivv_volume* vol, int n, const float* g, const int* block_of, float* p_out,
                            void* stream);

/* Inverse geometry map of world points (§5.1, Eq. 6 solved per point): g
 * [n][4] device floats (x, y, z, ignored) lying in blocks block_of [n]
 * (device int32); damped Newton with a halving line search from the initial
 * guess `guess` (IVV_GUESS_CENTER or IVV_GUESS_MLP) until ||phi(p) - g|| <=
 * tol (not below FP32 resolution).  p_out [n][4] device floats receives
 * (p, ||phi(p) - g||); iters [n] device int32 (may be NULL) the Newton
 * iterations used, or -1 - iterations where the tolerance was not reached.
 * Enqueued on `stream`. */
ivv_status ivv_invert_points(ivv_volume* vol, int n, const float* g, const int* block_of, int guess, float tol,
                             float* p_out, int* iters, void* stream);

/* One forward/backward pass of the training kernel (no update) on caller
 * samples of one block: x_hat [n][4] and p [n][4] device floats (normalised
 * inputs and targets).  grad (host, [IVV_GUESS_PARAMS]) and loss (host)
 * receive the gradient and value of the mean squared error.  Synchronises. */
ivv_status ivv_guess_loss_grad(ivv_volume* vol, int block, int n, const float* x_hat, const float* p,
                               float* grad, float* loss, void* stream);

/* Host copies of one block's parameters and normalisation (c[3], inv_h[3]). */
ivv_status ivv_get_guess_weights(ivv_volume* vol, int block, float* params, float* c, float* inv_h);
ivv_status ivv_set_guess_weights(ivv_volume* vol, int block, const float* params);

/* Capacities and iteration caps of a volume's renders (not in the paper:
 * the paper's linked-list A-buffer and shaders state none).  Pass NULL to
 * ivv_set_limits for the defaults in brackets; smaller values exist to
 * exercise the overflow and cap paths (a frame never faults on them: what
 * does not fit is dropped and counted).
 * max_frags        fragment slots per pixel, 1..32 [32]; hits beyond them
 *                  are dropped (ivv_stats.abuf_overflow)
 * max_pairs        entry/exit pair slots per pixel, 1..16 [16]; pairs beyond
 *                  them are dropped (ivv_stats.pair_overflow)
 * items_per_pixel  capacity of the (pixel, face patch) candidate list of
 *                  stage 1, per pixel of the window, 1..16 [16]; candidates
 *                  beyond it are dropped (ivv_stats.abuf_overflow)
 * max_rk_steps     RK steps per entry/exit pair of the error-controlled
 *                  integrator, >= 1 [200000]; a pair that reaches it ends
 *                  at its exit point (ivv_stats.step_cap)
 * max_newton       Newton iterations per sample of the RF method and per point
 *                  of ivv_invert_points, 1..64 [16]; a sample that misses
 *                  its tolerance is counted (ivv_stats.rf_unconverged) */
typedef struct {
  int max_frags;
  int max_pairs;
  int items_per_pixel;
  int max_rk_steps;
  int max_newton;
} ivv_limits;

ivv_status ivv_set_limits(ivv_volume* vol, const ivv_limits* limits);
ivv_status ivv_get_limits(const ivv_volume* vol, ivv_limits* limits);

/* Status of the renders since the last ivv_check_frame (or ivv_reset_stats):
 * synchronises the stream of the last render and reads the overflow and cap
 * counters that every render keeps.  Returns IVV_ERR_CUDA if a bounded
 * wait for tensor-core work gave up, else IVV_ERR_ABUF_OVERFLOW if any
 * fragment, pair or stage-1 candidate was dropped, else IVV_ERR_NONCONVERGED
 * if an entry/exit pair hit the RK step cap or an RF sample missed its
 * tolerance, else IVV_OK; ivv_last_error() names the counts.  The images
 * stay valid: only the pixels concerned lack the dropped parts. */
ivv_status ivv_check_frame(ivv_volume* vol);

/* Counters (see ivv_stats); synchronises the stream of the last render. */
ivv_status ivv_get_stats(ivv_volume* vol, ivv_stats* out);
ivv_status ivv_reset_stats(ivv_volume* vol);

/* Volume facts: blocks, Bezier elements, face patches, common degree P. */
ivv_status ivv_volume_info(const ivv_volume* vol, int* n_blocks, int* n_elements, int* n_faces,
                           int* degree);

/* ---------------------------------------------------------------------
 * Batched rendering: many views of several volumes, of uneven image sizes,
 * in one launch per stage, replayed from a captured CUDA graph.
 *
 * At creation every distinct volume of the batch is copied into one device
 * pool (blocks, Bezier elements, face patches and breakpoints concatenated
 * with rebased offsets), so a ray of any request finds its geometry through
 * the pool's block table alone.  The stages then run once over the whole
 * batch: K0 over every (request, face), K2 over every screen tile of every
 * request, K4 over every pixel, and the persistent K5 over one work queue
 * that spans all requests, so rays of short and long requests share the
 * machine until the last one finishes.  The library owns the workspace
 * (about 1.4 KB per pixel: fragment slots, stage-1 items and pair slots).
 * The volumes may be destroyed after creation; all of them must share the
 * common degree P (IVV_ERR_UNSUPPORTED otherwise). */
typedef struct ivv_batch ivv_batch;       /* opaque, library-owned */

#define IVV_BATCH_TF_MAX 64               /* knots of a per-request TF     */
#define IVV_BATCH_MAX_REQUESTS 4096      /* and fewer than 2^27 pixels in all */

/* One render request.
 * volume      a created volume; its data is copied at ivv_batch_create
 * camera      see ivv_camera; may be changed later by ivv_batch_set_camera
 * width, height  image size; the whole image is rendered
 * tf_n, tf_r, tf_rgba, tf_sigma, scalar_lo, scalar_hi
 *             the request's transfer function with the meaning of
 *             ivv_set_transfer_function (tf_n <= IVV_BATCH_TF_MAX knots);
 *             tf_r == NULL takes the volume's current transfer function and
 *             range, scalar_lo >= scalar_hi the volume's default range
 * out_rgba    device pointer, caller-owned, [height][width][4] float32,
 *             16-byte aligned; written by every ivv_batch_render */
typedef struct {
  const ivv_volume* volume;
  ivv_camera camera;
  int width, height;
  int tf_n;
  const float* tf_r;
  const float* tf_rgba;
  float tf_sigma;
  double scalar_lo, scalar_hi;
  float* out_rgba;
} ivv_request;

/* Launch shapes chosen by the autotuner.
 * tile_w, tile_h   K2 culling tile (one warp, one lane per pixel): 8x4, 4x8
 *                  or 16x2 [8x4]
 * k5_ctas_per_sm   resident CTAs of the persistent K5 per SM, 1..4 [4]
 * step_samples     the step batch: the longest RK step, in sample distances
 *                  (samples inside a step come from dense output), one of
 *                  4, 8, 16 [8] */
typedef struct {
  int tile_w, tile_h;
  int k5_ctas_per_sm;
  int step_samples;
} ivv_batch_tuning;

/* Build a batch of n requests (1..IVV_BATCH_MAX_REQUESTS) rendered with the
 * shared parameters `params` (NULL: defaults; method ODE with rk_method
 * IVV_RK_BS32, precision FP32 or MIXED, no window, no cutting or near-clip
 * planes; ds <= 0 gives each request its volume's diag/128; anything else is
 * IVV_ERR_UNSUPPORTED).  Uploads the pool and the request table on `stream`
 * and synchronises it.  The first render also sizes the batch's sample
 * buffer (one eager pass of stages 1-2 and a read-back of the sample total,
 * synchronising `stream` once). */
ivv_status ivv_batch_create(const ivv_request* requests, int n, const ivv_render_params* params, void* stream,
                            ivv_batch** out);

/* Render every request of the batch on `stream`.  flags = 0 replays the
 * batch's CUDA graph (captured on the first call and again after a tuning
 * change); IVV_FLAG_STATS and/or IVV_FLAG_TIMING launch the same stages
 * directly, with counters (ivv_batch_get_stats) or per-stage events
 * (ivv_batch_get_stage_times). */
ivv_status ivv_batch_render(ivv_batch* batch, int flags, void* stream);

/* Replace the camera of request i (enqueued on `stream`; the graph reads the
 * request table from device memory, so no re-capture is needed). */
ivv_status ivv_batch_set_camera(ivv_batch* batch, int i, const ivv_camera* camera, void* stream);

ivv_status ivv_batch_set_tuning(ivv_batch* batch, const ivv_batch_tuning* tuning);
ivv_status ivv_batch_get_tuning(const ivv_batch* batch, ivv_batch_tuning* tuning);

/* Time the candidate launch shapes on this batch (reps timed renders each,
 * after one warm-up, CUDA events on `stream`): the K2 culling tile by the
 * surface stage's time, then the K5 CTAs per SM and step batch by the
 * integration stage's time.  Applies and returns the fastest; *best_ms is the
 * frame time with it.  Synchronises `stream`. */
ivv_status ivv_batch_autotune(ivv_batch* batch, int reps, ivv_batch_tuning* best, float* best_ms, void* stream);

/* Counters of the batch (see ivv_stats); synchronises the last stream. */
ivv_status ivv_batch_get_stats(ivv_batch* batch, ivv_stats* out);
ivv_status ivv_batch_reset_stats(ivv_batch* batch);
/* Stage times of the last IVV_FLAG_TIMING render, as ivv_get_stage_times. */
ivv_status ivv_batch_get_stage_times(ivv_batch* batch, float* ms);
/* Requests, total pixels, library workspace bytes, whether a graph exists. */
ivv_status ivv_batch_info(const ivv_batch* batch, int* n_requests, long long* n_pixels, size_t* workspace_bytes,
                          int* graph_ready);
void ivv_batch_destroy(ivv_batch* batch);

const char* ivv_last_error(void);
void ivv_destroy_volume(ivv_volume* vol);

#ifdef __cplusplus
}
#endif
#endif /* IVV_H */
