/*
 * nlinv.h -- C interface of the GB300 NLINV library.
 *
 * NLINV (Schaetz & Uecker, "A multi-GPU programming library for real-time applications", Sec. 3.1) reconstructs
 * an MRI image rho and the coil sensitivities c_j jointly from undersampled multi-coil k-space data y by solving
 * the nonlinear equation F x = y, with
 *
 *     F = P_k FFT M_Omega C W^-1                                                        (Eq. 2)
 *
 * by the iteratively regularised Gauss-Newton method
 *
 *     (DF^H DF + alpha_n I)(x_{n+1} - x_n) = DF^H (y - F x_n) - alpha_n (x_n - x_ref)  (Eq. 3)
 *
 * whose linear systems are solved by conjugate gradients.  Every step runs in hand-written sm_103a CUDA kernels.
 *
 * Conventions shared by every entry point
 *   - Complex values are interleaved single precision (nlinv_c32).  A "plane" is n x n values, row-major, in
 *     natural FFT order: index i holds the signed coordinate g(i) = i for i < n/2 and i - n otherwise.
 *   - The unknown x = (rho, chat_1 .. chat_J) is 1 + J planes: plane 0 is the image rho, planes 1..J the
 *     k-space coil coefficients chat_j, whose image-domain coil maps are c_j = W^-1 chat_j
 *     = FFT^-1(w . chat_j) with the Sobolev weight w(k) = (1 + a |k|^2)^(-l/2), |k| in cycles per grid width.
 *   - k-space data y, residuals and operator outputs in data space are J planes.
 *   - The sampling pattern P (P_k of Eq. 2) is one n x n plane of bytes, 0 or 1, shared by all coils.
 *   - M_Omega keeps the centred square -fov <= g < fov of the image (fov = n/4: the un-oversampled image of a 2x
 *     grid, Sec. 3.2).  FFT is the unitary 2D DFT (FFT^-1 = FFT^H).
 *   - Work is queued on the context's CUDA stream and returns before it finishes unless stated otherwise.
 *   - Unless stated otherwise, pointers are DEVICE pointers owned by the caller, valid until the work is done.
 *   - No entry point throws; every one returns an nlinv_status.  Arguments are checked on the host before any
 *     work is queued; on error nothing is queued and nlinv_last_error() describes the problem.
 *
 * Entry points, in the order below: contexts (nlinv_default_params, nlinv_create, nlinv_destroy); the operators
 * F, DF, DF^H, DF^H DF + alpha, the display image and data synthesis; the reconstruction of Eq. 3
 * (nlinv_reconstruct) and the gradient through it (nlinv_reconstruct_checkpoints, nlinv_reconstruct_vjp);
 * gridding of radial samples (nlinv_gridder_*); batches of independent frames (nlinv_batch_*); waiting,
 * per-kernel timing, the launch-shape autotuner and launch counts; F without a context or allocation
 * (nlinv_forward_noalloc); error messages.
 */
#ifndef NLINV_H
#define NLINV_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define NLINV_API __attribute__((visibility("default")))
#else
#define NLINV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  float x, y; /* real, imaginary */
} nlinv_c32;

typedef enum {
  NLINV_OK = 0,
  NLINV_EINVAL = 1,      /* bad argument (null pointer, unsupported size, host pointer where a device one is due) */
  NLINV_ENOMEM = 2,      /* device memory for the context's workspace could not be allocated */
  NLINV_ECUDA = 3,       /* a CUDA runtime call failed; nlinv_last_error() has its message */
  NLINV_EBREAKDOWN = 4,  /* CG met a non-finite |r|^2 or Re<p, A p>; that solve stopped there (no further step) */
  NLINV_ETIMEOUT = 5     /* nlinv_wait() gave up before the context's queued work finished */
} nlinv_status;

/* Problem and solver description (Sec. 3.1-3.2).  Fill with nlinv_default_params() and adjust. */
typedef struct {
  int n;             /* grid side (twice the image matrix, Sec. 3.2); see nlinv_supported_size() */
  int ncoils;        /* J >= 1 (virtual) coils */
  int newton_steps;  /* Gauss-Newton steps per reconstruction, 1..64 */
  int cg_iters;      /* CG iterations per Newton step (a fixed count; stops earlier only at the rounding floor,
                        see nlinv_cg_stops), >= 0 */
  double alpha0;     /* alpha_0 of Eq. 3 (> 0) */
  double alpha_q;    /* alpha_{n+1} = max(alpha_q alpha_n, alpha_min), 0 < alpha_q <= 1 */
  double alpha_min;  /* floor of alpha_n, >= 0 */
  double sobolev_a;  /* a of the Sobolev weight, >= 0 (220 in the real-time setting) */
  double sobolev_l;  /* l of the Sobolev weight, >= 0 (32) */
  int fov;           /* half-width of Omega in pixels, 1..n/2 (n/4 by default) */
  int use_graph;     /* 1: replay each reconstruction as one captured CUDA graph; 0: launch kernel by kernel */
  int tensor_dft;    /* 1: the radix-16 DFT stages of the transforms run on the tensor cores in split-BF16 with
                        three passes (an optional precision path beside the paper's complex single precision,
                        Sec. 3.2); compiled for n = 256 and 512; not used by batches.  0 (default): FP32 stages */
} nlinv_params;

typedef struct nlinv_ctx nlinv_ctx;

/* 1 if the grid side n has a compiled transform, else 0.  Supported: 16, 32, 48, 64, 80, 96, 128, 160, 192, 256,
 * 320, 384, 512. */
NLINV_API int nlinv_supported_size(int n);

/* Defaults for an n x n grid with ncoils coils: 7 Newton steps, 30 CG iterations, alpha_0 = 1, alpha_q = 1/2,
 * alpha_min = 0, a = 220, l = 32, fov = n/4, use_graph = 1, tensor_dft = 0.  EINVAL if p is NULL. */
NLINV_API nlinv_status nlinv_default_params(nlinv_params* p, int n, int ncoils);

/* Creates a context on the current CUDA device: validates *params, allocates the device workspace (about
 * 9 (1+J) n^2 complex values) and builds the transform tables.  stream is a cudaStream_t on which the context
 * queues its work; NULL makes the context create (and later destroy) a non-blocking stream of its own, since the
 * legacy default stream cannot be captured into a graph.  On success *out owns the context.  Blocks until set-up
 * is done.  Errors: EINVAL (bad params, NULL out), ENOMEM (the workspace allocation failed; the environment
 * variable NLINV_TEST_FAIL_ALLOC=1, for tests, makes it fail without trying), ECUDA. */
NLINV_API nlinv_status nlinv_create(const nlinv_params* params, void* stream, nlinv_ctx** out);

/* Waits for the context's stream, then frees the context and its workspace.  NULL is accepted. */
NLINV_API nlinv_status nlinv_destroy(nlinv_ctx* ctx);

/* F x of Eq. 2: y_out_j = P FFT(M rho c_j), c_j = W^-1 chat_j.  x: 1+J planes; y_out: J planes. */
NLINV_API nlinv_status nlinv_forward(nlinv_ctx* ctx, const nlinv_c32* x, const uint8_t* mask, nlinv_c32* y_out);

/* DF_x dx (the derivative of Eq. 3): out_j = P FFT(M (drho c_j + rho W^-1 dchat_j)).  x, dx: 1+J planes;
 * out: J planes. */
NLINV_API nlinv_status nlinv_derivative(nlinv_ctx* ctx, const nlinv_c32* x, const uint8_t* mask, const nlinv_c32* dx,
                              nlinv_c32* out);

/* DF_x^H r (the adjoint of Eq. 3): with z_j = M FFT^-1(P r_j), out plane 0 = sum_j conj(c_j) z_j (the channel
 * summation of Table 1) and out plane j = w . FFT(conj(rho) z_j).  x: 1+J planes; r: J planes; out: 1+J planes. */
NLINV_API nlinv_status nlinv_adjoint(nlinv_ctx* ctx, const nlinv_c32* x, const uint8_t* mask, const nlinv_c32* r,
                           nlinv_c32* out);

/* The left-hand operator of Eq. 3: out = (DF_x^H DF_x + alpha I) d.  x, d, out: 1+J planes. */
NLINV_API nlinv_status nlinv_normal(nlinv_ctx* ctx, const nlinv_c32* x, const uint8_t* mask, const nlinv_c32* d,
                          double alpha, nlinv_c32* out);

/* Display image of an estimate x (1+J planes): rho * sqrt(sum_j |c_j|^2) on Omega, the customary coil-combined
 * NLINV output (the paper does not describe its post-processing).  image_out: (2 fov) x (2 fov) complex values,
 * row-major and centred (row i, column k hold the signed coordinates i - fov, k - fov). */
NLINV_API nlinv_status nlinv_image(nlinv_ctx* ctx, const nlinv_c32* x, nlinv_c32* image_out);

/* Gridded data of the signal equation (Eq. 1) for image-domain coil maps: y_out_j = P FFT(M rho coil_img_j).
 * rho: one plane; coil_img: J planes; y_out: J planes.  Used to synthesise test and benchmark data. */
NLINV_API nlinv_status nlinv_simulate(nlinv_ctx* ctx, const nlinv_c32* rho, const nlinv_c32* coil_img, const uint8_t* mask,
                            nlinv_c32* y_out);

/* One reconstruction by Eq. 3: params.newton_steps Gauss-Newton steps with alpha_n = max(alpha_0 q^n, alpha_min),
 * each solved from dx = 0 by params.cg_iters CG iterations; x_{n+1} = x_n + dx.
 *   y        J planes of gridded data
 *   mask     sampling pattern
 *   x_ref    regularisation centre x_ref of Eq. 3 (1+J planes), or NULL to use the start value
 *   x_inout  on entry the start value x_0, on return x_N (1+J planes)
 *   resid    NULL, or a HOST array of newton_steps+1 doubles receiving |y - F x_n| for n = 0..N
 * For a real-time series pass the previous frame's result as x_inout (and x_ref NULL): the frame is then
 * initialised from and regularised toward it (Sec. 3.2).
 * Pointers here may be device pointers or host pointers (pageable or pinned); host buffers are copied through
 * the context's workspace.  The call returns after the work is queued, except that it waits for the stream when
 * resid is given or x_inout is host memory.  Errors: EINVAL, ECUDA; EBREAKDOWN when the call waited and CG broke
 * down (the result is still written). */
NLINV_API nlinv_status nlinv_reconstruct(nlinv_ctx* ctx, const nlinv_c32* y, const uint8_t* mask, const nlinv_c32* x_ref,
                               nlinv_c32* x_inout, double* resid);

/* ------------------------------------------------------------------- gradient through the reconstruction ----
 * The paper differentiates nothing; these two calls give the gradient of a real loss L(x_N) of the reconstruction
 * with respect to its data, start value and regularisation centre, for training systems that put NLINV inside a
 * larger model.  Every Gauss-Newton step of Eq. 3 is differentiated implicitly, its CG solve taken as exact (the
 * gradient of the method when CG has converged).  With A = DF^H DF + alpha_n I at x_n, dx_n = x_{n+1} - x_n and
 * s = y - F(x_n) - DF_{x_n} dx_n, one step backwards is: u = A^-1 g by the reconstruction's CG (params.cg_iters
 * iterations); dL/dy += DF_{x_n} u; dL/dx_ref += alpha_n u; g <- DF_u^H s - DF_{dx_n}^H DF_{x_n} u (F is bilinear).
 * Gradients are taken with respect to the real inner product Re sum conj(a) b (the convention of PyTorch's
 * complex autograd).  All pointers are DEVICE pointers; every call is queued on the context's stream. */

/* nlinv_reconstruct, plus the iterates x_0 .. x_N written to ckpt (DEVICE, (newton_steps+1) x (1+J) planes,
 * owned by the caller): the per-Newton-step checkpoints of the gradient.  Launches the passes one by one (no graph).
 * Waits for the stream only when resid (HOST, newton_steps+1 doubles) is given.  Errors: EINVAL (NULL or host
 * pointers), ECUDA; EBREAKDOWN when the call waited and CG broke down. */
NLINV_API nlinv_status nlinv_reconstruct_checkpoints(nlinv_ctx* ctx, const nlinv_c32* y, const uint8_t* mask,
                                                     const nlinv_c32* x_ref, nlinv_c32* x_inout, nlinv_c32* ckpt,
                                                     double* resid);

/* Backward pass from grad_x = dL/dx_N (1+J planes) over the checkpoints of nlinv_reconstruct_checkpoints with the
 * same y and mask.  Writes grad_y (J planes, zero off the sampling pattern), grad_x0 (1+J planes) and, unless
 * grad_xref is NULL, grad_xref (1+J planes).  tied = 1 when the reconstruction regularised toward its start value
 * (x_ref NULL): grad_x0 then receives dL/dx_0 + dL/dx_ref, the gradient with respect to that start value.  The
 * first call allocates 4 unknown-space vectors and 2 data arrays of scratch, held until nlinv_destroy.  The
 * context's workspace (and so the state left for nlinv_profile_cg) is overwritten.  Errors: EINVAL, ENOMEM,
 * ECUDA. */
NLINV_API nlinv_status nlinv_reconstruct_vjp(nlinv_ctx* ctx, const nlinv_c32* y, const uint8_t* mask,
                                             const nlinv_c32* ckpt, const nlinv_c32* grad_x, int tied,
                                             nlinv_c32* grad_y, nlinv_c32* grad_x0, nlinv_c32* grad_xref);

/* --------------------------------------------------------------------------------------------- gridding ----
 * Sec. 3.1 interpolates the measured radial samples onto the Cartesian grid on the CPU before the reconstruction,
 * without saying how.  Here it runs on the GPU as nearest-neighbour gridding with averaging: sample i of spoke s
 * lies at t_i d_s with t_i = -n/2 + i/2 (i < 2n) and d_s the spoke's unit direction; each coordinate goes to the
 * grid point floor(v + 1/2), the sample is kept when both lie in [-n/2, n/2), and a grid point (row = ky,
 * column = kx, natural FFT order) holds the mean of its samples (0 if none); the sampling pattern marks the grid
 * points that received a sample.  With the spoke angles of the real-time series this pattern is the one the
 * reconstruction's mask describes. */
typedef struct nlinv_gridder nlinv_gridder;

/* Builds the gridding of nspokes spokes of 2n samples on the n x n grid (n even, 8..2048).  directions (HOST,
 * 2 * nspokes doubles): (cos, sin) of each spoke's angle.  stream: a cudaStream_t, or NULL for a stream of its own.
 * Errors: EINVAL, ENOMEM, ECUDA (message in nlinv_last_error(NULL)). */
NLINV_API nlinv_status nlinv_gridder_create(int n, int nspokes, const double* directions, void* stream,
                                            nlinv_gridder** out);

/* y_out (DEVICE, ncoils x n x n) and mask_out (DEVICE, n x n) from samples (DEVICE, ncoils x nspokes x 2n, spoke-major
 * within a coil).  Queued on the gridder's stream.  Errors: EINVAL (NULL or host pointers, ncoils outside 1..64),
 * ECUDA. */
NLINV_API nlinv_status nlinv_grid(nlinv_gridder* g, int ncoils, const nlinv_c32* samples, nlinv_c32* y_out,
                                  uint8_t* mask_out);

/* Waits for the gridder's stream and frees it.  NULL is accepted. */
NLINV_API nlinv_status nlinv_gridder_destroy(nlinv_gridder* g);

/* ---------------------------------------------------------------------------------------------- batches ----
 * Many independent frames (slices, series of different patients, ...) of uneven grid side and coil count,
 * reconstructed together: every pass of Eq. 3 is one launch per grid side covering all frames of that side, and
 * the sides run as parallel branches of one captured graph.  Each frame has its own workspace and its own CG and
 * Newton scalars, so a frame's result is its single-frame reconstruction up to the summation order of the FP64
 * scalars (the block partition of a batched pass differs from a single-frame pass). */
typedef struct {
  int n;                    /* grid side of the frame (see nlinv_supported_size); fov = n/4 */
  int ncoils;               /* coils of the frame, 1..64 */
  const nlinv_c32* y;       /* J planes of gridded data */
  const uint8_t* mask;      /* sampling pattern */
  const nlinv_c32* x_ref;   /* regularisation centre (1+J planes) or NULL for the start value */
  nlinv_c32* x_inout;       /* start value in, result out (1+J planes) */
  double* resid;            /* NULL or a HOST array of newton_steps+1 doubles (|y - F x_n|) */
} nlinv_frame_desc;

typedef struct nlinv_batch nlinv_batch;

/* Creates a batch for nframes frames whose shapes are frames[i].n and frames[i].ncoils (the pointers are not used
 * here).  params supplies the solver schedule and the Sobolev weight (its n, ncoils, fov, use_graph and tensor_dft
 * are ignored).  stream as for nlinv_create.  Allocates one workspace per frame and captures the whole batched
 * reconstruction as one CUDA graph: per grid side, one persistent launch per pass (as many blocks as fit on the
 * GPU at once, each looping over the work items of all frames of that side), the sides as parallel branches.  With
 * the environment variable NLINV_BATCH_MULTI=1, the sides 128, 192, 256, 320 and 384 share one launch per pass
 * instead (a kernel that dispatches on each work item's side; slower on GB300: the side bodies spill registers).
 * Errors: EINVAL, ENOMEM, ECUDA (message via nlinv_last_error(NULL)). */
NLINV_API nlinv_status nlinv_batch_create(const nlinv_params* params, int nframes, const nlinv_frame_desc* frames,
                                          void* stream, nlinv_batch** out);

/* Reconstructs all frames (Eq. 3 with the batch's schedule): frames must have the shapes given at creation, in
 * the same order.  Pointers may be device or host memory as for nlinv_reconstruct.  Returns after queuing, unless
 * a resid array is given or an x_inout is host memory (then it waits).  Errors: EINVAL, ECUDA, EBREAKDOWN (any
 * frame, when the call waited). */
NLINV_API nlinv_status nlinv_reconstruct_batch(nlinv_batch* batch, int nframes, const nlinv_frame_desc* frames);

/* Times the batched kernels of one CG iteration (the second of the first Newton step) with CUDA events on the
 * batch's stream, on the workspaces left by the last nlinv_reconstruct_batch (whose CG state it advances; every
 * frame's solve is first marked running, so that each kernel does its full work): each kernel is launched for all
 * grid sides, one side after another, reps times back to back between two events.  ms_out (HOST, 6 doubles) gets
 * the mean duration of one launch set, in the order of nlinv_profile_cg.  Waits for the stream.  Errors: EINVAL
 * (reps < 1, NULL pointers, no reconstruction yet, fewer than two CG iterations), ECUDA. */
NLINV_API nlinv_status nlinv_batch_profile_cg(nlinv_batch* batch, int reps, double* ms_out);

/* Kernel launches of one batched reconstruction (the graph's kernel nodes); -1 for NULL. */
NLINV_API long nlinv_batch_launch_count(const nlinv_batch* batch);

/* Waits for the batch's stream and frees it.  NULL is accepted. */
NLINV_API nlinv_status nlinv_batch_destroy(nlinv_batch* batch);

/* Waits up to timeout_s seconds (< 0: no limit) for the context's queued work.  ETIMEOUT if it is still running,
 * EBREAKDOWN if a CG breakdown was flagged since the last check (the flag is then cleared), ECUDA on a CUDA
 * error or when a kernel's wait for its own asynchronous copies or tensor-core stage ran past its time limit (about
 * a second; the kernel then stopped waiting and its results are not valid). */
NLINV_API nlinv_status nlinv_wait(nlinv_ctx* ctx, double timeout_s);

/* Times the kernels of one CG iteration of Eq. 3 with CUDA events on the context's stream, on the workspace left
 * by the last nlinv_reconstruct (whose CG state it advances -- a solve that had stopped at its rounding floor is
 * marked running again, so that every kernel does its full work; x is not changed): each kernel is launched reps times
 * back to back between two events, so ms_out gets its steady-state launch duration (consecutive launches overlap
 * their ramp and drain, as the passes of a graph replay do; the first one and the CG step issue their loads of p, r and
 * dx after their wait here, since back to back each launch would read what the one before writes, while in a
 * reconstruction they issue them before).  With reps = 1 the six kernels run once each, in order.  ms_out (HOST, 6 doubles) receives the mean duration in milliseconds of, in order:
 *   [0] row pass  p = r + beta p, W^-1 (first axis)   [1] column pass  W^-1, C (products), FFT
 *   [2] row pass  PSF                                  [3] column pass  FFT^-1, C^H (channel products), FFT
 *   [4] row pass  W^-H + alpha p, Re<p, q>             [5] CG step  dx += alpha p, r -= alpha q, |r|^2
 * Waits for the stream.  Errors: EINVAL (reps < 1, NULL pointers, no reconstruction yet), ECUDA. */
NLINV_API nlinv_status nlinv_profile_cg(nlinv_ctx* ctx, int reps, double* ms_out);

/* Launch shapes picked by nlinv_autotune (one record per timed candidate in its table). */
typedef struct {
  int vec_blocks_per_sm;  /* blocks per SM of the vector passes (CG step, x update): 2, 4 or 8 */
  int pdl;                /* 1: passes use programmatic dependent launch */
  double ms_per_frame;    /* the measured time of one whole reconstruction with these shapes */
  int split_n1;           /* N1 of the four-step split n = N1 * N2 of the transforms */
  int col_strip;          /* adjacent columns per block of the column passes: 4, 8 or 16 */
  int row_blocks_per_sm;  /* row-pass blocks per SM: 1, 2 or 3 */
  int stage;              /* table entries: the tuning stage that timed it (0 split, 1 column strip, 2 row blocks,
                             3 vector blocks x dependent launch) */
} nlinv_tuning;

/* Autotuner of the transforms' tile shapes and the launch shapes (not part of the paper's method): reconstructs the
 * caller's representative frame (y, mask, start value x0; DEVICE pointers, as for nlinv_reconstruct) as graph
 * replays, reps timed replays per candidate after one untimed, every one from a cold L2 (a temporary buffer of twice
 * the L2 size is written before it, outside the timing).  It searches one dimension per stage, each from the best
 * shapes so far: (0) the four-step split n = N1 * N2 of every transform (the compiled split and, for n = 128 ... 384,
 * an alternative, e.g. 384 = 12 * 32 beside 16 * 24), (1) the column-strip width of the column passes (4, 8, 16),
 * (2) the row-pass blocks per SM (1, 2, 3), (3) the vector-pass blocks per SM (2, 4, 8) x dependent launch off/on.
 * Within a stage a candidate replaces the incumbent only when it is 3 % faster (closer shapes swap places with
 * small changes of conditions); candidates whose passes do not fit in shared memory are skipped.  The tensor-core
 * passes (tensor_dft = 1) keep the compiled split and column strips.  Whole frames of real data are timed: the passes
 * overlap their neighbours inside a graph, so a pass timed alone can rank shapes wrongly, and an all-zero
 * workspace times differently from data.  The workspace is overwritten.  The choice is cached per (device, n,
 * ncoils, fov, newton_steps, cg_iters, tensor_dft) for the process, so a second context of the same shape takes it
 * without timing.  out (HOST) receives the choice and table (HOST, table_len >= 16 entries) every timed candidate in
 * order (unused entries zeroed); either may be NULL.  Errors: EINVAL (NULL or host pointers, reps outside 1..1000,
 * a short table, a batch frame), ENOMEM, ECUDA. */
NLINV_API nlinv_status nlinv_autotune(nlinv_ctx* ctx, const nlinv_c32* y, const uint8_t* mask, const nlinv_c32* x0,
                                      int reps, nlinv_tuning* out, nlinv_tuning* table, int table_len);

/* Applies the shapes of t (split_n1, col_strip, row_blocks_per_sm, vec_blocks_per_sm, pdl; ms_per_frame and stage
 * are ignored) to the context, e.g. a choice of nlinv_autotune stored earlier.  Synchronous.  Errors: EINVAL (NULL
 * t, a split / strip combination not compiled for n, shapes outside the ranges of nlinv_tuning, passes that do not
 * fit in shared memory, a batch frame, other splits with tensor_dft = 1), ECUDA. */
NLINV_API nlinv_status nlinv_set_shapes(nlinv_ctx* ctx, const nlinv_tuning* t);

/* Kernel launches queued by the last nlinv_reconstruct, nlinv_forward, ... call (the graph's kernel nodes when a
 * graph was replayed).  -1 for a NULL context. */
NLINV_API long nlinv_last_launch_count(const nlinv_ctx* ctx);

/* Where the CG solves of the last reconstruction on ctx stopped (the CG steps of Eq. 3, Sec. 3.1).  CG runs
 * params.cg_iters iterations; it stops earlier only at the rounding floor of its single-precision arithmetic --
 * |r| <= 2^-24 |b| (the FP32 unit roundoff relative to the right-hand side b, which includes b = 0),
 * Re<p, A p> <= 0 (impossible in exact arithmetic for the positive definite system of Eq. 3) or a non-finite
 * value -- and the rest of that solve then leaves dx unchanged (its remaining CG launches return at once).  out (HOST, len >= newton_steps ints) receives per Newton step the index of
 * the CG iteration that stopped, or -1 when all iterations ran.  Waits for the context's stream.  Errors: EINVAL
 * (NULL or short out, no reconstruction yet), ECUDA. */
NLINV_API nlinv_status nlinv_cg_stops(nlinv_ctx* ctx, int* out, int len);

/* F x like nlinv_forward, but without a context and without allocating any device memory.  The paper has no
 * counterpart; it serves callers that may not allocate device memory when they apply F: a real-time loop that
 * reserves its GPU memory up front and must not see a cudaMalloc fail or stall mid-series, or a host framework
 * that owns every device allocation.  Such callers cannot use nlinv_create, whose workspace is allocated.
 * The scratch (the twiddle and Sobolev tables at fixed offsets, then the Omega-column transform buffer and the
 * coil maps) lives in one file-scope device array of 16 MiB that every GPU loading this library holds until the
 * process exits; a call whose n, ncoils and fov need more than that is rejected with EINVAL (384 x 384 with 10
 * coils and fov = n/4 fits; 512 x 512 with 16 coils does not).  The caller passes x (1+J planes), mask and y_out
 * (J planes), device (or managed) memory of the current device, and a cudaStream_t (NULL = legacy default stream);
 * params supplies n, ncoils, fov, sobolev_a and sobolev_l (the other fields are ignored).
 * Set-up: the first call on a device (with that device current) finds the array's device address, and the first
 * call, and every call whose n or Sobolev parameters differ from the previous call's on that device, writes the
 * tables and waits for the stream -- so make such a call before any stream capture.  The device address and the
 * record of the tables are kept for the process: do not call this after cudaDeviceReset.
 * All calls on a device share the one array and every call overwrites its buffers (nothing in it has to start at
 * zero): calls that overlap on the GPU -- on different streams or host threads -- race and give wrong results.
 * Errors: EINVAL (bad params, NULL pointers, memory of another device or of the host, sizes beyond the scratch),
 * ECUDA; message via nlinv_last_error(NULL). */
NLINV_API nlinv_status nlinv_forward_noalloc(const nlinv_params* params, void* stream, const nlinv_c32* x,
                                             const uint8_t* mask, nlinv_c32* y_out);

/* Message of the last failed call on ctx (or of the last failed nlinv_create when ctx is NULL).  The string is
 * owned by the library and stays valid until the next call on the same context. */
NLINV_API const char* nlinv_last_error(const nlinv_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* NLINV_H */
