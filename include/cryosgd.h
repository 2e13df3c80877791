/*
 * cryosgd.h -- C ABI of libcryosgd: the GPU hot path of known-pose,
 * diagonally preconditioned SGD for cryo-EM volume refinement
 * (Toader, Brubaker & Lederman, "Efficient high-resolution refinement in
 * cryo-EM with stochastic gradient descent", arXiv 2311.16100).
 *
 * Conventions (all entry points)
 * ------------------------------
 * Grid.  M is the grid side, even, 4 <= M <= CS_MAX_M.  Voxel (iz, iy, ix)
 *   has linear index (iz*M + iy)*M + ix and Fourier coordinates
 *   (kx, ky, kz) = (ix - M/2, iy - M/2, iz - M/2); DC sits at index M/2.
 *   Image pixel (iy, ix) has (kx, ky) as above and index iy*M + ix.  (Section
 *   2.1 only requires the images to be the z = 0 plane of the volume grid.)
 * Complex data.  A complex64 array is interleaved (re, im) float pairs:
 *   a volume is float[M^3 * 2], a stack of B images float[B * M * M * 2].
 * Poses.  rot is float[B][9], the row-major rotation matrix R_i of each image.
 *   Pixel r = (kx, ky, 0) reads the volume at R_i^T r (Section 2.1:
 *   (R v)(r) = v(R^T r)).  No in-plane shift (T_i = I).
 * Disc.  Only pixels with kx^2 + ky^2 <= r_max^2 belong to the model
 *   (1 <= r_max <= M/2 - 1).  slice_project writes 0 elsewhere; the adjoint,
 *   loss and gradient ignore the other pixels.
 * Interpolation.  CS_NEAREST (Eq. def nn interp): voxel at rint() of each
 *   coordinate c_a = R[0][a]*kx + R[1][a]*ky, evaluated as two single
 *   precision products and one sum without fused multiply-add, rounded half
 *   to even.  CS_TRILINEAR (Eq. def tri interp): the eight corners of the
 *   cell holding R^T r with trilinear weights.  Corners outside the grid
 *   contribute nothing.
 * CTF.  When enabled, C_i(q) = -(sqrt(1-A^2) sin chi + A cos chi) with
 *   chi = pi lam df_i s^2 - (pi/2) Cs lam^3 s^4, s^2 = q / (M pixel)^2,
 *   q = kx^2 + ky^2, lam the relativistic electron wavelength at kv.
 *   (The paper only requires C_i real, diagonal, radially symmetric.)
 * Memory.  Every array argument is a device pointer unless stated
 *   otherwise; the caller owns it.  The library owns only the opaque handle
 *   and the workspace inside it.
 * Streams.  stream is a cudaStream_t (NULL = legacy default stream).  All
 *   work is enqueued asynchronously on it; no call synchronises unless
 *   stated.
 * Errors.  Every call returns a cs_status.  Arguments are validated on the
 *   host before anything is enqueued; on error nothing is enqueued and
 *   cs_last_error() describes the cause.  The library never aborts, traps or
 *   exits.  CS_ERR_CUDA reports a failed CUDA runtime call (launch or
 *   allocation) with its message.
 */
#ifndef CRYOSGD_H
#define CRYOSGD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CS_MAX_M 512

typedef enum {
  CS_OK = 0,
  CS_ERR_ARG = 1,      /* null pointer, bad enum, non-finite scalar */
  CS_ERR_SHAPE = 2,    /* M, r_max, B or a count out of range */
  CS_ERR_CUDA = 3,     /* a CUDA runtime call failed */
  CS_ERR_TIMEOUT = 4,  /* a bounded device-side wait ran out */
  CS_ERR_INTERNAL = 5, /* an internal consistency check failed */
  CS_ERR_ALLOC = 6     /* workspace allocation failed */
} cs_status;

typedef enum { CS_NEAREST = 0, CS_TRILINEAR = 1 } cs_interp;

typedef enum {
  CS_PLAIN = 0,       /* no preconditioner, D-hat = I */
  CS_HUTCHINSON = 1,  /* Algorithm 1: D estimated on the fly */
  CS_FIXED = 2        /* D given (precomputed or learned), thresholded */
} cs_sgd_mode;

/* Microscope parameters of the CTF (Sections 2.1, 3.3). */
typedef struct {
  float kv;       /* accelerating voltage, kV (> 0) */
  float cs_mm;    /* spherical aberration, mm (>= 0) */
  float amp;      /* amplitude contrast A, 0 <= A < 1 */
  float pixel_A;  /* pixel size, Angstrom (> 0) */
  int enabled;    /* 0: C_i = I and defocus may be NULL */
} cs_ctf;

/* Geometry shared by every operator call. */
typedef struct {
  int M;        /* grid side (even, 4..CS_MAX_M) */
  int r_max;    /* disc / ball radius in pixels (1..M/2-1) */
  int interp;   /* cs_interp */
  cs_ctf ctf;
} cs_geom;

typedef struct cs_handle cs_handle;

/* Create a handle bound to CUDA device `device` (made current for the
 * call).  *h receives the handle (NULL on failure).  The handle holds a
 * lazily grown workspace; it is not thread safe: use one per host thread. */
int cs_create(cs_handle** h, int device);
/* Free the handle and its workspace (synchronises the device first).
 * NULL is accepted. */
int cs_destroy(cs_handle* h);
/* Message of the last failed call on h ("" if none).  Owned by h. */
const char* cs_last_error(const cs_handle* h);
/* Static name of a status code. */
const char* cs_status_string(int status);
/* Grow the workspace for grids of side <= M and batches of <= max_batch
 * images, so that later calls with those sizes allocate nothing (and can be
 * captured in a CUDA graph).  Synchronous. */
int cs_reserve(cs_handle* h, int M, int max_batch);
/* Bytes of device workspace currently held by h. */
size_t cs_workspace_bytes(const cs_handle* h);

/* Scatter algorithm of the adjoint-type passes (backproject_adjoint,
 * loss_grad, hvp, hutchinson_diag and the SGD step):
 *   CS_ALGO_VECTOR -- one thread per disc pixel; the trilinear adjoint is
 *                     packed into 16-byte vector reductions into
 *                     parity-split accumulators, then folded back (default
 *                     for trilinear interpolation; CS_ALGO_AUTO selects it);
 *                     in the SGD step the Hutchinson estimate shares the
 *                     gradient's traversal;
 *   CS_ALGO_PIXEL  -- one thread per pixel, one FP32 reduction per corner
 *                     into global memory (AUTO's choice for nearest);
 *   CS_ALGO_TILED  -- volume tiles binned by image, adjoint accumulated in
 *                     shared memory and added to global memory once per tile
 *                     and work item (requires orthonormal rotations: the
 *                     binning assumes |R^T r| = |r|).
 * All compute the same sums (in different orders). */
enum { CS_ALGO_AUTO = 0, CS_ALGO_PIXEL = 1, CS_ALGO_TILED = 2, CS_ALGO_VECTOR = 3 };
int cs_set_algo(cs_handle* h, int algo);

/* Pose -> rotation.  quat float[B][4] unit quaternions (w, x, y, z),
 * Hamilton convention (R v = q (0, v) q*; normalised first); rot float[B][9]
 * row-major R.  The paper's pose carries R directly (Definition 2.1); this
 * converts the usual quaternion parameterisation. */
int cs_quat_to_rot(cs_handle* h, const float* quat, int B, float* rot,
                   void* stream);

/* Forward operator (Eq. fwd model without noise): out_i = C_i P_i v for
 * i < B.  vol complex64[M^3]; out complex64[B][M][M] (overwritten, 0 outside
 * the disc); defocus float[B] in Angstrom (may be NULL if CTF disabled). */
int cs_slice_project(cs_handle* h, const cs_geom* g, const float* vol,
                     const float* rot, const float* defocus, int B, float* out,
                     void* stream);

/* Adjoint (Definition 2.1, P^* = conjugate transpose):
 * vol_accum += scale * sum_i P_i^* C_i y_i.  images complex64[B][M][M];
 * vol_accum complex64[M^3] is ACCUMULATED into (the caller zeroes it), so a
 * batch split across calls (or devices) sums to the unsplit result. */
int cs_backproject_adjoint(cs_handle* h, const cs_geom* g, const float* images,
                           const float* rot, const float* defocus, int B,
                           float scale, float* vol_accum, void* stream);

/* Mini-batch loss and gradient (Eq. optim cp with batch scale, Section 3):
 *   f = scale/2 sum_i |x_i - C_i P_i v|^2 + lambda/2 |v|^2,
 *   grad = scale sum_i P_i^* C_i (C_i P_i v - x_i) + lambda v.
 * vol, images as above; grad complex64[M^3] is OVERWRITTEN; loss is a
 * device double (may be NULL) OVERWRITTEN with f.  scale = N/|I| for a batch
 * I of a dataset of N images.  The loss sum is deterministic. */
int cs_loss_grad(cs_handle* h, const cs_geom* g, const float* vol,
                 const float* images, const float* rot, const float* defocus,
                 int B, float lambda, float scale, float* grad, double* loss,
                 void* stream);

/* Hessian-vector product (Eq. hessian with CTF):
 *   Hz = scale sum_i P_i^* C_i^2 P_i z + lambda z,  z, Hz real float[M^3]
 * (Hz overwritten; z and Hz must not alias). */
int cs_hvp(cs_handle* h, const cs_geom* g, const float* z, const float* rot,
           const float* defocus, int B, float lambda, float scale, float* Hz,
           void* stream);

/* Hutchinson's diagonal estimate (Eq. hutch) with K = n_probes (1..32)
 * Rademacher probes on the mini-batch Hessian:
 *   diag_out = (1/K) sum_k z_k (.) H z_k   (float[M^3], overwritten).
 * Probe k of voxel j is -1 if bit k of W_j is set, +1 otherwise, where the
 * words of voxels 2i and 2i+1 are the low and high 32 bits of output number
 * probe_block*M^3/2 + i of a SplitMix64 stream seeded with `seed`.  Computed exactly (up to rounding) without
 * forming the K products separately. */
int cs_hutchinson_diag(cs_handle* h, const cs_geom* g, const float* rot,
                       const float* defocus, int B, float lambda, float scale,
                       int n_probes, uint64_t seed, uint64_t probe_block,
                       float* diag_out, void* stream);

/* Precomputed preconditioner (Section 4, the comparison arm that estimates
 * the diagonal in advance with Eq. diag est rule before SGD starts):
 *   for epoch e = 1..n_epochs, for batch b = 1..ceil(N/B) (images b*B ..
 *   b*B + |I_b| - 1 in the given order, the last batch possibly short):
 *     k = k + 1,  est = cs_hutchinson_diag(batch, lambda, scale = N/|I_b|,
 *                                          n_probes, seed, probe_block = k),
 *     D_out = ((k-1)/k) D_out + (1/k) est.
 * rot_all float[N][9] and defocus_all float[N] (NULL without CTF) cover the
 * whole dataset; D_out float[M^3] is overwritten (its previous contents are
 * never read).  Probe blocks 1..n_epochs*ceil(N/B) are used, so the result
 * averages n_epochs * ceil(N/B) * n_probes probes; its expectation is the
 * diagonal of the full-data Hessian (plus lambda) when B divides N.  Errors:
 * CS_ERR_SHAPE for N, B or n_epochs < 1, n_probes outside [1, 32], or more
 * than 2^31 - 1 iterations; CS_ERR_ARG for NULL pointers or non-finite
 * lambda. */
int cs_precompute_preconditioner(cs_handle* h, const cs_geom* g, const float* rot_all,
                                 const float* defocus_all, int N, int B, int n_epochs,
                                 float lambda, int n_probes, uint64_t seed, float* D_out,
                                 void* stream);

/* Hutchinson's diagonal estimate without device allocation.  The paper has
 * no counterpart: this is a deployment variant of cs_hutchinson_diag for
 * callers that cannot allocate device memory when they need the estimate
 * (inside another application's stream capture, under a caching allocator
 * that must not be bypassed, or after a start-up-only allocation phase).
 * Same arguments and result as cs_hutchinson_diag (per-pixel algorithm), on
 * the current CUDA device, without a handle.  Its only scratch, one probe
 * word per voxel, is a fixed 8 MiB device array inside the library that
 * every GPU loading the library holds until exit, so M is limited to 128:
 * larger grids return CS_ERR_SHAPE and enqueue nothing.  Other argument
 * errors return CS_ERR_ARG / CS_ERR_SHAPE as in cs_hutchinson_diag (no
 * message is recorded: there is no handle).  No cudaMalloc or cudaFree is
 * made.  The first call on a device looks up the array's device address
 * (make it before any stream capture); that address is kept for the life of
 * the process, so do not call this entry point on a device after a
 * cudaDeviceReset of it.  Each device holds its own copy of the array; all
 * calls on one device share that copy and find the last call's probe words
 * in it (every call rewrites the words it reads), so calls that overlap on
 * the same GPU (different streams) race on it: serialise them on one stream
 * per device. */
int cs_hutchinson_diag_noalloc(const cs_geom* g, const float* rot,
                               const float* defocus, int B, float lambda,
                               float scale, int n_probes, uint64_t seed,
                               uint64_t probe_block, float* diag_out,
                               void* stream);

/* Exact diagonal of the mini-batch Hessian (Eq. hessian; under nearest
 * interpolation without CTF it is |Omega_j| + lambda, Eq. H diag):
 *   diag_out_j = lambda + scale sum_i sum_p C_ip^2 w_pj^2,
 * and the per-voxel features coverage_j = scale sum_i sum_p w_pj (the pose
 * coverage count |Omega_j| of Section 3.1 under nearest interpolation) and
 * ctf2w_j = scale sum_i sum_p C_ip^2 w_pj; with scale = N/B the batch's
 * sums estimate the dataset's.  All float[M^3], overwritten; each of the
 * three outputs may be NULL. */
int cs_exact_diag(cs_handle* h, const cs_geom* g, const float* rot,
                  const float* defocus, int B, float lambda, float scale,
                  float* diag_out, float* coverage_out, float* ctf2w_out,
                  void* stream);

/* Threshold alpha of Eq. (thresh value) at R = r_max:
 *   alpha = P_x(R)/P_v(R) * scale_alpha * sum_{i<N} C_i(R)^2 + lambda,
 * with 1-voxel Fourier shells (round(|k|) = R) counted on the grid and
 * C_i(R) the CTF of image i at |k| = R (1 without CTF).  defocus_all
 * float[N] (may be NULL without CTF); alpha_out one device double. */
int cs_threshold_alpha(cs_handle* h, const cs_geom* g, const float* defocus_all,
                       int N, double lambda, double scale_alpha,
                       double* alpha_out, void* stream);

/* Scalars of the SGD state, one device double each (index into
 * cs_sgd_state.scalars). */
enum {
  CS_S_ETA = 0,      /* in/out: step size eta (eta^(k-1) in, eta^(k) out) */
  CS_S_K = 1,        /* in/out: iterations done; the step runs k+1 */
  CS_S_ALPHA = 2,    /* in: threshold alpha of Eq. (thresh) */
  CS_S_LOSS = 3,     /* out: f_I(v^(k)) before the step */
  CS_S_G = 4,        /* out: |grad|^2 in the D-hat^{-1} norm */
  CS_S_Q = 5,        /* out: curvature of f_I along the step direction */
  CS_S_HALVINGS = 6, /* out: number of halvings of eta in this step */
  CS_S_STATUS = 7,   /* out: 0 ok, 1 no descent (G = 0 or Q <= 0) */
  CS_NSCALARS = 8
};

/* State of Algorithm 1 (Section 3.4).  Arrays are device float[M^3]
 * (v complex64[M^3]); all are owned by the caller and updated in place. */
typedef struct {
  float* v;          /* iterate v^(k) */
  float* D;          /* HUTCHINSON: D^(k-1) in (init I), D^(k) out; FIXED: D */
  float* D_avg;      /* HUTCHINSON: running Hutchinson mean (init 0) */
  double* scalars;   /* device double[CS_NSCALARS] */
  int mode;          /* cs_sgd_mode */
  int n_probes;      /* Rademacher probes per step (1..32, HUTCHINSON) */
  uint64_t seed;     /* probe seed; step k uses probe block k */
  float beta;        /* EMA weight of Eq. (exp avg update), 0 < beta < 1 */
  float c;           /* Armijo constant of Eq. (stochastic armijo), 0 < c < 1 */
  int max_halvings;  /* cap on halvings per step (>= 0) */
} cs_sgd_state;

/* One iteration of Algorithm 1 on the mini-batch (images, rot, defocus):
 *   HUTCHINSON: D_est = Hutchinson(batch, probe block k+1);
 *     D_avg = k/(k+1) D_avg + D_est/(k+1); D = beta D + (1-beta) D_avg;
 *   D-hat = max(|D|, alpha) (PLAIN: I);  g = grad f_I(v);  d = g / D-hat;
 *   eta = eta_prev 2^-m with the smallest m >= 0 such that the stochastic
 *   Armijo condition holds: since f_I is quadratic, f_I(v - eta d) =
 *   f_I(v) - eta G + eta^2 Q / 2 with G = <g, d>, Q = <d, H_I d>, so the
 *   condition is eta <= 2 (1 - c) G / Q, tested without re-evaluating f_I;
 *   v = v - eta d; k = k + 1.
 * Stream ordered, no host synchronisation; uses the handle's workspace
 * (call cs_reserve first to make the step capturable in a CUDA graph). */
int cs_precond_sgd_step(cs_handle* h, const cs_geom* g, cs_sgd_state* st,
                        const float* images, const float* rot,
                        const float* defocus, int B, float lambda, float scale,
                        void* stream);

/* cs_precond_sgd_step on a batch held in HOST memory: images_host
 * complex64[B][M][M], quat_host float[B][4] (unit quaternions, w first),
 * defocus_host float[B] (NULL without CTF).  Two ways to move the batch
 * (cs_set_host_mode; staged by default):
 *   staged: the batch is copied into one of two device staging slots owned
 *     by the handle, on the handle's own copy stream, after the step that
 *     last used that slot has finished; the step runs on `stream` once its
 *     copy is done, so issuing step n+1 while step n runs overlaps the copy
 *     of batch n+1 with the compute of step n;
 *   direct: when images_host is page-locked memory that the runtime maps
 *     into the device's address space (cudaPointerGetAttributes reports a
 *     host allocation with a device pointer), the traversal reads each disc
 *     pixel straight from it over the host link (every pixel once, outside
 *     the disc nothing), and only the poses and defoci are copied, on
 *     `stream`; otherwise the staged path is taken.
 * The step (quaternions -> rotations, then Algorithm 1) runs on `stream`;
 * if loss_host is not NULL the batch loss is copied to *loss_host (a host
 * double) after it.  Everything is asynchronous: the call returns at once.
 * Host buffers should be page-locked (pinned); they must stay valid and
 * unmodified, and *loss_host unread, until `stream` has completed the step.
 * Issue all steps of one handle on one stream.  Staging grows on demand
 * (device synchronisation, CS_ERR_ALLOC on failure).  Errors as
 * cs_precond_sgd_step, plus CS_ERR_ARG for NULL host pointers. */
int cs_precond_sgd_step_host(cs_handle* h, const cs_geom* g, cs_sgd_state* st,
                             const float* images_host, const float* quat_host,
                             const float* defocus_host, int B, float lambda, float scale,
                             double* loss_host, void* stream);

/* Pixels of an M x M image inside the disc of radius r_max (kx^2 + ky^2 <=
 * r_max^2): the only pixels the model of Eq. fwd model uses (Section 2.1's
 * images restricted to the band the volume is refined to).  A pure host
 * function; returns -1 for M or r_max out of range. */
int cs_disc_pixels(int M, int r_max);

/* cs_precond_sgd_step_host with the images given as their disc pixels only:
 * images_disc_host complex64[B][n_px], n_px = cs_disc_pixels(M, r_max),
 * each image's pixels with kx^2 + ky^2 <= r_max^2 in row-major order (ky
 * ascending, then kx ascending within a row).  Pixels outside the disc take
 * no part in the loss, gradient or Hessian, so the step is the same as with
 * the full images; the host-to-device copy carries n_px instead of M^2
 * pixels per image (76% of them for r_max = M/2 - 1).  The batch is
 * always staged: copied into the handle's staging slot on its copy stream,
 * then stepped on `stream`, double-buffered as in cs_precond_sgd_step_host
 * (the host mode does not apply); the vector traversal reads the packed
 * pixels where they land, the other scatter algorithms get them spread
 * into image layout by a small kernel on the copy stream first.  Arguments, synchronisation and errors otherwise as
 * cs_precond_sgd_step_host.  The paper has no counterpart: it is a data
 * layout for feeding the step from host memory. */
int cs_precond_sgd_step_host_disc(cs_handle* h, const cs_geom* g, cs_sgd_state* st,
                                  const float* images_disc_host, const float* quat_host,
                                  const float* defocus_host, int B, float lambda, float scale,
                                  double* loss_host, void* stream);

/* Phases of cs_precond_sgd_step timed by the profiler. */
enum {
  CS_PH_PRECOND = 0,   /* probe words, Hutchinson estimate, D update (vector
                          algorithm: probe words and accumulator reset only) */
  CS_PH_LOSS_GRAD = 1, /* forward, residual, loss and adjoint scatter (vector
                          algorithm: the one traversal that also accumulates
                          Hutchinson's estimate) */
  CS_PH_DIRECTION = 2, /* d = g / D-hat and its norms (vector algorithm: also
                          the accumulator folds and the D update) */
  CS_PH_CURVATURE = 3, /* |C P d|^2 for the Armijo step */
  CS_PH_UPDATE = 4,    /* eta and v -= eta d */
  CS_NPHASES = 5
};

/* Per-phase device timing of cs_precond_sgd_step with CUDA events recorded
 * on the call's stream.  cs_profile_enable(h, 1) starts a fresh record (up to
 * max_steps steps; later steps are not timed), 0 stops recording.
 * cs_profile_read synchronises on the recorded events and writes, per phase,
 * the summed milliseconds and the number of timed steps (arrays of
 * CS_NPHASES, host memory). */
int cs_profile_enable(cs_handle* h, int enable, int max_steps);
int cs_profile_read(cs_handle* h, double* ms, int* counts);

/* Kernels launched by this library in this process so far (all handles). */
uint64_t cs_kernel_launches(void);

/* Calibration: the rate, in G operations/s, at which this device executes
 * 16-byte floating-point reductions into global memory (random addresses in
 * a 16 MiB L2-resident buffer) -- the ceiling of the adjoint passes.
 * Synchronous; allocates and frees a 16 MiB buffer. */
int cs_measure_reduction_rate(cs_handle* h, double* gops);

/* ------------------------------------------------------------------------
 * Several volumes in one launch, CUDA graphs and launch-shape autotuning.
 * None of this is in the paper: it batches independent refinements (for
 * example volumes of different box sizes) so that the dominant traversal of
 * all of them is one kernel launch, and makes a whole step replayable as a
 * CUDA graph.
 * ------------------------------------------------------------------------ */
#define CS_MAX_PROBLEMS 8

/* One refinement problem of a multi-volume step.  Its images, quaternions
 * and defocus values for all n_batches batches of B images stay in device
 * memory; step k (state.scalars[CS_S_K] = iterations done) uses batch
 * (k mod n_batches), chosen on the device, so a captured step replays over
 * the batches without host involvement. */
typedef struct {
  cs_geom geom;          /* trilinear interpolation only */
  cs_sgd_state state;    /* as for cs_precond_sgd_step */
  const float* images;   /* complex64 [n_batches*B][M][M] */
  const float* quat;     /* float [n_batches*B][4] unit quaternions (w,x,y,z) */
  const float* defocus;  /* float [n_batches*B] (NULL if the CTF is off) */
  int B;                 /* images per step (>= 1) */
  int n_batches;         /* >= 1 */
  float lambda;
  float scale;           /* N/|I| of this problem */
} cs_problem;

/* One Algorithm 1 iteration for each of n (1..CS_MAX_PROBLEMS) problems:
 * pose conversion of the selected batch, then the same computation as
 * cs_precond_sgd_step per problem, with the fused loss / gradient /
 * Hutchinson traversal of all problems in one kernel launch and the Armijo
 * curvature traversal in another.  All problems must use the same
 * cs_sgd_mode.  Stream ordered; grows the handle's multi-volume workspace on
 * first use (synchronous then). */
int cs_multi_step(cs_handle* h, const cs_problem* probs, int n, void* stream);

typedef struct cs_graph cs_graph;
/* Captures one cs_multi_step of these problems into an executable CUDA
 * graph (workspace and pixel tables prepared first, synchronously).  Each
 * cs_graph_launch replays one step: batches advance on the device.  The
 * graph keeps the problems' device pointers and the handle's workspace; it
 * is invalid once the handle is destroyed, and cs_graph_launch returns
 * CS_ERR_ARG if the handle's multi-volume workspace was reallocated, or its
 * pixel tables rebuilt (other problems, another launch shape), since the
 * capture.  Problems whose grids are split into z-slabs (cs_set_slabs) run
 * their traversals as their own launches inside the step.  A replay uses
 * that workspace: do not run other calls of the same handle concurrently
 * with it (other streams), use another handle. */
int cs_multi_step_graph(cs_handle* h, const cs_problem* probs, int n, cs_graph** graph);
int cs_graph_launch(cs_graph* graph, void* stream);
int cs_graph_destroy(cs_graph* graph);

/* Launch shape of the trilinear traversal kernels: threads per block
 * (128 or 256) and blocks per SM (1..32 for 256 threads, 1..64 for 128).
 * Default 256 x 8. */
int cs_set_launch_shape(cs_handle* h, int block_threads, int blocks_per_sm);
/* z-slabs of the trilinear vector traversals: each pass is split into
 * `slabs` launches, launch s processing the 16 x 16 pixel tiles (of every
 * image) whose centre's cell lies in the s-th slab of the grid along z,
 * grouped by region of the slab, so that the accumulators and the gathered
 * volume a launch touches stay in L2 on large grids.  0 (default): chosen
 * from the grid's footprint (1 slab up to 128^3; for the passes with
 * reductions 2 at 160^3, 3 at 192^3 and 6 at 256^3; for the curvature 1 up
 * to 192^3 and 2 at 256^3).  At most M/16 slabs are used.  Results are the
 * same sums in another order.  0 <= slabs <= 16. */
int cs_set_slabs(cs_handle* h, int slabs);
/* How cs_precond_sgd_step_host moves a batch: CS_HOST_STAGED (default:
 * double-buffered staging copies) or CS_HOST_DIRECT (the traversal reads
 * the images from the host buffer when it is device-mapped page-locked
 * memory, staged copies otherwise).  Measured on GB300 at 128^3, batch 1024:
 * staged 1.54 M images/s, direct 1.21 M (the link reads stall the
 * traversal); at 256^3 the two are equal.  CS_ERR_ARG for another value. */
enum { CS_HOST_STAGED = 0, CS_HOST_DIRECT = 1 };
int cs_set_host_mode(cs_handle* h, int mode);
/* Autotuner: times the fused traversal of these problems (without changing
 * their state) for a set of launch shapes, keeps the fastest on the handle
 * and returns it.  Synchronous. */
int cs_autotune(cs_handle* h, const cs_problem* probs, int n, int* block_threads,
                int* blocks_per_sm);

/* ------------------------------------------------------------------------
 * Learned diagonal preconditioner (not in the paper): a 3 -> 64 -> 64 -> 1
 * network with GELU (tanh form) activations predicts log D per voxel from
 * the features (|k| / (M/2), log1p(coverage_j), log1p(ctf2w_j)) where
 * coverage and ctf2w are the outputs of cs_exact_diag; it is trained by mean
 * squared error against log of Hutchinson estimates (Eq. hutch).  The
 * 64 x 64 layer runs on BF16 tensor cores (tcgen05) with FP32 accumulation:
 * its operands (first hidden activations, weights, and in the backward pass
 * the second hidden layer's gradient) are rounded to BF16.
 * Parameters: float[CS_MLP_NPARAMS], FP32 master copy, layout
 *   W1[64][3] | b1[64] | W2[64][64] (out, in) | b2[64] | w3[64] | b3.
 * ------------------------------------------------------------------------ */
#define CS_MLP_NPARAMS 4481

/* out_j = network(features_j) + offset for all M^3 voxels (exp_out:
 * exp(network(features_j)) + offset, the preconditioner D = exp(log D) +
 * lambda when offset = lambda).  use_tensor_cores = 0 runs the FP32
 * reference kernel (same rounding points).  CS_ERR_ARG for a non-finite
 * offset. */
int cs_mlp_forward(cs_handle* h, int M, const float* params, const float* coverage,
                   const float* ctf2w, float* out, int exp_out, float offset,
                   int use_tensor_cores, void* stream);
/* grad += gradient of L = mean over voxels with |k| <= r_ball of
 * (network_j - target_j)^2; *sse += sum of squared residuals (device
 * double).  The caller zeroes grad and sse. */
int cs_mlp_grad(cs_handle* h, int M, int r_ball, const float* params, const float* coverage,
                const float* ctf2w, const float* target, float* grad, double* sse,
                int use_tensor_cores, void* stream);
/* One Adam step (Kingma & Ba 2015) on params with moments m, v (caller
 * zeroes them before step 1), on the gradient grad_scale * grad (e.g.
 * 1 / number of accumulated samples: the mean of per-sample gradients);
 * grad is read and zeroed.  step >= 1; CS_ERR_ARG for a non-finite or
 * non-positive grad_scale or hyper-parameters out of range. */
int cs_mlp_adam_step(cs_handle* h, float* params, float* m, float* v, float* grad,
                     float grad_scale, int step, float lr, float beta1, float beta2, float eps,
                     void* stream);
/* Training target of the network from n_est >= 1 Hutchinson estimates of
 * the diagonal (Eq. hutch), estimates float[n_est][M^3] (e.g. independent
 * probe blocks of cs_hutchinson_diag with lambda = 0):
 *   m_j = (1/n_est) sum_e estimates[e][j],
 *   target_j = log(max(m_j, floor_rel * mean of the positive m_j))
 * (floor_rel alone when no m_j is positive).  target float[M^3],
 * overwritten.  CS_ERR_ARG for NULL pointers or floor_rel not in (0, 1];
 * CS_ERR_SHAPE for M or n_est out of range. */
int cs_mlp_target(cs_handle* h, int M, int n_est, const float* estimates, float floor_rel,
                  float* target, void* stream);
/* Failure-handling self-test (no counterpart in the paper): launches one
 * block whose mbarrier wait can never complete; the wait gives up after
 * `spins` polls (1 .. 2^24) and records the expiry in the handle's device
 * status word exactly as the tensor-core kernels do, so the next
 * cs_check_device_status returns CS_ERR_TIMEOUT (and clears the word).
 * Nothing faults or traps and the context stays usable; it lets a caller
 * verify its error path.  Asynchronous on `stream`. */
int cs_selftest_wait_timeout(cs_handle* h, long long spins, void* stream);
/* Synchronises the handle's device and reports whether a bounded
 * device-side wait ran out since the last check (CS_ERR_TIMEOUT, and the
 * word is cleared) or not (CS_OK).  In the debug variant of the library
 * (cs_build_flags() & CS_BUILD_DEBUG_BOUNDS) every gather and scatter index
 * of the traversal kernels is range-checked on the device; an index out of
 * range skips its access and the next call returns CS_ERR_INTERNAL (the
 * flags are cleared).  No counterpart in the paper. */
int cs_check_device_status(cs_handle* h);

/* Build options of the loaded library: CS_BUILD_DEBUG_BOUNDS when it is the
 * debug variant with device-side index range checks. */
#define CS_BUILD_DEBUG_BOUNDS 1
int cs_build_flags(void);

/* In-plane shift operator T_i of Definition 2.1 (a diagonal phase):
 *   images[i][y][x] *= T_i(k)      (sign = +1)
 *   images[i][y][x] *= conj T_i(k) (sign = -1),
 *   T_i(k) = exp(-2 pi i (kx tx_i + ky ty_i) / M),  k = (x, y) - M/2,
 * i.e. a real-space shift of image i by +(tx_i, ty_i) pixels.  images
 * complex64[B][M][M] in place (all pixels); shifts float[B][2] (tx, ty),
 * finite, |t| < 8192.  T_i is unitary and commutes with the CTF, so
 * |x_i - C_i T_i S_i v| = |T_i^* x_i - C_i S_i v|: every operator of this
 * library works with the unshifted slice S_i, a dataset with known shifts is
 * corrected once with sign -1, and the shifted forward model is
 * cs_slice_project followed by sign +1.  Errors: CS_ERR_SHAPE (M, B),
 * CS_ERR_ARG (NULL pointers, sign not +-1). */
int cs_phase_shift(cs_handle* h, int M, float* images, const float* shifts, int B, int sign,
                   void* stream);

/* Fourier shell correlation (Eq. fsc, Section 4) of complex volumes u, v
 * (complex64[M][M][M], grid as above) over the shells
 *   S_r = { k : round(|k|) = r },  r = 0 .. n_shells-1  (1 <= n_shells <= 1024;
 * voxels beyond the last shell are ignored):
 *   sums[r] = (Re sum_{S_r} u conj(v), sum_{S_r} |u|^2, sum_{S_r} |v|^2)
 * (device double[n_shells][3], overwritten) and, if fsc is not NULL,
 *   fsc[r] = sums[r][0] / sqrt(sums[r][1] sums[r][2])  (0 for an empty or
 * all-zero shell; device double[n_shells]).  The real part is reported: it
 * is the whole value for Hermitian-symmetric volumes.  Sums are FP64 with
 * atomics, so the last bits may vary between runs. */
int cs_fsc(cs_handle* h, int M, const float* u, const float* v, int n_shells, double* sums,
           double* fsc, void* stream);

/* Per-shell statistics of a real field x (float[M][M][M], finite values),
 * shells as in cs_fsc: count_out[r] = |S_r| (int), min_out[r] / max_out[r] =
 * min / max of x over S_r (float; +inf / -inf for an empty shell).  With x
 * = diag(H) (cs_exact_diag) this gives the condition number of the
 * diagonal restricted to the ball of radius R, max_{r <= R} max_out[r] /
 * min_{r <= R} min_out[r] (Section 3.1, Proposition 3.1).  Exact (no
 * rounding). */
int cs_shell_minmax(cs_handle* h, int M, const float* x, int n_shells, float* min_out,
                    float* max_out, int* count_out, void* stream);

/* Relative error over the ball |k| <= r_max:
 *   |v - v_ref| / |v_ref| -> *out (device double). */
int cs_rel_err(cs_handle* h, const cs_geom* g, const float* v, const float* v_ref,
               double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CRYOSGD_H */
