/*
 * sdft_ipm.h -- C ABI of the GB300 (sm_103a) solver for sparse-DFT recovery
 * from a masked, noisy real signal (arXiv 2502.04217).
 *
 * The library solves the LASSO problem of Sec. 3, Eq. (realopt),
 *     beta* = argmin_beta 1/2 || b - M_perp beta ||^2 + lambda || beta ||_1,
 * where A = C^H B^H is the real orthogonal operator of Eq. (map) (orthonormal
 * inverse DFT composed with the real parametrisation beta = B v of a
 * conjugate-symmetric spectrum, Eq. (beta)), M_perp = A restricted to the
 * observed samples (Eq. (MMperp)), and b the observed samples.  It runs the
 * primal-dual interior-point method of Sec. 3.3 on the slack QP
 * Eq. (slackproblem); each Newton system is reduced to the condensed KKT
 * system Eq. (condensedkkt) and solved matrix-free by conjugate gradients with
 * the preconditioner P of Sec. 3.5 (closed-form inverse Eq. (invprecond1)).
 * Every product with M_perp^T M_perp is a pair of hand-written FFTs with the
 * mask in between (Sec. 3.1); no cuFFT, no CPU fallback.
 *
 * Conventions
 *  - Every function returns an ipm_status; nothing is thrown across the ABI.
 *    On error, ipm_last_error() describes the failure.
 *  - Arguments are checked on the host before any GPU work: a bad argument
 *    returns IPM_ERR_ARG and leaves the handle unchanged.
 *  - The library never frees caller memory; caller buffers are copied where
 *    stated, and never retained after the call returns.
 *  - Grids are row-major with the LAST axis contiguous; every extent must be
 *    of the form 2^a 3^b 5^c 7^d (the FFT's radices: 2, 4, 8, 16, 3, 5, 7),
 *    at least 2 and at most 1024.  Extents may be even or odd: Sec. 3 defines
 *    the conjugate-symmetric subspace F for both (for odd n only v_0 is real)
 *    and treats the even case in detail; the odd case uses the same map with
 *    no Nyquist entry.  Odd extents without a factor 3 must be at most 512
 *    (625 and 875 have no launchable FFT tile: IPM_ERR_ARG).  gapply_noalloc
 *    takes even extents 2^a 3^b up to 512.
 *  - "beta layout": vectors indexed like beta are held as 2H doubles, where
 *    H = N_0 ... N_{d-2} (floor(N_{d-1}/2) + 1) is the number of half-spectrum
 *    slots.  Slot s carries two doubles; coordinates that are not LASSO
 *    variables (imaginary parts of self-conjugate frequencies, conjugate twins
 *    on the edge planes k_{d-1} = 0 and, for even N_{d-1}, k_{d-1} = N_{d-1}/2)
 *    are "ghosts" and are always 0.  The order of slots is internal; use
 *    ipm_pack_beta / ipm_unpack_beta to move between the beta layout and the
 *    canonical half spectrum.
 *  - "canonical half spectrum": the orthonormal DFT v of Sec. 3 restricted to
 *    k_{d-1} in [0, floor(N_{d-1}/2)], row-major with the halved axis last, as
 *    interleaved (re, im) doubles: 2H doubles (the layout of numpy's rfftn).
 *  - Two-block vectors of the condensed system (p, q, r, z in kkt_apply and
 *    precond_apply) are [beta block | z block], 4H doubles.
 *  - Pointers documented as "device" must be device (or managed) memory of
 *    the handle's device; pointers documented as "host or device" may be
 *    either (copies use unified addressing, cudaMemcpyDefault).
 *  - All work is queued on the handle's CUDA stream.  Functions that return
 *    results to the host synchronise that stream before returning.
 */
#ifndef SDFT_IPM_H
#define SDFT_IPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdft_ipm sdft_ipm; /* opaque; owns every device buffer it allocates */

typedef enum {
  IPM_OK = 0,
  IPM_ERR_ARG = 1,          /* invalid argument; no GPU work was done            */
  IPM_ERR_CUDA = 2,         /* a CUDA call failed; see ipm_last_error()           */
  IPM_ERR_OOM = 3,          /* device allocation failed                          */
  IPM_MAXITER = 4,          /* the IPM stopped at max_ipm before reaching gap_tol */
  IPM_KRYLOV_MAXITER = 5,   /* a PCG solve stopped at max_cg (solve continued)    */
  IPM_NUMERICAL = 6,        /* non-finite value or loss of positive definiteness */
  IPM_TIMEOUT = 7           /* a bounded device-side wait expired: the kernel gave up,
                               released what it held and returned; the context stays
                               usable (see ws_test_conv_stall, ipm_test_stage_stall) */
} ipm_status;

typedef enum { IPM_FP64 = 0, IPM_MIXED = 1 } ipm_precision;

typedef struct {
  int precision;        /* ipm_precision; IPM_FP64 is the plain method                       */
  double gap_tol;       /* stop when (P - D) / max(1, |P|) <= gap_tol (default 1e-6)          */
  double cg_tol;        /* PCG tolerance on sqrt(r^T P^{-1} r) (default 1e-6: an inexact Newton
                           direction; measured, the same IPM iterations and certified gaps as
                           1e-10 from gap_tol 1e-6 down to 1e-10 with 40-45 % fewer PCG
                           iterations; at gap_tol 1e-12 it may cost one or two more IPM
                           iterations, where 1e-10 suits better)                             */
  int cg_relative;      /* 1: relative to the initial residual (default); 0: absolute,
                           as the paper's 1e-12 rule (Sec. 5)                                  */
  int max_ipm;          /* IPM iteration cap (default 200)                                     */
  int max_cg;           /* PCG iteration cap per IPM iteration (default 500)                   */
  double sigma;         /* centring parameter (default 0.1)                                    */
  double sigma_slow;    /* centring after a short step alpha < 0.1 (default 0.5)               */
  double tau;           /* fraction to the boundary (default 0.995)                            */
  int lambda_relative;  /* 1: lambda is a fraction of lambda_max = ||M_perp^T b||_inf          */
  int cg_chunk;         /* host-driven mode: PCG iterations queued between host checks (4)     */
  int use_graph;        /* 1 (default): the whole solve is one CUDA graph whose IPM and PCG
                           loops are conditional WHILE nodes decided on the device; 0: the
                           host drives the loops (also used while profiling is on)             */
  int autotune;         /* 1 (default): at ipm_create, time every launchable tile shape
                           (pencils per block, per-thread radix budget) of each FFT pass on
                           the device and keep the fastest (cached per shape for the
                           process); 0: a fixed heuristic                                     */
  int tile_e;           /* 0 (default): chosen as above; else force this per-thread element
                           budget (4, 8 or 16, or 6 or 12 for lengths with a factor 3)
                           wherever launchable                                                */
  int tile_p;           /* 0 (default): chosen as above; else force this many pencils per
                           tile (a power of two) wherever launchable                          */
  int refine_every;     /* IPM_MIXED only.  0 (default): PCG runs on FP32 products and the
                           IPM recomputes its residuals in FP64 every iteration.  k > 0: in
                           addition, every k PCG iterations and whenever PCG converges, the
                           PCG residual is replaced by rhs - K x computed with FP64 products
                           and PCG restarts from x; it stops only when that FP64 residual
                           passes the test (bounded by max_cg)                                */
  int tile_engine;      /* FFT pass engine.  0 (default): with autotune, the faster of the two
                           per pass shape, else the shared-memory one; 1: the shared-memory
                           Stockham engine (every stage through shared memory); 2: the
                           register engine (16 values per thread, first and last stage in
                           registers straight from / to global memory) wherever the length
                           allows it (32, 64, 128, 256 or 512; the middle pass uses Nl/2),
                           else the shared-memory one.  tile_e is ignored by engine 2.       */
  int sigma_rule;       /* centring parameter of each direction.  2 (default): the single-step
                           predictor-corrector (Mehrotra's method adapted to one Krylov solve
                           per iteration, as Sec. 5 proposes): the affine predictor is
                           P^{-1} rhs_aff (no product with G), sigma = (mu_aff / mu)^3
                           clamped to [sigma_min, 1], and the corrector's complementarity
                           rows target sigma mu - ds_aff o dnu_aff; after a PCG solve
                           stopped at max_cg the next direction takes the fixed rule.
                           1: adaptive, sigma = clamp((1 - alpha)^3, sigma_min, sigma_slow)
                           from the last step alpha (the previous step standing in for an
                           affine predictor; the first direction uses sigma; the fixed rule
                           after a capped PCG solve); 0: sigma, or sigma_slow after a step
                           alpha < 0.1                                                      */
  double sigma_min;     /* lower clamp of sigma for rules 1 and 2 (default 0.01; rule 1 wants
                           0.03: at 0.01 its PCG broke down on tiny problems below a 1e-12
                           gap; rule 2 at 0 stalled on a 64^3 problem at a 1e-10 gap)        */
  int exact_residual;   /* 0 (default): G beta is carried along with beta (the last pass of
                           each PCG product also stores (G p)_beta -- from FP32 products in
                           IPM_MIXED --, PCG accumulates G x = sum alpha G p in FP64 beside x,
                           the step adds alpha G x), and an FP64 product recomputes it exactly
                           only to confirm a stop test that passed on the carried value, so
                           the reported gap is always an exact one; a confirmation that fails
                           switches the rest of the solve to 1.  The cold start needs no first
                           product (G 0 = 0); from a given point an FP64 product forms the
                           first G beta.  1: an FP64 product recomputes G beta every IPM
                           iteration.  Carrying applies with krylov = 0 and
                           refine_every = 0; otherwise G beta is recomputed every iteration */
  double precond_rho;   /* identity scale rho of the preconditioner
                           P = [rho I + Lambda1, Lambda2; Lambda2, Lambda1] (Sec. 3.5).
                           1 (default): the paper's P; 0: rho = n / m with m the number of
                           observed samples (the scaled identity of Fountoulakis et al. that
                           the paper compares with); any other rho > 0 is used as given      */
  int pdl;              /* 1 (default): the kernels of a solve (and of gapply / kkt_apply) are
                           launched with programmatic dependent launch: each may start while
                           its predecessor drains and waits on the device until that
                           predecessor has completed (same results, shorter gaps between the
                           many small kernels of a solve); 0: plain stream order            */
  int krylov;           /* Krylov method for the Newton systems (Sec. 3.5 names CG, CR and CAr
                           for these SPD systems).  0 (default): preconditioned conjugate
                           gradients; 1: preconditioned conjugate residuals (one product K z
                           per iteration, two update kernels); 2: conjugate A-residuals (CAr:
                           the iterate minimising (K P^{-1} r)^T P^{-1} (K P^{-1} r) over the
                           Krylov space; one product K y per iteration with y = P^{-1} K z
                           kept by recurrence, one more product at each PCG start and at each
                           restart, which happens when y^T K y has fallen by the unit round-off
                           of the products' precision since the last start; restart products
                           count in kkt_products).  With 1 or 2, G beta is recomputed every
                           iteration and refine_every must be 0.  Changing the method with
                           ipm_set_options allocates its vectors (4 x 4H doubles at most). */
  int tile_kstage;      /* (fixed at ipm_create, like the tile shape) how the last FFT pass of
                           a product with K (2D and 3D grids) brings
                           the FP64 operands of its epilogue (p on both blocks, Lambda1,
                           Lambda2: 64 bytes per slot).  0 (default): with autotune, the
                           fastest of the three forms below for the tuned tile, else 1;
                           1: per-slot loads after the tile's transform; 2: one L2 bulk
                           prefetch (cp.async.bulk.prefetch) of the tile's operands when the
                           block starts; 3: bulk copies (cp.async.bulk) of them into shared
                           memory when the block starts, completing on an mbarrier that the
                           epilogue waits on (bounded: IPM_TIMEOUT).  2 and 3 apply to the
                           shared-memory engine and where the stage fits a block's shared
                           memory, else 1 is used                                             */
} ipm_options;

typedef struct {
  int status;           /* ipm_status of the solve                                   */
  int ipm_iters;        /* Newton directions computed                                */
  int cg_iters_total;   /* PCG iterations (= products with K) over the solve         */
  int cg_iters_max;     /* largest PCG count of one IPM iteration                    */
  double primal;        /* P = 1/2 ||b - M_perp beta||^2 + lambda ||beta||_1         */
  double dual;          /* D of the scaled dual point (never above the optimum)      */
  double rel_gap;       /* (P - D) / max(1, |P|)                                     */
  double mu;            /* final duality measure                                     */
  double lambda;        /* the lambda actually used                                  */
  double lambda_max;    /* ||M_perp^T b||_inf                                        */
  double seconds;       /* wall time of ipm_solve                                    */
  int kkt_products;     /* products with M_perp^T M_perp (PCG; the products that formed
                           G beta; FP64 residual replacements)                         */
  int refinements;      /* FP64 residual replacements inside PCG (refine_every > 0)  */
  int exact_products;   /* the FP64 products that formed G beta exactly (none for the
                           cold start, whose G beta = G 0 = 0)                         */
} ipm_result;

/* Fill *opt with the defaults listed above. */
void ipm_default_options(ipm_options* opt);

/* Create a solver for one problem on the current CUDA device.
 *  ndim      1, 2 or 3.
 *  dims      ndim extents (row-major, last contiguous), see Conventions.
 *  mask      n = prod(dims) bytes, 1 = observed, 0 = missing (the paper's set
 *            M, Sec. 3); host or device; copied.  At least one sample observed.
 *  y         n doubles, the noisy signal; values at missing samples are
 *            ignored (b_hat of Sec. 3.1 is formed on the device); host or device; copied.
 *  lambda    > 0: the penalty, or its fraction of lambda_max when
 *            opt->lambda_relative is set.
 *  opt       NULL for defaults.
 *  stream    cudaStream_t to queue work on (NULL = legacy default stream).
 * Computes M_perp^T b once (Eq. (xi)) and lambda_max. */
ipm_status ipm_create(sdft_ipm** out, int ndim, const int64_t* dims, const uint8_t* mask, const double* y,
                      double lambda, const ipm_options* opt, void* stream);

/* Replace mask, y and lambda of an existing handle (same grid); host or
 * device pointers, copied.  Recomputes M_perp^T b and lambda_max. */
ipm_status ipm_set_problem(sdft_ipm* h, const uint8_t* mask, const double* y, double lambda);

/* Replace the options (grid and data unchanged). */
ipm_status ipm_set_options(sdft_ipm* h, const ipm_options* opt);

/* Run the interior-point method from the cold start of Sec. 3.3 (or from the
 * point set by ipm_set_point since the last solve).  Fills *res (may be NULL).
 * Returns IPM_OK on convergence to gap_tol, IPM_MAXITER, or an error. */
ipm_status ipm_solve(sdft_ipm* h, ipm_result* res);

/* Sizes: *nslots = H (beta-layout vectors have 2H doubles), *n = prod(dims). */
ipm_status ipm_sizes(const sdft_ipm* h, int64_t* nslots, int64_t* n);

/* q = M_perp^T M_perp p for a beta-layout vector (Sec. 3.1); device pointers,
 * 2H doubles each, 16-byte aligned; p's ghost coordinates must be 0, q's are
 * written as 0. */
ipm_status gapply(sdft_ipm* h, const double* p, double* q);

/* q = K p with K = [G + Lambda1, Lambda2; Lambda2, Lambda1] (Eq. (condensedkkt)),
 * G = M_perp^T M_perp, Lambda1 = Sigma1 + Sigma2, Lambda2 = Sigma1 - Sigma2
 * for the Sigma set by ipm_set_sigma (or the last IPM iterate).  Device
 * pointers, 4H doubles each ([beta block | z block]), 16-byte aligned. */
ipm_status kkt_apply(sdft_ipm* h, const double* p, double* q);

/* Failure-detection test of the staged K epilogue (not for production use): the
 * NEXT kkt_apply on h leaves out, in every block of its last pass, the fourth of
 * the four operand copies that its mbarrier expects, and every wait on that
 * barrier gives up after 2^wait_log2 polls (8..24).  That call must return
 * IPM_TIMEOUT without hanging (q is then incomplete) and the handle stays usable.
 * IPM_ERR_ARG for an out-of-range wait_log2 or when the last pass of h's product
 * does not stage its operands in shared memory (tile_kstage = 3 forces that). */
ipm_status ipm_test_stage_stall(sdft_ipm* h, int wait_log2);

/* z = P^{-1} r by the closed form Eq. (invprecond1) with D = Sigma1 + Sigma2 +
 * 4 Sigma1 Sigma2 (Prop. exprbd).  Device pointers, 4H doubles each. */
ipm_status precond_apply(sdft_ipm* h, const double* r, double* z);

/* Set Sigma_i = S_i^{-1} V_i (Eq. (defsigma)) from slacks s_i > 0 and bound
 * multipliers nu_i > 0 in the beta layout (device pointers, 2H doubles each;
 * ghost entries ignored). */
ipm_status ipm_set_sigma(sdft_ipm* h, const double* s1, const double* nu1, const double* s2, const double* nu2);

/* Start the next ipm_solve from w = (beta, z, s1, s2, nu1, nu2), each 2H
 * doubles in the beta layout, host or device; s and nu must be > 0 on every
 * non-ghost coordinate.  Used for warm starts and to resume a solve. */
ipm_status ipm_set_point(sdft_ipm* h, const double* const w[6]);

/* Copy the current iterate (beta, z, s1, s2, nu1, nu2) to six buffers of 2H
 * doubles (host or device). */
ipm_status ipm_get_point(sdft_ipm* h, double* const w[6]);

/* The recovered spectrum v = B^H beta of the current iterate as the canonical
 * half spectrum (2H doubles, host or device). */
ipm_status ipm_get_spectrum(sdft_ipm* h, double* v_half);

/* beta layout <-> canonical half spectrum (Eq. (beta) / Eq. (v)); device
 * pointers, 2H doubles each.  pack ignores the entries of twins on the edge
 * planes; unpack fills them with the conjugate of their representative. */
ipm_status ipm_pack_beta(sdft_ipm* h, const double* v_half, double* beta);
ipm_status ipm_unpack_beta(sdft_ipm* h, const double* beta, double* v_half);

/* Per-kernel timing with CUDA events around every launch (0 = off, default;
 * each call resets the counters).  ipm_profile_get returns, for kernel class
 * k (0: FFT row pass, 1: column pass, 2: middle pass, 3: PCG update, 4: other
 * IPM kernels, 6: the Newton-system kernel that forms Sigma, P^{-1} and the
 * right-hand side, 7: the step-length and step kernels, 8: the duality-gap
 * certificate), the number of launches and their summed duration in
 * milliseconds since the last reset (timed only while profiling is on); for
 * k = 5 it returns the number of kernels the library launched since the last
 * reset, timed or not, and *ms = 0. */
ipm_status ipm_profile_enable(sdft_ipm* h, int on);
ipm_status ipm_profile_get(sdft_ipm* h, int k, int64_t* launches, double* ms);

/* q = M_perp^T M_perp p, like gapply, but without a handle and without
 * allocating any device memory (the paper has no counterpart: this entry point
 * serves callers that cannot call cudaMalloc -- hosts that hand out all device
 * memory through their own allocator or a fixed budget, code that must not take
 * the implicit device synchronisation of cudaMalloc/cudaFree, plugins running in
 * another program's CUDA context).
 *  ndim, dims  as for ipm_create; the half spectrum may have at most 262144
 *              slots (H = N_0..N_{d-2} (N_{d-1}/2 + 1)); 512 x 512 and
 *              64 x 64 x 64 fit, larger grids return IPM_ERR_ARG.
 *  mask        device pointer, n = prod(dims) bytes, 1 = observed.
 *  p, q        device pointers, 2H doubles each in the beta layout of the
 *              handle-based API (the layout depends only on dims); p's ghost
 *              coordinates must be 0, q's are written as 0.
 *  stream      cudaStream_t the work is queued on (NULL = legacy default
 *              stream).  The call queues one memset and kernels only (the
 *              twiddle tables are built on the device) and returns without
 *              waiting for the stream.
 * The caller still owns every input and output.  Scratch is one fixed
 * file-scope device array of about 4.7 MB that each GPU loading the library
 * keeps until the process exits.  The first call in each CUDA context (with
 * the device current) looks up the array's device address once and caches it
 * for that context; make that first call before any stream capture.  After
 * cudaDeviceReset destroys a context that has made a call, do not call again
 * in the process.  All calls share the array and each rewrites what it needs,
 * so calls that overlap on the GPU (other streams, other host threads on the
 * same device) race: order them on one stream.  FP64 arithmetic. */
ipm_status gapply_noalloc(int ndim, const int64_t* dims, const uint8_t* mask, const double* p, double* q,
                          void* stream);

/* ---- batches of independent problems ------------------------------------
 * A batch holds `count` problems of possibly different grids and solves them
 * together: ipm_solve_batch is ONE CUDA graph launch whose branches are the
 * problems' whole solves (each with its IPM and PCG loops as conditional WHILE
 * nodes), so the problems' kernels run concurrently and the host waits once.
 * Each problem keeps its own device buffers; FFT tile shapes are tuned per grid
 * shape once per process and shared by equal shapes. */
typedef struct sdft_ipm_batch sdft_ipm_batch;

/* Create a batch.  ndims[i], dims[3i .. 3i + ndims[i] - 1], masks[i], ys[i] and
 * lambdas[i] describe problem i exactly as for ipm_create (host or device
 * pointers, copied).  One options struct (NULL = defaults) and one stream for
 * all.  On failure nothing is kept and ipm_last_error(NULL) names the problem. */
ipm_status ipm_create_batch(sdft_ipm_batch** out, int count, const int* ndims, const int64_t* dims,
                            const uint8_t* const* masks, const double* const* ys, const double* lambdas,
                            const ipm_options* opt, void* stream);

/* Solve every problem of the batch from the cold start of Sec. 3.3 in one graph
 * launch; results (may be NULL) receives `count` entries (seconds = the wall
 * time of the whole batch).  Returns IPM_OK when every problem reached gap_tol,
 * else the status of the first problem that did not. */
ipm_status ipm_solve_batch(sdft_ipm_batch* b, ipm_result* results);

/* Number of problems; the handle of problem i (owned by the batch: use it for
 * ipm_get_spectrum, ipm_get_point, ... but never destroy it); NULL if out of range. */
int ipm_batch_size(const sdft_ipm_batch* b);
sdft_ipm* ipm_batch_member(sdft_ipm_batch* b, int i);

/* Message of the last failure of the batch (NULL: of the last failed create). */
const char* ipm_batch_last_error(const sdft_ipm_batch* b);

/* Destroy the batch and every member handle.  NULL is accepted. */
void ipm_destroy_batch(sdft_ipm_batch* b);

/* ---- learned warm start ---------------------------------------------------
 * Not in the paper (which cold-starts its IPM).  A 4-layer 3D convolution
 * network (3x3x3 kernels, 8 -> 32 -> 32 -> 32 -> 4 channels, BF16 weights and
 * activations, FP32 accumulation on tensor cores) runs over the grid of
 * half-spectrum slots of a handle.  Its inputs per slot are
 * [c0, c1, soft(c0,1), soft(c1,1), |c|, kl/(Hl-1), f0, f1] with (c0, c1) the
 * slot's coordinates of M_perp^T b / lambda and f_i = min(k_i, N_i - k_i)/(N_i/2);
 * its outputs y correct the soft-threshold guess, beta0 = lambda (soft(c) + y[0:2]),
 * and give logits y[2:4] of "coordinate non-zero".  ws_predict turns them into a
 * strictly interior start point with every s_i nu_i = mu0 = mu_scale lambda^2:
 * z = |beta0| + (mu0/lambda)(2 - p), s1 = z + beta0, s2 = z - beta0, nu = mu0 / s.
 * The cold start of ipm_solve remains the fallback: a handle solves from the
 * predicted point only on the next ipm_solve after ws_predict. */
typedef struct sdft_ws sdft_ws;

/* A network with He-uniform weights from a counter-based hash of seed. */
ipm_status ws_create(sdft_ws** out, uint64_t seed, void* stream);
void ws_destroy(sdft_ws* net);
/* Number of FP32 parameters; copy them out / in (host or device pointers). */
int64_t ws_num_params(const sdft_ws* net);
ipm_status ws_get_params(sdft_ws* net, float* dst);
ipm_status ws_set_params(sdft_ws* net, const float* src);
/* Gradients of the last ws_train_step (same layout as the parameters). */
ipm_status ws_get_grads(sdft_ws* net, float* dst);
/* Outputs y of the network on handle h (FP32, 8 per slot, 4 used; y may be NULL). */
ipm_status ws_forward(sdft_ws* net, sdft_ipm* h, float* y);
/* Predict and set the start point of h's next ipm_solve (mu_scale > 0). */
ipm_status ws_predict(sdft_ws* net, sdft_ipm* h, double mu_scale);
/* One training step on problem h with target beta_star (device, beta layout,
 * e.g. from ipm_get_point after a solve): loss = mean squared error of y[0:2]
 * against beta* / lambda - soft(c/lambda, 1) plus 0.1 x mean cross-entropy of the
 * logits against 1[|beta*| > 1e-6 lambda], over LASSO coordinates.  Gradients by
 * the hand-written backward kernels; an Adam step (betas 0.9, 0.999) when lr > 0.
 * *loss (may be NULL) receives the loss before the step. */
ipm_status ws_train_step(sdft_ws* net, sdft_ipm* h, const double* beta_star, float lr, double* loss);
/* The convolution kernels on caller buffers (device pointers, BF16 as uint16):
 * x [V][cin], w [27][cout][cin] (tap (a+1)*9 + (b+1)*3 + (c+1) for offset (a,b,c)),
 * bias [cout] or NULL, aux [V][cout] or NULL (output multiplied by aux > 0),
 * y [V][cout] FP32; (cin, cout) in {16, 32} x {8, 32}; V = d0 d1 d2. */
ipm_status ws_conv_forward(int cin, int cout, int d0, int d1, int d2, const uint16_t* x, const uint16_t* w,
                           const float* bias, int relu, const uint16_t* aux, float* y, void* stream);
/* Failure-detection test of the tensor-core convolution pipeline (not for
 * production use): the NEXT ws_conv_forward / network call that runs the
 * tcgen05 kernel skips, in every CTA, the copy of its input triple number
 * drop_triple (>= 1) together with its barrier arrival, and every pipeline wait
 * gives up after 2^wait_log2 polls (8..24).  That call must then return
 * IPM_TIMEOUT ("a pipeline wait expired") without hanging, and the context
 * stays usable.  IPM_ERR_ARG for out-of-range arguments. */
ipm_status ws_test_conv_stall(int drop_triple, int wait_log2);
/* Weight and bias gradients of such a convolution: dw[t][o][i] = sum_v dy[v][o]
 * x[v + off(t)][i] for o < mout (dy [V][m], m in {16, 32}), db[o] = sum_v dy[v][o]. */
ipm_status ws_conv_wgrad(int cin, int m, int mout, int d0, int d1, int d2, const uint16_t* x, const uint16_t* dy,
                         float* dw, float* db, void* stream);

/* The chosen FFT tile plan of every pass (FP64 and FP32 variants) as a JSON
 * object written into buf (at most len bytes, NUL-terminated); returns the
 * full length.  For logs and benchmarks. */
int ipm_describe(const sdft_ipm* h, char* buf, int len);

/* Message of the last failure on this handle (or of the last failed create
 * when h is NULL).  Owned by the library. */
const char* ipm_last_error(const sdft_ipm* h);

/* Free every device buffer of the handle.  NULL is accepted. */
void ipm_destroy(sdft_ipm* h);

#ifdef __cplusplus
}
#endif

#endif /* SDFT_IPM_H */
