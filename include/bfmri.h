/*
 * bfmri -- GB300 (sm_103a) sampler for the spatial Bayesian fMRI GLM of
 * Siden, Eklund, Bolin & Villani, "Fast Bayesian whole-brain fMRI analysis with spatial 3D
 * priors" (the "paper" below).
 *
 * Model (Section 2; Appendix A, temporal noise model): Y = X W + E for T time points and N
 * in-mask voxels, AR(P) noise per voxel with coefficients A (P x N) and innovation
 * precisions lambda (N), priors W_k ~ N(0, (alpha_k D_w)^-1) and A_p ~ N(0, (beta_p D_a)^-1)
 * with D_w = D_a the unweighted graph Laplacian (UGL) of the in-mask voxel lattice, Gamma
 * hyperpriors on lambda, alpha, beta.
 *
 * Conventions for every call:
 *  - Every function returns a bfmri_status: BFMRI_OK (0) or a negative error code; no C++
 *    exception crosses this boundary. bfmri_last_error() gives a message.
 *  - Matrices indexed by voxel use the mask's compact raster order (x fastest, then y, then
 *    z), independent of the device layout. W is K x N row-major (the paper's W), A is P x N
 *    row-major, lambda is N, alpha is K, beta is P. All FP64.
 *  - Unless stated otherwise, pointer arguments are HOST pointers; the library copies them.
 *    Outputs named *_out may be NULL (nothing is copied back).
 *  - A handle is not thread-safe: serialise calls on one handle. All device work of a handle
 *    runs on the CUDA stream given in its options, in issue order.
 *  - Device memory is obtained through the allocator callbacks in the options (the Python
 *    binding routes them to PyTorch's caching allocator); with NULL callbacks the library
 *    calls cudaMalloc / cudaFree itself.
 */
#ifndef BFMRI_H
#define BFMRI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int bfmri_status;

#define BFMRI_OK                 0
#define BFMRI_ERR_INVALID_ARG   -1  /* bad size, NULL pointer, non-finite input, bad option */
#define BFMRI_ERR_OOM           -2  /* the allocator returned NULL */
#define BFMRI_ERR_NOT_SPD       -3  /* a per-voxel block failed its Cholesky factorisation */
#define BFMRI_ERR_NOT_CONVERGED -4  /* PCG hit max_iter; the last iterate is kept */
#define BFMRI_ERR_TIMEOUT       -5  /* a device-side grid barrier waited past its limit */
#define BFMRI_ERR_CUDA          -6  /* a CUDA runtime call failed */
#define BFMRI_ERR_INTERNAL      -7
#define BFMRI_ERR_STATE         -8  /* call out of order, e.g. sampling before statistics */
#define BFMRI_PENDING            1  /* server: the request has not finished yet (not an error) */

/* Voxel lattice: nx * ny * nz sites; neighbourhood 6 (3D: +-x, +-y, +-z) or 4 (slice-wise
 * 2D: +-x, +-y only). The UGL prior of Section 2 links in-mask face neighbours. */
typedef struct {
  int nx, ny, nz;
  int neighbourhood;
} bfmri_lattice;

#define BFMRI_F32 0
#define BFMRI_F64 1

#define BFMRI_PRECOND_NONE         0
#define BFMRI_PRECOND_BLOCK_JACOBI 1  /* per-voxel (block + alpha * degree) Cholesky */
#define BFMRI_PRECOND_SSOR         2  /* red-black symmetric SOR over those voxel blocks:
                                         M = (Dg + w L) Dg^-1 (Dg + w U) / (w (2 - w)), w =
                                         ssor_omega, red = voxels with x + y + z even. Single
                                         solves (FP64, and the FP32 inner iterations of mixed),
                                         SVB samples and grouped chains; the log-det / trace
                                         probes always use block-Jacobi */
#define BFMRI_PRECOND_RB_REDUCED   3  /* CG on the red-black reduced system (the black
                                         voxels' Schur complement S = Dg_b - L Dg_r^-1 U,
                                         preconditioned by Dg_b; for D <= 6 the FP64
                                         resident solver runs it in the split form
                                         L_b^-1 S L_b^-T, Dg_b = L_b L_b'), which takes the
                                         iterates of SSOR with omega = 1 at fewer barriers
                                         and block products per iteration. The FP64 and
                                         mixed resident solvers, the mixed streaming solver
                                         and the multi-RHS solver (at most one right-hand
                                         side per warp) run it; the FP64 streaming solver
                                         and larger batches use SSOR with omega = 1 */

#define BFMRI_PRECOND_MULTIGRID    4  /* aggregation multigrid V-cycle (a replacement of
                                         Section 3.1's incomplete Cholesky): levels of 2x2x2
                                         aggregates (2x2 in-slice for the 4-neighbour
                                         prior), at most 3, Galerkin coarse operators (summed
                                         blocks, coarse Laplacian of the summed fine edge
                                         weights), red-black block Gauss-Seidel smoothing
                                         (red, black before the coarse correction; black, red
                                         after), two symmetric red-black steps on the
                                         coarsest level; single FP64 W and A solves (the
                                         multi-RHS and mixed-precision solves use
                                         block-Jacobi) */

#define BFMRI_PREC_FP64  0  /* FP64 PCG */
#define BFMRI_PREC_MIXED 1  /* FP32 inner PCG inside an FP64 iterative-refinement loop */

#define BFMRI_AR_SPATIAL     0  /* A_p ~ N(0, (beta_p D_a)^-1), D_a = D_w (paper's model) */
#define BFMRI_AR_INDEPENDENT 1  /* no spatial prior on A: per-voxel AR draws, beta unused */

#define BFMRI_Y_MASKED  0  /* Y is T x N, columns = in-mask voxels in compact order */
#define BFMRI_Y_LATTICE 1  /* Y is T x (nx ny nz), columns = all lattice sites */

typedef void* (*bfmri_alloc_fn)(size_t bytes, void* ctx);
typedef void (*bfmri_free_fn)(void* ptr, void* ctx);

typedef struct {
  /* Gamma hyperpriors Ga(scale, shape) of Section 2: q1, q2 (alpha), u1, u2 (lambda),
   * r1, r2 (beta). Defaults 10, 0.1, 10, 0.1, 10000, 0.1. */
  double q1, q2, u1, u2, r1, r2;
  double eps;          /* ridge added to every per-voxel data block of W (default 0) */
  double delta;        /* PCG stop: true relative residual ||b - B x|| / ||b|| <= delta */
  int max_iter;        /* PCG iteration cap per solve (default 2000) */
  int precond;         /* BFMRI_PRECOND_* (default block-Jacobi) */
  int precision;       /* BFMRI_PREC_* (default FP64) */
  int ar_prior;        /* BFMRI_AR_* (default spatial) */
  int y_layout;        /* BFMRI_Y_* (default masked) */
  double inner_tol;    /* mixed precision: relative tolerance of each FP32 inner solve
                          (default 1e-6; the last one stops where the outer delta is met) */
  uint64_t seed;       /* Philox key */
  uint32_t stream_id;  /* 24-bit chain id folded into every Philox counter */
  void* cuda_stream;   /* cudaStream_t for all device work (NULL = legacy default stream) */
  bfmri_alloc_fn dev_alloc;  /* device allocator (NULL: cudaMalloc) */
  bfmri_free_fn dev_free;
  void* alloc_ctx;
  double barrier_timeout_s;  /* limit of each device-side grid-barrier wait (default 2 s) */
  int debug_skip_block;      /* test hook: this CTA never arrives at the first barrier of the
                                next solve (forces BFMRI_ERR_TIMEOUT); -1 = off (default) */
  int profile;               /* 1: time every kernel launch with CUDA events on the handle's
                                stream; 2: time only the single-solve PCG launches (less
                                overhead); read with bfmri_get_timing. 0 (default): off */
  int pcg_variant;           /* BFMRI_PCG_AUTO (default): the register-resident solver when the
                                voxels fit one CTA per SM, else the streaming one;
                                BFMRI_PCG_STREAMING: always the streaming solver */
  int sm_budget;             /* most SMs one solver grid may span (0 = all). Concurrent
                                handles whose budgets sum to at most the SM count can run
                                their cooperative solves side by side. */
  double ssor_omega;         /* relaxation of BFMRI_PRECOND_SSOR, in (0, 2) (default 1:
                                symmetric Gauss-Seidel) */
  int use_graph;             /* nonzero: bfmri_gibbs_sweep replays one captured CUDA graph
                                per sweep (captured at the first call; the draw counter lives
                                in device memory and the graph advances it), with the same
                                results as direct launches. On the first handle of a
                                bfmri_gibbs_sweep_group call it does the same for the group's
                                sweeps (one graph per list of chains, kept while the chains
                                and the group's workspace stay the same; not for the sweep of
                                bfmri_gibbs_sweep_group_probes). Ignored while profile or
                                debug_skip_block is set, or while a chain summary is open in a
                                group; if capture is unavailable the handle falls back to
                                direct launches. Default 0. */
  double edge_weight[3];     /* weighted graph-Laplacian (WGL) prior (Discussion): the prior
                                precision of W_k is alpha_k G_w' C G_w (and that of A_p is
                                beta_p G_w' C G_w) with C the weight of each edge's direction
                                x, y, z, e.g. from anisotropic voxel sizes; Algorithm 2 scales
                                each edge's noise by sqrt(C). All > 0; default 1, 1, 1 (the
                                UGL prior of Section 2). */
  int stats_kernel;          /* sufficient statistics of FP32 series: BFMRI_STATS_AUTO
                                (default: the tensor-core kernel where it applies, P <= 3
                                and K <= 16, else FP64 CUDA cores), BFMRI_STATS_FP64 (always
                                the FP64 CUDA-core kernel) or BFMRI_STATS_TENSOR (the
                                tensor-core kernel, INVALID_ARG where it does not apply).
                                FP64 series always take the FP64 kernel. */
  int mrhs_tile;             /* FP32 log-det / trace probe solves: right-hand sides per thread
                                (1, 2 or 4, interleaved per voxel and component); 0 (default):
                                the autotuner times 1, 2 and 4 on the first probe call of each
                                shape (K or P, probe count, N, sm_budget) and keeps the fastest
                                for the process (bfmri_probe_tuning reports it) */
  int w_prior;               /* spatial prior of W: BFMRI_PRIOR_UGL (default: D_w = L, the
                                graph Laplacian of Section 2, weighted by edge_weight) or
                                BFMRI_PRIOR_LTL (D_w = L'L, the alternative Section 2 names:
                                a 25-point stencil in 3D, 13-point in 2D). With LTL, W is
                                solved by FP64 PCG (register-resident where the voxels fit
                                and pcg_variant is AUTO, else streaming) with block-Jacobi (blocks plus
                                diag(alpha) times the diagonal of L'L) or no preconditioner
                                (precond BLOCK_JACOBI or NONE, precision FP64, else INVALID_ARG
                                at create); the A prior stays the graph Laplacian; grouped
                                sweeps, probes and SVB steps reject LTL handles with
                                INVALID_ARG; the log joint takes |L w_k|^2 in its W prior
                                term. BFMRI_PRIOR_ANISO: the anisotropic prior with random
                                alpha per direction (see its #define). */
  int pcg_lanes;             /* lanes of the register-resident FP64 solver on the red-black
                                reduced system (BFMRI_PRECOND_RB_REDUCED, K or P <= 6):
                                2 = lane pairs, each pair holding one red and one black voxel
                                and each lane half of their components (block products by
                                rows, neighbour sums and updates by components); 1 = one lane
                                per voxel; 0 (default) = lane pairs for 6 x 6 blocks, one lane
                                otherwise. Same iterates up to rounding. */
  double aniso_step;         /* BFMRI_PRIOR_ANISO: standard deviation of the log-normal
                                random-walk proposal of the exchange step (log alpha_{d,k}
                                moves by aniso_step times a standard normal); <= 0 (default 0)
                                means 1 / sqrt(N). */
} bfmri_options;

#define BFMRI_PRIOR_UGL 0
#define BFMRI_PRIOR_LTL 1
/* The anisotropic prior the Discussion proposes: the prior precision of W_k is
 * G_w' C_k G_w with C_k = diag(alpha_x,k I, alpha_y,k I, alpha_z,k I) (times edge_weight),
 * the alpha_{d,k} random with the Ga(q1, q2) prior of alpha. The paper leaves its inference
 * open because the prior's determinant no longer factors out of the alphas; the alphas are
 * updated here in two moves per k. First the common scale, exactly: alpha -> lam alpha with
 *   lam ~ Ga(shape nd q2 + (N - c)/2, rate sum_d alpha_d (1/q1 + Q_d(w)/2))
 * (the posterior along that ray; nd directions, c connected parts of the voxel graph, the
 * Gamma generator of alpha with Philox tag 4, site k). Then the exchange algorithm (Murray,
 * Ghahramani & MacKay, UAI 2006), which needs no determinant, for the ratios between the
 * directions: a log-normal random-walk proposal theta' (normals from Philox tag 7,
 * site k, subs 0-1), an auxiliary field w' drawn from the prior at theta' by the Algorithm 2
 * perturbation without a data term (edge normals from tag 8) and PCG from zero to delta, and
 * acceptance when log u < log a (u from tag 7, site k, sub 2) with
 *   log a = sum_d [ -(theta'_d - theta_d)(Q_d(w) - Q_d(w')) / 2
 *                   + q2 (log theta'_d - log theta_d) - (theta'_d - theta_d) / q1 ],
 * Q_d the direction-d edge sums. W and the auxiliary field are solved by FP64 PCG (the
 * register-resident kernels where the voxels fit and pcg_variant is AUTO, else the streaming
 * one) with block-Jacobi (blocks plus diag_k sum_d alpha_{d,k} deg_d; for the auxiliary
 * field, Jacobi on sum_d theta'_d deg_d), with CG on the red-black reduced system built on
 * those blocks (precond RB_REDUCED, K <= 6, where the voxels fit the resident kernel; else
 * block-Jacobi streaming on the same blocks), or with no preconditioner; other precond values
 * or a precision other than FP64 are INVALID_ARG at create; bfmri_apply_preconditioner
 * rejects W under RB_REDUCED. The A prior stays the graph Laplacian. Grouped
 * sweeps, probes, SVB steps, the log joint and per-edge factors reject it (INVALID_ARG).
 * bfmri_set_state's alpha sets alpha_{d,k} = alpha_k for every d; bfmri_get_state's alpha
 * returns the mean over the lattice's directions; bfmri_sample_alpha runs the ray move and
 * one exchange step for every k (the sweep's alpha step). */
#define BFMRI_PRIOR_ANISO 2

#define BFMRI_STATS_AUTO   0
#define BFMRI_STATS_FP64   1
#define BFMRI_STATS_TENSOR 2

#define BFMRI_PCG_AUTO      0
#define BFMRI_PCG_STREAMING 1

/* Fills *opt with the defaults listed above. */
void bfmri_default_options(bfmri_options* opt);

typedef struct bfmri_handle bfmri_handle;

typedef struct {
  int iterations;        /* PCG iterations (mixed: total inner FP32 iterations) */
  int refinements;       /* mixed: FP64 outer refinement steps; FP64: true-residual restarts */
  double rel_residual;   /* final true relative residual in FP64 */
  double rel_residual0;  /* relative residual of the starting value */
} bfmri_solve_info;

typedef struct {
  int sweeps;
  long long pcg_iterations_W;  /* summed over sweeps */
  long long pcg_iterations_A;
  double last_rel_residual_W;
  long long gamma_exhausted;   /* Marsaglia-Tsang draws that used all attempts */
  int captured;                /* 1 when the sweeps ran as replays of a captured CUDA graph */
} bfmri_sweep_info;

/* Creates a handle for one subject (paper Section 2, Eq. Pennymodel; Appendix A).
 *  lat, mask: lattice and nx*ny*nz mask bytes (x fastest; nonzero = in mask).
 *  X: T x K design, column-major FP64 (X[t + T k]).
 *  Y: T x N (or T x nx ny nz with y_layout = BFMRI_Y_LATTICE) row-major, element (t, n) at
 *     Y[t * N + n], FP32 or FP64 per y_dtype. Copied to the device; the host array is not
 *     referenced after return.
 *  K in [1, 12], P in [0, 4], T > P + K.
 * The state starts at the prior means (Appendix C, trick 2): W = 0, A = 0, lambda = u1 u2,
 * alpha = q1 q2, beta = r1 r2. Errors: INVALID_ARG (sizes, empty mask, non-finite X or Y),
 * OOM, CUDA. On error *out is NULL; the message is available from bfmri_last_error(NULL). */
bfmri_status bfmri_create(const bfmri_lattice* lat, const uint8_t* mask, const double* X,
                          const void* Y, int y_dtype, int T, int K, int P,
                          const bfmri_options* opt, bfmri_handle** out);

/* Releases all device memory of the handle (after synchronising its stream). NULL is a no-op. */
bfmri_status bfmri_destroy(bfmri_handle* h);

/* Message of the last failed call on h (handle-owned), or of the last failed bfmri_create
 * when h is NULL (process-wide). Never NULL. */
const char* bfmri_last_error(const bfmri_handle* h);

/* Number of in-mask voxels N, and the problem sizes. */
int bfmri_num_voxels(const bfmri_handle* h);
/* Device bytes the handle holds now and at most so far (its own allocations, each as
 * requested from the allocator: rounded up to 256 bytes). */
bfmri_status bfmri_device_bytes(const bfmri_handle* h, size_t* now, size_t* peak);
/* Right-hand-side tile of the handle's last probe solve, and the autotuner's solve times in
 * ms for tiles 1, 2 and 4 (ms[3], -1 where not timed: a cached or fixed choice). */
bfmri_status bfmri_probe_tuning(const bfmri_handle* h, int* tile, double* ms);
bfmri_status bfmri_sizes(const bfmri_handle* h, int* N, int* T, int* K, int* P);

/* Sufficient statistics (Appendix A, Eq. log-like: Y enters only through lagged
 * cross-products, "pre-computed outside the Gibbs algorithm"). For every voxel and lags
 * p, q in 0..P, summed over t = P+1..T:
 *   Syy[p][q]    = sum_t y_{t-p} y_{t-q}              (p <= q stored)
 *   Sxy[p][q][k] = sum_t y_{t-p} x_{t-q,k}
 * The device copy of Y is released afterwards. Must precede every sampling call.
 * FP32 series (the serving input) take, where options.stats_kernel allows, the tensor-core
 * kernel: the common-window products sum_s y_s x_{s+d,k} as an exact BF16 digit product
 * (every FP32 value of Y that is within 2^-24 of its voxel's largest value is represented
 * exactly; X to 48 bits relative to its column's largest value; the digit levels below
 * 2^-48 of the leading one are dropped), the rest in FP64. Errors: TIMEOUT if a pipeline
 * wait of that kernel gave up. */
bfmri_status bfmri_precompute_stats(bfmri_handle* h);

/* Copies the statistics to the host: out is N x S row-major with S = (P+1)(P+2)/2 + K (P+1)^2,
 * per voxel first Syy (p <= q, row-major over p), then Sxy in (p, q, k) order. */
bfmri_status bfmri_get_stats(bfmri_handle* h, double* out);

/* Per-edge weights of the spatial prior: a general diagonal C in D_w = G_w' C G_w (Eq. 7
 * with C the edge weights of the WGL prior in the Discussion; here one weight per edge instead
 * of per direction). factors is host memory, [3][nx*ny*nz] float32, indexed by direction
 * (x, y, z) and lattice-linear site x + nx (y + ny z): entry [d][site] multiplies
 * options.edge_weight[d] for the edge from that site to its +d neighbour; entries of
 * sites outside the mask or of edges leaving it are not read, the z plane is not read with
 * the 4-neighbourhood. Each factor is rounded to the nearest BF16 (ties to even) and kept on
 * the device, 2 bytes per voxel and direction; the rounded value is the factor the model
 * uses everywhere (W and A precisions, the perturbation's sqrt(C) G_w noise of Algorithm 2,
 * the alpha and beta quadratic forms). The caller keeps ownership of factors. NULL removes
 * the factors (back to per-direction weights). Needs the graph-Laplacian prior, precision
 * FP64 and precond RB_REDUCED (CG on the red-black reduced system, K or P <= 6, where the
 * voxels fit the register-resident kernel; else block-Jacobi streaming on the same blocks),
 * BLOCK_JACOBI or NONE, else INVALID_ARG; bfmri_apply_preconditioner rejects such a handle
 * under RB_REDUCED; factors
 * must be positive and finite, else INVALID_ARG with nothing changed. With factors set,
 * grouped sweeps, probes and SVB steps reject the handle with INVALID_ARG; the log joint takes
 * the factors in its edge sums (their pseudo-determinant does not depend on the sampled
 * parameters and is left out with the other constants).
 * Drops a captured sweep graph. Errors: INVALID_ARG, OOM, CUDA. */
bfmri_status bfmri_set_edge_factors(bfmri_handle* h, const float* factors);

/* Anisotropic prior (BFMRI_PRIOR_ANISO only, else INVALID_ARG): sets / reads alpha_{d,k}.
 * alpha is host memory, K x 3 row-major (x, y, z per k; the z entry of a 4-neighbourhood
 * lattice is kept but not used); values must be positive and finite (INVALID_ARG, nothing
 * changed). accepted (K, may be NULL) receives the exchange steps accepted per k since the
 * handle was created. */
bfmri_status bfmri_set_alpha_dirs(bfmri_handle* h, const double* alpha);
bfmri_status bfmri_get_alpha_dirs(bfmri_handle* h, double* alpha, long long* accepted);

/* Anisotropic prior: the last alpha step's quantities (any pointer may be NULL): Q and
 * Q_aux (K x 3) the direction edge sums of W and of the auxiliary field, log_a (K) the log
 * acceptance ratio, lam (K) the ray move's factor, w_aux (K x N) the auxiliary field (its
 * constant part along each connected component is whatever PCG from zero left there; the
 * edge sums ignore it). */
bfmri_status bfmri_aniso_last_step(bfmri_handle* h, double* Q, double* Q_aux, double* log_a,
                                   double* lam, double* w_aux);

/* Sets / reads the chain state (any pointer may be NULL to leave that part unchanged / not
 * read). Values are validated: lambda, alpha, beta > 0 and finite. */
bfmri_status bfmri_set_state(bfmri_handle* h, const double* W, const double* A,
                             const double* lambda, const double* alpha, const double* beta);
bfmri_status bfmri_get_state(bfmri_handle* h, double* W, double* A, double* lambda,
                             double* alpha, double* beta);

/* One draw of W from its full conditional (Eq. full cond W temporal) by Algorithm 2:
 * b = b_w + sum_k sqrt(alpha_k) G_w' z1_k + H_w' L_data H_w z2 (normals from Philox with
 * draw counter `counter`), then PCG on B~ w = b from the current W (warm start) until the
 * true relative residual is <= delta. The draw replaces W in the state; W_out (K x N) may be
 * NULL. info may be NULL; when given, the call waits for the device.
 * Errors: STATE (no statistics), NOT_SPD, NOT_CONVERGED, TIMEOUT, CUDA. */
bfmri_status bfmri_sample_W(bfmri_handle* h, uint64_t counter, double* W_out,
                            bfmri_solve_info* info);

/* One draw of A from its full conditional (Eq. fullcondTempA) given the current W, lambda,
 * beta: spatial prior -> the same perturbation + PCG with P in place of K and beta in place
 * of alpha; independent prior -> per-voxel P x P Cholesky draws. No-op when P = 0. */
bfmri_status bfmri_sample_A(bfmri_handle* h, uint64_t counter, double* A_out,
                            bfmri_solve_info* info);

/* lambda_n ~ Ga(1 / (1/u1 + RSS_n / 2), (T - P)/2 + u2) (Eq. fullcondTemplambda). */
bfmri_status bfmri_sample_lambda(bfmri_handle* h, uint64_t counter, double* lambda_out);

/* alpha_k ~ Ga(1 / (W_k D_w W_k' / 2 + 1/q1), N/2 + q2) (Eq. fullcondTempa). */
bfmri_status bfmri_sample_alpha(bfmri_handle* h, uint64_t counter, double* alpha_out);

/* beta_p ~ Ga(1 / (A_p D_a A_p' / 2 + 1/r1), N/2 + r2) (Eq. fullcondTempbeta); spatial AR
 * prior only (a no-op otherwise). */
bfmri_status bfmri_sample_beta(bfmri_handle* h, uint64_t counter, double* beta_out);

/* n_sweeps Gibbs sweeps (Section 3.2) W -> A -> lambda -> alpha -> beta; sweep s uses draw
 * counter first_counter + s.
 * info != NULL: the call waits for the sweeps and reports their errors and counts.
 * info == NULL: the call only enqueues the sweeps on the handle's stream and returns
 * BFMRI_OK (argument and launch errors are still returned at once). The device-side error
 * words and PCG counters then accumulate over such calls until a synchronising call reads
 * them: the next bfmri_gibbs_sweep with info, any other compute call, or bfmri_synchronize;
 * that call reports the first error of the whole span and its counts cover the whole span. */
bfmri_status bfmri_gibbs_sweep(bfmri_handle* h, int n_sweeps, uint64_t first_counter,
                               bfmri_sweep_info* info);

/* Waits for the handle's enqueued work and reports the errors of the calls since the last
 * synchronising call (see bfmri_gibbs_sweep). info (may be NULL) receives the PCG counts of
 * that span (sweeps = 0). Errors: as bfmri_gibbs_sweep, CUDA. */
bfmri_status bfmri_synchronize(bfmri_handle* h, bfmri_sweep_info* info);

/* n independent chains advanced together, each by n_sweeps Gibbs sweeps of Section 3.2
 * (the chains are the handles hs[0..n-1], each with its own state and seed, so their draws
 * are independent). Each sweep step runs for every chain; the n W systems (one matrix per
 * chain) are solved by one cooperative multi-right-hand-side PCG launch, which shares its
 * barriers and reductions among the chains, and likewise the n A systems under the spatial
 * AR prior. Chain c's draws follow the same equations, random numbers and stop rule
 * (relative residual <= delta, confirmed by the true residual) as bfmri_gibbs_sweep on
 * hs[c]; they agree with it to the solver tolerance, not bitwise.
 * The chains may be different subjects on different lattices and masks (uneven masks): every
 * right-hand side of the launch then carries its own lattice, and the launch's work units
 * are shared out in proportion to the chains' voxels.
 * Requirements: 1 <= n <= 64; equal K, P, AR prior, delta, max_iter and preconditioner (and
 * ssor_omega under SSOR), FP64 precision, statistics precomputed, on the current device.
 * All work runs on hs[0]'s stream; the call returns when it has finished.
 * info: [n] per-chain results (may be NULL). hs and info are host arrays the caller owns.
 * Errors: INVALID_ARG (mismatched or bad handles), STATE, NOT_SPD, NOT_CONVERGED, TIMEOUT,
 * CUDA; on error the states of all n chains are unspecified. */
bfmri_status bfmri_gibbs_sweep_group(bfmri_handle* const* hs, int n, int n_sweeps,
                                     uint64_t first_counter, bfmri_sweep_info* info);

/* One Gibbs sweep of the chains hs[0..n-1] (as bfmri_gibbs_sweep_group with n_sweeps = 1,
 * draw counter `counter`) whose W step solves, in the same cooperative launch as the n
 * chains' W systems (one matrix per chain), n_probes log-determinant probes of the W
 * precision B~ of probe_handle at its current state (one matrix, n_probes right-hand sides;
 * as bfmri_logdet_probe with which = 0, probe draws from probe_counter, lanczos_steps CG
 * coefficients recorded per probe). probe_handle may be one of the chains (then the probes
 * see the system of that chain's W draw in this sweep) or another handle with the chains' K
 * (FP64), on any lattice. The Lanczos quadrature needs plain block-Jacobi PCG, so this launch
 * solves every right-hand side with block-Jacobi, whatever the chains' preconditioner; the
 * chains' A systems use their own. Outputs as bfmri_logdet_probe: logdet, std_err (may be
 * NULL), per_probe [n_probes] (may be NULL); info [n] per chain (may be NULL).
 * Requirements: those of bfmri_gibbs_sweep_group; 1 <= n_probes <= 127; with different
 * lattices among the chains and probe_handle, n + n_probes <= 128.
 * Errors: those of bfmri_gibbs_sweep_group and bfmri_logdet_probe. */
bfmri_status bfmri_gibbs_sweep_group_probes(bfmri_handle* const* hs, int n, uint64_t counter,
                                            bfmri_handle* probe_handle, int n_probes,
                                            int lanczos_steps, uint64_t probe_counter,
                                            double* logdet, double* std_err, double* per_probe,
                                            bfmri_sweep_info* info);

/* Log-determinant and trace probes of the W (which = 0) or A (which = 1) full-conditional
 * precision B~ at the current state. The paper leaves the log-determinant to future work
 * (Discussion: model evidence, collapsed alpha); this is stochastic Lanczos quadrature:
 *   log det B~ = log det M + tr log(L^-1 B~ L^-T),  M = L L' the block-Jacobi preconditioner,
 * with n_probes Rademacher vectors v_i (Philox, draw counter `counter`, stream = probe
 * index), each solved by the multi-right-hand-side PCG from x = 0 on B~ x = L v_i to relative
 * residual `delta` of the options (at most lanczos_steps iterations, whose CG coefficients
 * form the Lanczos tridiagonal T_i): estimate_i = ||v_i||^2 e1' log(T_i) e1.
 *  logdet   : log det M + mean_i estimate_i
 *  std_err  : standard error of the mean over probes (may be NULL)
 *  traces   : dim values, mean_i (L^-T v_i)' D_w^(k) y_i with y_i = B~^-1 L v_i, an unbiased
 *             estimate of tr(D_w^(k) B~^-1), the trace term of the SVB alpha update
 *             (Eq. quad-form-expectation); may be NULL
 *  per_probe: n_probes values estimate_i (may be NULL)
 *  iterations: n_probes PCG iteration counts (may be NULL)
 * With precision BFMRI_PREC_MIXED the probe solves run in FP32 storage and arithmetic per
 * voxel (CG scalars, inner-product sums, quadrature and log det accumulation in FP64); use a
 * delta an FP32 recurrence can reach (e.g. 1e-5).
 * Errors: STATE, NOT_CONVERGED (a probe hit lanczos_steps), NOT_SPD, CUDA, OOM. */
bfmri_status bfmri_logdet_probe(bfmri_handle* h, int which, int n_probes, int lanczos_steps,
                                uint64_t counter, double* logdet, double* std_err,
                                double* traces, double* per_probe, int* iterations);

/* One spatial-VB iteration (Section 3.3; Appendix B, Eq. NFVBw / NFVBbB; Appendix C).
 * The handle's lambda, alpha, beta are the current means E[lambda], E[alpha], E[beta]; the
 * handle keeps n_samples samples of W and A (created from the current W and A on the first
 * call or when n_samples changes, later samples kept as warm starts):
 *  1. q(W): per-voxel blocks and right-hand sides averaged over the A samples with E[lambda],
 *     and E[alpha] on the prior; n_samples draws by Algorithm 2 with the SAME random numbers
 *     at every iteration (draw counter `counter`, stream = sample index), solved together by
 *     the multi-right-hand-side PCG from the previous samples;
 *  2. q(A): the same with the lagged residual Gram averaged over the new W samples;
 *  3. E[lambda_n] from the mean over sample pairs of RSS_n (paired by index);
 *  4. E[alpha_k] (E[beta_p]) from the mean over samples of W_k D_w W_k' (A_p D_a A_p');
 *     with `extrapolate`, every other iteration from the third on, Appendix C's trick 1.
 * alpha_vb / beta_vb (may be NULL) receive the VB values before the extrapolation. */
typedef struct {
  int iteration;               /* SVB iterations run on this handle */
  int samples;
  long long pcg_iterations_W;  /* summed over samples */
  long long pcg_iterations_A;
  double max_rel_residual_W;
  int extrapolated;            /* 1 if trick 1 replaced the VB value this iteration */
} bfmri_svb_info;
bfmri_status bfmri_spvb_step(bfmri_handle* h, int n_samples, uint64_t counter, int extrapolate,
                             double* alpha_vb, double* beta_vb, bfmri_svb_info* info);
/* Read / overwrite SVB sample j (W is K x N, A is P x N; either may be NULL). */
bfmri_status bfmri_svb_get_sample(bfmri_handle* h, int j, double* W, double* A);
bfmri_status bfmri_svb_set_sample(bfmri_handle* h, int j, const double* W, const double* A);

/* ---- Posterior summaries -----------------------------------------------------------
 * Voxel-indexed outputs are row-major with N columns in the compact order of the mask;
 * covariances are packed per voxel: row i (i + 1) / 2 + j holds Cov(W_i,n, W_j,n), j <= i.
 * Contrasts: C is n_contrasts x K row-major, gamma has n_contrasts thresholds,
 * 0 <= n_contrasts <= BFMRI_MAX_CONTRASTS; a contrast value c'W_.,n is summed over k in
 * order with one rounding per product and per addition (no fused multiply-add). */
#define BFMRI_MAX_CONTRASTS 16

/* Opens a chain summary (Section 3.2): from now on every Gibbs sweep of this handle
 * (bfmri_gibbs_sweep, bfmri_gibbs_sweep_group) adds its W draw as one sample, on the device:
 * per voxel the sample moments of W_.,n (shifted by the W at this call), per voxel and
 * contrast the number of samples with c'W_.,n > gamma (the marginal PPM of Eq. MCMCPPM), and
 * per contrast the number of samples in which every voxel of joint_set exceeds gamma (the
 * joint probability of Eq. MCMCjointPPM; joint_set holds n_joint compact voxel indices, may
 * repeat; with n_joint = 0 every sample counts). Reopening discards the previous summary.
 * The captured sweep graph (options.use_graph) is re-captured with the accumulation.
 * Errors: INVALID_ARG (contrasts, indices), OOM, CUDA. */
bfmri_status bfmri_summary_begin(bfmri_handle* h, int n_contrasts, const double* C,
                                 const double* gamma, const int* joint_set, int n_joint);

/* Adds the current W as one sample (enqueued on the handle's stream; no host wait). */
bfmri_status bfmri_summary_add(bfmri_handle* h);

/* Waits for the handle's work (reporting errors of asynchronous sweeps) and reads the open
 * summary: n_samples; mean (K x N); cov (K(K+1)/2 x N, divisor n - 1, zero for n = 1);
 * ppm (n_contrasts x N, count / n); joint_count (n_contrasts; joint PPM = count / n). Any
 * output may be NULL. Errors: STATE (no summary, or outputs asked with no sample). */
bfmri_status bfmri_summary_get(bfmri_handle* h, long long* n_samples, double* mean, double* cov,
                               double* ppm, long long* joint_count);

/* Closes the summary and frees its device memory (no-op when none is open). */
bfmri_status bfmri_summary_end(bfmri_handle* h);

/* Summary of the N_s SVB samples of q(W) held by the handle (Section 3.3): sample mean
 * (K x N), sample covariance (packed, divisor N_s - 1) and, per contrast, the PPM of the
 * Gaussian with those moments, P(c'W_.,n > gamma) = erfc((gamma - c'mu_n) /
 * sqrt(2 c'Sigma_n c)) / 2 (the indicator c'mu_n > gamma when c'Sigma_n c = 0). Outputs may
 * be NULL. Errors: STATE (no SVB samples), INVALID_ARG, OOM, CUDA. */
bfmri_status bfmri_svb_summary(bfmri_handle* h, int n_contrasts, const double* C,
                               const double* gamma, double* mean, double* cov, double* ppm);

/* Unnormalised log joint posterior at the current state (Appendix A, Eq.
 * UnnormalisedJointPosterior): terms[0] log-likelihood without its constant (Eq. log-like,
 * sums over t = P+1..T), [1] log p~(W | alpha) = sum_k N/2 log alpha_k - alpha_k W_k D_w W_k'/2,
 * [2] the same for A and beta (0 under the independent AR prior), [3..5] the Gamma
 * log-priors of lambda, alpha, beta without constants (Ga(scale, shape)), [6] the total.
 * W_k D_w W_k' is |L W_k'|^2 under the L'L prior and takes per-edge factors in its edge
 * sums; the anisotropic prior is INVALID_ARG (its normaliser, log pdet sum_d alpha_d L_d,
 * does not separate from the alphas). Differences between two states are log posterior
 * ratios. Errors: STATE (statistics not computed), INVALID_ARG, CUDA. */
bfmri_status bfmri_log_joint(bfmri_handle* h, double* terms);

/* Gauss quadrature value e1' log(T) e1 of the Lanczos tridiagonal T built from m CG
 * coefficients (alpha_0..alpha_{m-1}, beta_0..beta_{m-2}) of a preconditioned CG run from
 * x = 0; host-only helper used by bfmri_logdet_probe. */
bfmri_status bfmri_lanczos_log_quadrature(int m, const double* cg_alpha, const double* cg_beta,
                                          double* value);

/* Per-kernel device time, accumulated since the last reset when options.profile is set
 * (CUDA events recorded around each launch on the handle's stream). Classes: */
#define BFMRI_T_STATS      0  /* sufficient statistics */
#define BFMRI_T_ASSEMBLE_W 1  /* W blocks + perturbed rhs + preconditioner */
#define BFMRI_T_PCG_W      2  /* W solve */
#define BFMRI_T_ASSEMBLE_A 3  /* lagged residual Gram + A system */
#define BFMRI_T_PCG_A      4  /* A solve */
#define BFMRI_T_LAMBDA     5
#define BFMRI_T_HYPER      6  /* alpha and beta */
#define BFMRI_T_OTHER      7
#define BFMRI_T_SUMMARY    8  /* posterior summaries and the log joint posterior */
#define BFMRI_T_CLASSES    9
typedef struct {
  double ms[BFMRI_T_CLASSES];
  long long launches[BFMRI_T_CLASSES];
  long long pcg_iterations[BFMRI_T_CLASSES];  /* PCG iterations of the timed solves */
} bfmri_timing;

/* Waits for the handle's stream, then returns the accumulated timing (zeros if profiling is
 * off). bfmri_reset_timing clears it. */
bfmri_status bfmri_get_timing(bfmri_handle* h, bfmri_timing* t);
bfmri_status bfmri_reset_timing(bfmri_handle* h);

/* Inspection of the W or A system (which = 0: W with K, 1: A with P) at the current state.
 *  bfmri_apply_precision: y = B~ x (x, y dim x N row-major) with B~ the full-conditional
 *    precision (block diagonal data term + scale (x) D).
 *  bfmri_build_system: per-voxel data blocks (N x dim x dim, full symmetric), the mean
 *    right-hand side b_w (dim x N) and the perturbed right-hand side b of Algorithm 2
 *    for draw counter `counter` (dim x N). Any output may be NULL. */
bfmri_status bfmri_apply_precision(bfmri_handle* h, int which, const double* x, double* y);
/*  bfmri_apply_preconditioner: y = M^-1 x (dim x N row-major) with M the solver's
 *    preconditioner for the current state's system: block-Jacobi (blocks B_n + diag(scale)
 *    deg_n), identity, red-black SSOR over those blocks, or one multigrid V-cycle
 *    (BFMRI_PRECOND_MULTIGRID; the first call builds the hierarchy). Section 3.1 uses an
 *    incomplete Cholesky factor instead. */
bfmri_status bfmri_apply_preconditioner(bfmri_handle* h, int which, const double* x, double* y);
bfmri_status bfmri_build_system(bfmri_handle* h, int which, uint64_t counter, double* blocks,
                                double* b_mean, double* b_pert);

/* ---------------------------------------------------------------------------------------
 * Serving: many subjects on one GPU with continuous admission.
 *
 * A server owns max_slots slots, each with a host worker thread and a CUDA stream, and a
 * device-memory budget. Submitted requests wait in FIFO order; the oldest starts as soon as
 * a slot is free and its device-memory estimate (bfmri_request_device_bytes) fits in the
 * budget left by the running requests, so requests that arrive while others run are
 * admitted as slots and memory free up, and their kernels overlap on the device. A request
 * runs bfmri_create, bfmri_precompute_stats, n_sweeps Gibbs sweeps (draw counters
 * first_counter, first_counter + 1, ...) and copies the final W (and alpha) to the caller's
 * buffers, then releases its memory. Each slot's solver grids span at most sm_budget SMs
 * (0 = all); budgets whose sum does not exceed the SM count let every slot's cooperative
 * solve be resident at once. A request's result does not depend on what else runs (fixed
 * grids, fixed-order reductions, counter-based random numbers). The server is internally
 * synchronised; the host arrays of a request must stay valid until it completes. */
typedef struct bfmri_server bfmri_server;

typedef struct {
  bfmri_lattice lat;
  const uint8_t* mask;
  const double* X;
  const void* Y;
  int y_dtype;
  int T, K, P;
  bfmri_options opt;        /* per-request options; the server sets cuda_stream, sm_budget
                               and the allocator (stream-ordered, from the server's pool) */
  int n_sweeps;
  uint64_t first_counter;
  double* W_out;            /* K x N, may be NULL */
  double* alpha_out;        /* K, may be NULL */
} bfmri_request;

typedef struct {
  int status;               /* BFMRI_OK, an error code, or BFMRI_PENDING */
  int N;
  double submit_s, start_s, end_s;  /* host clock, seconds since the server was created */
  long long pcg_iterations;
  size_t device_bytes;      /* the admission estimate */
} bfmri_result;

/* Admission estimate of one request: every device allocation bfmri_create makes for a handle
 * of this shape (Y included, although the statistics step releases it), each rounded as the
 * library rounds it, plus a margin of 1/32 and 2 MiB for the pool's own rounding. 0 for
 * invalid sizes. A request with precond = BFMRI_PRECOND_MULTIGRID also builds the
 * multigrid hierarchy of its mask on its first solve; bfmri_server_submit adds those bytes
 * (from the mask) and 1/32 of them to this estimate, and reports the sum in
 * bfmri_result.device_bytes. */
size_t bfmri_request_device_bytes(int N, int T, int K, int P, int y_dtype, int precision);
/* High-water mark of the bytes in use from the server's memory pool
 * (cudaMemPoolAttrUsedMemHigh); reset != 0 restarts it from the current use. */
bfmri_status bfmri_server_pool_usage(bfmri_server* s, size_t* used_high, int reset);
bfmri_status bfmri_server_create(size_t budget_bytes, int max_slots, int sm_budget,
                                 bfmri_server** out);
/* Errors: INVALID_ARG, OOM (the request alone exceeds the budget). */
bfmri_status bfmri_server_submit(bfmri_server* s, const bfmri_request* req, long long* ticket);
/* BFMRI_OK with the result when the request has finished (the ticket is then released),
 * BFMRI_PENDING otherwise; wait != 0 blocks until it finishes. */
bfmri_status bfmri_server_poll(bfmri_server* s, long long ticket, int wait, bfmri_result* res);
/* Largest device-memory estimate and number of requests in flight at once so far. */
bfmri_status bfmri_server_stats(bfmri_server* s, size_t* peak_bytes, int* peak_running,
                                size_t* in_use);
/* Waits for every submitted request, then stops the workers. */
bfmri_status bfmri_server_destroy(bfmri_server* s);

/* ---------------------------------------------------------------------------------------
 * Allocation-free solve (the paper has no counterpart: this is an interface addition).
 *
 * For callers that cannot allocate device memory while they run: code that executes inside
 * another framework's memory pool or arena and may not call cudaMalloc behind its back, a
 * process that must not grow its device footprint after start-up, or a real-time loop where
 * an allocation (and the implicit device synchronisation of cudaMalloc / cudaFree) would
 * stall. bfmri_pcg_solve_static solves B~ x = b with the FP64 block-Jacobi PCG that
 * bfmri_sample_W runs under its default options (options.precond = BFMRI_PRECOND_BLOCK_JACOBI,
 * precision FP64; the reduced red-black and mixed-precision solvers are not offered here), on
 * device arrays the caller owns, and allocates nothing: its scratch (the
 * preconditioner factor, five work vectors, reduction and barrier words) lives in one
 * static device array of bfmri_pcg_static_capacity() bytes (32 MiB) that every GPU which
 * loads the library holds until the process exits.
 *
 *  N, D          voxels and unknowns per voxel (1 <= D <= 12)
 *  neighbourhood 4 or 6: how many of the six neighbour planes are used
 *  nbr           device, int32 [6][ld]: compact index of the -x,+x,-y,+y,-z,+z neighbour of
 *                each voxel, or -1
 *  ld            leading dimension of every [rows][ld] device array: >= N and a multiple
 *                of 32 (the other entry points use N rounded up to 32); anything else is
 *                rejected with BFMRI_ERR_INVALID_ARG
 *  blocks        device, FP64 [D(D+1)/2][ld]: per-voxel data block, packed lower triangle
 *                (entry (i, j), i >= j, in plane i(i+1)/2 + j)
 *  scale         device, FP64 [D]: prior scale per component (alpha or beta)
 *  b             device, FP64 [D][ld]: right-hand side
 *  x             device, FP64 [D][ld]: start value in, solution out (stop when
 *                ||b - B~ x|| <= delta ||b||, or after max_iter iterations)
 *  cuda_stream   stream for all work (NULL: legacy default stream); every call copies its
 *                status words into host memory and synchronises this stream before it
 *                returns
 *  info          may be NULL
 * Set-up: the first call on each device looks up the device address of the static array
 * (cudaGetSymbolAddress, with that device current) and caches it for later calls. Every call
 * reuses the same array and clears what must
 * start at zero, so calls that overlap on the GPU (other streams or threads, same device)
 * race and must be serialised by the caller. Problems whose scratch need
 * (bfmri_pcg_static_bytes(ld, D)) exceeds the capacity are rejected with
 * BFMRI_ERR_INVALID_ARG; errors are reported through bfmri_last_error(NULL). */
size_t bfmri_pcg_static_capacity(void);
size_t bfmri_pcg_static_bytes(size_t ld, int D);
bfmri_status bfmri_pcg_solve_static(int N, int D, int neighbourhood, const int* nbr, size_t ld,
                                    const double* blocks, const double* scale, const double* b,
                                    double* x, double delta, int max_iter, void* cuda_stream,
                                    bfmri_solve_info* info);

#ifdef __cplusplus
}
#endif

#endif /* BFMRI_H */
