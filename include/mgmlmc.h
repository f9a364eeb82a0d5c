/*
 * mgmlmc.h -- C ABI of the GB300 MG-MLMC++ trace-estimation library.
 *
 * The library estimates tr(D^{-1}) for the 2D Schwinger Wilson-Dirac operator
 * with multigrid multilevel Monte Carlo and Hutch++ deflation of every level
 * difference (Frommer & Nasr Khalil, "MG-MLMC++ as a Variance Reduction Method
 * for Estimating the Trace of a Matrix Inverse", Lattice 2022).  Every step of
 * the computation runs in the library's own CUDA kernels (sm_103a).
 *
 * Conventions shared by all calls
 *   Status      every call returns an int: MGMLMC_OK (0) or a negative
 *               mgmlmc_status; mgmlmc_last_error(ctx) gives a message.
 *   Memory      vectors and gauge fields are DEVICE pointers owned by the
 *               caller unless a parameter says "host".  Objects created by the
 *               library (mgmlmc_ctx, mgmlmc_hier, mgmlmc_sketch) own their
 *               device memory and are released by their destroy call.
 *   Stream      all device work of a call is issued on the stream given to
 *               mgmlmc_ctx_create.  Calls that take decisions on the host
 *               (set-up, solves, sketches, estimates, anything that writes to
 *               a host pointer) synchronise that stream before returning;
 *               schwinger_apply, mg_apply, mg_restrict, mg_prolong, mg_vcycle
 *               and mgmlmc_rademacher are asynchronous.
 *   Complex     interleaved (re, im): complex128 for MGMLMC_FP64 and
 *               MGMLMC_MIXED, complex64 for MGMLMC_FP32.
 *   Gauge field U[t][x][mu] complex128, mu = 0 the x direction, mu = 1 the t
 *               direction, L x L sites, U_mu(x) = exp(i theta_mu(x)).
 *   Vectors     [rhs][site][dof] with site = t * L_l + x (x fastest) and
 *               dof 0..d_l-1 (d = 2 spins on the fine level, 2 * ntv on coarse
 *               levels; on coarse levels dof < ntv has chirality +1).
 *   Levels      0-based: level 0 is the fine operator D_1 of the paper,
 *               level nlev-1 the coarsest D_L.
 */
#ifndef MGMLMC_H
#define MGMLMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum mgmlmc_status {
  MGMLMC_OK = 0,
  MGMLMC_ERR_INVALID_ARG = -1,   /* bad size, null pointer, unsupported shape */
  MGMLMC_ERR_OOM = -2,           /* device allocation failed */
  MGMLMC_ERR_NOT_CONVERGED = -3, /* solver hit its iteration limit; results are the last iterate */
  MGMLMC_ERR_CUDA = -4,          /* a CUDA runtime call or kernel failed */
  MGMLMC_ERR_TIMEOUT = -5,       /* a bounded device wait ran out */
  MGMLMC_ERR_NAN = -6,           /* a norm or sample became NaN/Inf */
  MGMLMC_ERR_NOT_POSDEF = -7     /* CholeskyQR Gram matrix not positive definite (rank-deficient sketch) */
};

enum mgmlmc_prec {
  MGMLMC_FP64 = 0,   /* everything in FP64 */
  MGMLMC_FP32 = 1,   /* everything in FP32 */
  MGMLMC_MIXED = 2,  /* FP64 vectors and true residuals, FP32 inner Krylov + V-cycle */
  MGMLMC_TF32 = 3,   /* FP32 vectors, TF32 tensor-core products (mg_apply / mg_smooth on coarse levels of a
                        hierarchy set up with tensor_cores = 2) */
  MGMLMC_BF16 = 4,   /* FP32 vectors, BF16 tensor-core products with FP32 accumulation (same calls, a hierarchy
                        set up with tensor_cores = 1) */
  MGMLMC_FP16 = 5    /* FP32 vectors, FP16 tensor-core products with FP32 accumulation (same calls, a hierarchy
                        set up with tensor_cores = 3) */
};

enum mgmlmc_form {
  MGMLMC_ACCUMULATED = 0, /* fine-size Rademacher vectors restricted by Rhat_l (Algorithm 2 as printed) */
  MGMLMC_REDUCED = 1      /* level-size Rademacher vectors (eq. mlmc_dec_trace_reduced) */
};

enum mgmlmc_policy { MGMLMC_OPTIMAL = 0, MGMLMC_UNIFORM = 1 };

enum mgmlmc_noise { /* distribution of the random vectors (Section 1, eq. random_props; Section 2) */
  MGMLMC_NOISE_RADEMACHER = 0, /* real +-1 entries */
  MGMLMC_NOISE_Z4 = 1          /* entries 1, i, -1, -i: variance ||offdiag(A)||_F^2 instead of 1/2 ||offdiag(A+A^T)||_F^2 */
};

enum mgmlmc_weight { /* the matrix whose trace is estimated (Section 1: traces "after multiplication with gamma-matrices") */
  MGMLMC_TRACE_PLAIN = 0,  /* tr(D^{-1}) */
  MGMLMC_TRACE_GAMMA5 = 1  /* tr(gamma5 D^{-1}), gamma5 = sigma_3 (chirality sign; on coarse levels the sign of the
                              chirality block, which the aggregation preserves) */
};

enum mgmlmc_phase { /* streams of the counter-based Rademacher generator */
  MGMLMC_PHASE_STOCH = 0, MGMLMC_PHASE_SKETCH = 1, MGMLMC_PHASE_TESTVEC = 2, MGMLMC_PHASE_HUTCH = 3,
  MGMLMC_PHASE_DEFL = 4,   /* start block of the deflation subspace iteration */
  MGMLMC_PHASE_HARVEST = 5 /* right-hand sides of the learned preconditioner's training pairs */
};

#define MGMLMC_MAX_LEVELS 8

typedef struct mgmlmc_ctx mgmlmc_ctx;
typedef struct mgmlmc_hier mgmlmc_hier;
typedef struct mgmlmc_sketch mgmlmc_sketch;

/* ---- context ------------------------------------------------------------ */

/* Create a context bound to `cuda_stream` (a cudaStream_t, may be NULL for the
 * legacy default stream) on the current device.  *out receives the handle. */
int mgmlmc_ctx_create(void* cuda_stream, mgmlmc_ctx** out);
void mgmlmc_ctx_destroy(mgmlmc_ctx* ctx);
/* Message of the last failing call on this context ("" if none).  Owned by ctx. */
const char* mgmlmc_last_error(const mgmlmc_ctx* ctx);
/* Number of this library's kernel launches issued on ctx since creation. */
int64_t mgmlmc_launch_count(const mgmlmc_ctx* ctx);
int mgmlmc_version(void);
/* Kernel timer (measurement, not part of the paper's method): while on, every
 * launch of a kernel whose name contains `filter` (NULL or "" = all) is
 * bracketed by CUDA events on the context's stream together with its
 * algorithmic bytes and flops (counted over the right-hand sides still
 * iterating).  The report resolves the events and writes one line per kernel
 * "name\tlaunches\tms\tbytes\tflops\n" into buf (host, len bytes), then clears
 * the records. */
int mgmlmc_timing_enable(mgmlmc_ctx* ctx, int on, const char* filter);
int mgmlmc_timing_report(mgmlmc_ctx* ctx, char* buf, int64_t len);
/* Measured FMA throughput of the CUDA cores (fp64 != 0: FP64, else FP32) in TFLOP/s: eight independent FMA
 * chains per thread over a grid of 8 x 256-thread blocks per SM, best of three launches (CUDA events on the
 * context stream).  The roofline of ALU-bound kernels is taken against it. */
int mgmlmc_alu_peak(mgmlmc_ctx* ctx, int fp64, double* tflops);

/* ---- operator ----------------------------------------------------------- */

/* y = D x for the fine Schwinger Wilson-Dirac operator (Section 4; the
 * formula is the standard Wilson form with sigma_1, sigma_2 hops):
 *   (D x)(s) = (m0+2) x(s) - 1/2 sum_mu [(1-sigma_mu) U_mu(s) x(s+mu)
 *                                       + (1+sigma_mu) U_mu(s-mu)^* x(s-mu)]
 * periodic in x, antiperiodic in t.  U: device complex128 [L][L][2].
 * x, y: device, nrhs vectors of n = 2 L^2 complex, precision `prec`
 * (MGMLMC_MIXED reads as FP64).  L even, >= 4.  x and y must not alias. */
int schwinger_apply(mgmlmc_ctx* ctx, const double* U, int L, double m0,
                    const void* x, void* y, int nrhs, int prec);

/* Fill out[rhs][i] (device complex128, imaginary part 0) with the real
 * Rademacher stream (seed, level, phase, sample0 + rhs), i = 0..n-1 (the
 * isotropic vectors of eq. random_props).  Generator: SplitMix64 finaliser
 * mix64; key = mix64(seed ^ mix64(level<<56 | phase<<48 | sample));
 * word(i) = mix64(key + 0x9E3779B97F4A7C15 * (i+1)); sign = top bit. */
int mgmlmc_rademacher(mgmlmc_ctx* ctx, uint64_t seed, int level, int phase,
                      int64_t sample0, int64_t n, int nrhs, double* out);
/* Same streams with the distribution `kind` (mgmlmc_noise): MGMLMC_NOISE_RADEMACHER gives the vectors of
 * mgmlmc_rademacher, MGMLMC_NOISE_Z4 entry i = i^q with q = word(i) >> 62 (the top two bits). */
int mgmlmc_noise(mgmlmc_ctx* ctx, int kind, uint64_t seed, int level, int phase,
                 int64_t sample0, int64_t n, int nrhs, double* out);

/* ---- multigrid hierarchy (Section 3.1; set-up of Section 4) ------------- */

typedef struct {
  int levels;            /* number of levels, 0 = coarsen while side > 8 and side % (4 agg) == 0 */
  int agg;               /* aggregate side in sites (4) */
  int ntv;               /* test vectors per chirality (8): 2 ntv coarse dof per site */
  int sap_block_fine;    /* SAP block side on level 0 (4) */
  int sap_block_coarse;  /* SAP block side on coarse levels (2) */
  int setup_sweeps;      /* SAP sweeps for D v = 0 that smooth each test vector (4) */
  int pre_smooth;        /* V-cycle SAP sweeps before the coarse correction (1) */
  int post_smooth;       /* ... and after (1) */
  uint64_t seed;         /* test-vector stream seed (phase TESTVEC, level l, sample m) */
  int bootstrap;         /* bootstrap rounds after the initial set-up (0): each replaces the test
                            vectors of every level by bootstrap_its FGMRES iterations on D_l v_new = v
                            preconditioned by the current hierarchy, then rebuilds P_l and D_{l+1}
                            (the adaptive part of the DD-alpha-AMG set-up; with 0 the hierarchy is
                            the deterministic one the CPU oracle reproduces).  With bootstrap > 0 the
                            seed hierarchy and all rounds but the last only drive FP32 bootstrap
                            solves: their test-vector smoothing and SAP / coarsest inverses are
                            FP32; the last round builds the full FP64 hierarchy */
  int bootstrap_its;     /* (6) */
  int kcycle_its;        /* 0 = V-cycle; k > 0 = K-cycle: the coarse correction of levels below the
                            first runs k FGMRES iterations preconditioned by the next V/K-cycle (0) */
  double kcycle_tol;     /* relative residual at which a K-cycle stops early (0.1) */
  int tensor_cores;      /* inside the FP32 V-cycle, coarse levels with 16 dof per site run their SAP sweeps
                            and residuals as tcgen05 GEMMs over the rhs: 1 = BF16 operands (FP32 accumulation),
                            2 = TF32 operands, 3 = FP16 operands (11-bit significands like TF32 at the 16-bit
                            instruction rate), 0 = CUDA cores only */
  int graphs;            /* 1: the V-cycle preconditioner is captured once per shape as a CUDA graph
                            and replayed (not while the kernel timer runs or with K-cycles) (1) */
  int autotune;          /* 1: at the end of mg_setup, run mg_autotune for batches of 8..256 rhs unless the
                            process-wide tuning table already holds this hierarchy's shapes (0) */
} mg_params;

int mg_params_default(mg_params* p);

/* Build the aggregation hierarchy for D(U, m0): per level l < nlev-1 the ntv
 * complex Rademacher test vectors are smoothed by setup_sweeps SAP sweeps for
 * D_l v = 0, split by aggregate (agg x agg sites) and chirality, orthonormalised
 * (QR with real positive diagonal) into P_l; D_{l+1} = P_l^H D_l P_l
 * (Galerkin, Section 3) is stored as a 5-point block stencil; the coarsest
 * operator is inverted densely in FP64.  L must be a multiple of 16. */
int mg_setup(mgmlmc_ctx* ctx, const double* U, int L, double m0,
             const mg_params* params, mgmlmc_hier** out);
void mg_destroy(mgmlmc_hier* h);
int mg_num_levels(const mgmlmc_hier* h);
/* side, dof per site and n of level l (any pointer may be NULL). */
int mg_level_info(const mgmlmc_hier* h, int level, int* side, int* dof, int64_t* n);
/* tr(D_L^{-1}) of the coarsest level (= tau_L of Algorithm 2), host complex128. */
int mg_coarsest_trace(const mgmlmc_hier* h, double* tau_L);

/* y = D_l x on level l (vectors of n_l, precision prec).  With BF16 / FP16 (16-bit tensor-core images) the
 * library rounds x to a 16-bit workspace copy first where the 2x2-block stencil kernel is selected for this
 * level and batch (launch-shape table), so x itself is only read. */
int mg_apply(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, const void* x, void* y, int nrhs, int prec);
/* xc = P_l^H xf  (level l -> l+1). */
int mg_restrict(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, const void* xf, void* xc, int nrhs, int prec);
/* xf = P_l xc  (level l+1 -> l, overwrites xf). */
int mg_prolong(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, const void* xc, void* xf, int nrhs, int prec);
/* Copy P_l to host: complex128 [aggregate T*Lc+X][chirality 2][agg*agg*d_l/2][ntv];
 * row j of a block is local site (jt*agg+jx) times the dof of that chirality. */
int mg_get_prolongator(mgmlmc_ctx* ctx, const mgmlmc_hier* h, int level, double* host_out);
/* Copy the stencil of level l >= 1 to host: complex128 [site][dir 5][d][d],
 * dir = self, +x, -x, +t, -t; block (s, dir) = D_l[rows of s, cols of s+dir]. */
int mg_get_stencil(mgmlmc_ctx* ctx, const mgmlmc_hier* h, int level, double* host_out);

/* `sweeps` SAP sweeps for D_l x = f (the multigrid smoother): per sweep the
 * colour-0 blocks, then the colour-1 blocks, x_B += D_BB^{-1} (f - D_l x)_B
 * (block side sap_block_fine on level 0, sap_block_coarse above).  x is read
 * and updated in place.  prec FP64, FP32, or TF32 / BF16 / FP16 (tensor cores,
 * coarse levels with 16 dof and images of that format only; the 16-bit forms keep
 * a 16-bit workspace copy of x alongside the FP32 x for the 2x2-block kernels). */
int mg_smooth(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, const void* f, void* x, int nrhs, int prec, int sweeps);

/* Launch-shape autotuner (measurement of this machine, not part of the paper's method).  Several kernels have
 * launch variants that compute the same result: the tensor-core coarse stencil (variant bit 0: MMA tile of 128
 * rather than 64 right-hand sides, bits 1-3: pipeline-depth cap, bit 4: with BF16 / FP16 images, the kernel
 * that takes a 2x2 block of sites per item and shares the block's slabs across its sites, else one site per
 * item), the tensor-core SAP block update (pipeline depth) and the FP32 fine stencil (1, 2 or 4 right-hand
 * sides per thread).  The library keeps one process-wide table
 * (device, kernel, lattice side, batch bucket, weight format) -> variant, consulted by every launch (batch
 * bucket: the power of two >= nrhs in 8..256; keys without an entry take the default variant).  mg_autotune
 * times every variant of h's kernels (CUDA events, median of 5, on scratch vectors) for each of the `count`
 * batch sizes and records the fastest; force = 0 keeps entries already present.  Synchronous. */
int mg_autotune(mgmlmc_ctx* ctx, mgmlmc_hier* h, const int* nrhs_list, int count, int force);
/* The table as text, one line per entry "device kind side bucket format variant microseconds\n" (kind 0 = FP32
 * fine stencil, 1 = tensor-core stencil, 2 = tensor-core SAP block update); buf: host, len bytes. */
int mgmlmc_tune_report(char* buf, int64_t len);
/* Set one entry (for instance from a saved report) on the current device.  format: 0 TF32, 1 BF16, 2 FP16 images
 * (0 for the FP32 fine stencil); MGMLMC_ERR_INVALID_ARG for an unknown kind, a bucket that is not a power of two
 * in 8..256, a variant the kernel does not have (fine stencil: 1, 2 or 4; bit 4 only for the tensor-core stencil
 * with 16-bit images on a side divisible by 4). */
int mgmlmc_tune_set(int kind, int side, int bucket, int format, int variant);
/* Drop every entry of the current device: later launches take the default variants again. */
int mgmlmc_tune_clear(void);

/* MGMLMC_ERR_TIMEOUT if a tensor-core kernel of this hierarchy ran out of a
 * bounded wait (it then stopped early and freed its tensor memory), else OK. */
int mg_tc_status(mgmlmc_ctx* ctx, mgmlmc_hier* h);

/* In-place inverse of one dense n x n matrix on the device (the coarsest-level
 * direct solve of Section 3.1: tau_L of Algorithm 2 is the trace of D_L^{-1}):
 * Gauss-Jordan elimination with partial pivoting (largest |A_ik|, ties to the
 * smallest row) in one cooperative kernel whose CTAs meet at a grid barrier per
 * column.  A: device, row-major, complex128 (prec MGMLMC_FP64) or complex64
 * (MGMLMC_FP32), 1 <= n <= 8192 (the pivot row is staged in shared memory).
 * barrier_polls: poll limit of every barrier wait (0 = the default, about a
 * second); negative = self-test of the bounded wait: the barrier then waits for
 * one arrival more than the grid has, so every wait runs out after
 * -barrier_polls polls and the call returns MGMLMC_ERR_TIMEOUT with A left
 * partly eliminated (the kernel stops at the first expired wait; the device
 * stays usable).  Returns MGMLMC_ERR_NAN for a zero pivot (singular A). */
int mg_dense_inverse(mgmlmc_ctx* ctx, void* A, int n, int prec, int64_t barrier_polls);

/* One V-cycle from level l as an approximate solve x ~ D_l^{-1} b: SAP
 * pre-smoothing, coarse correction P_l V(l+1)(P_l^H r), SAP post-smoothing;
 * the coarsest level applies its dense inverse.  prec FP64 or FP32. */
int mg_vcycle(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, const void* b, void* x, int nrhs, int prec);

/* ---- batched solver ----------------------------------------------------- */

typedef struct {
  int m;             /* FGMRES restart length (16) */
  double tol;        /* stop at true relative residual ||b - D x|| / ||b|| <= tol, per rhs (1e-10) */
  int maxit;         /* total inner iteration limit per solve (2000) */
  int precond;       /* 1 = V-cycle preconditioner, 0 = none (GMRES), 2 = V-cycle + learned correction
                        on the fine level (FP32 inner solves; needs mg_attach_nn) */
  int prec;          /* mgmlmc_prec */
  double inner_tol;  /* MIXED: relative reduction of each FP32 inner solve (1e-5; FP32 arithmetic floors near 1e-6) */
} solve_params;

typedef struct {
  int iters;          /* inner iterations of the slowest rhs */
  int outer;          /* FP64 refinement / restart cycles */
  double max_relres;  /* largest true relative residual at return */
  int converged;      /* 1 if every rhs reached tol */
  int64_t total_iters;/* sum of inner iterations over rhs */
} solve_stats;

int solve_params_default(solve_params* p);

/* Solve D_l x = b for nrhs right-hand sides with flexible GMRES(m),
 * preconditioned by the V-cycle, each rhs stopping on its own true residual.
 * b, x: device, complex128 for FP64/MIXED, complex64 for FP32 (x is output,
 * its input value is ignored).  iters_out: host int[nrhs] or NULL. */
int fgmres_batched(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, const void* b, void* x,
                   int nrhs, const solve_params* sp, solve_stats* st, int* iters_out);

/* ---- MG-MLMC level differences (Section 3.1, Algorithm 2) -------------- */

/* Level difference l (0 <= l < nlev-1) applied to nrhs vectors; solves to sp->tol.
 *   form MGMLMC_REDUCED:      y = (D_l^{-1} - P_l D_{l+1}^{-1} P_l^H) zeta
 *                             (eq. mlmc_dec_trace_reduced), zeta and y level-size [nrhs][n_l];
 *   form MGMLMC_ACCUMULATED:  y = (Phat_l D_l^{-1} Rhat_l - Phat_{l+1} D_{l+1}^{-1} Rhat_{l+1}) zeta
 *                             (eq. mlmc_decomp_matrix), zeta and y fine-size [nrhs][n_0]; computed as
 *                             Phat_l A_l Rhat_l zeta with the reduced A_l (Rhat_l = Phat_l^H).
 * zeta, y: device complex128, must not alias. */
int mlmc_level_sample(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, int form, const double* zeta,
                      double* y, int nrhs, const solve_params* sp, solve_stats* st);

/* out = Rhat_l zeta = P_{l-1}^H ... P_0^H zeta (fine -> level l), FP64. */
int mg_restrict_to_level(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, const double* zeta_fine,
                         double* out, int nrhs);

/* ---- Hutch++ deflation (Sections 2.4 and 3.2) -------------------------- */

/* Deflation part of Algorithm 2 for level difference l: S = d Rademacher
 * vectors (phase SKETCH, samples 0..d-1, restricted by Rhat_l in the
 * accumulated form), k block power sweeps Y = A_l S, Q = qr(Y) (CholeskyQR2 in
 * FP64, R with real positive diagonal), S = Q; then the low-rank part
 * tau_lr = sum_i q_i^H A_l q_i.  Q is kept at level size (Q_fine = Phat_l Q).
 * 1 <= d <= 64, k >= 1.  tau_lr: host complex128.  *out owns Q (n_l x d, FP64). */
int hutchpp_sketch_qr(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, int d, int k, uint64_t seed,
                      int form, const solve_params* sp, mgmlmc_sketch** out, double* tau_lr);
void hutchpp_sketch_destroy(mgmlmc_sketch* s);
/* The QR step of the sketch (Algorithm 2, "Compute QR-factoriz. Y_l = Q_l K_l") in place on a caller's
 * basis: Y (device complex128 [d][n], vector i at Y + i n) becomes Q with Q^H Q = I by CholeskyQR2 (Gram
 * matrix G = Y^H Y in FP64, Cholesky G = R^H R with real positive diagonal, Y <- Y R^{-1}, done twice).
 * 1 <= d <= 64, n >= d.  Returns MGMLMC_ERR_NOT_POSDEF when a Gram matrix is not positive definite (Y of
 * rank < d); Y is then left partly transformed. */
int hutchpp_cholqr2(mgmlmc_ctx* ctx, double* Y, int d, int64_t n);
/* Copy Q to a device buffer complex128 [d][n_l]. */
int hutchpp_sketch_get_q(mgmlmc_ctx* ctx, const mgmlmc_sketch* s, double* q_dev, int* d, int64_t* n);

/* Projected samples of Algorithm 2: tau_r = z_r^H y_r with z_r = zeta_r - Q Q^H zeta_r,
 * computed as zeta^H y - (Q^H zeta)^H (Q^H y).  zeta, y: device complex128
 * [nrhs][n_l]; s may be NULL (no deflation: tau = zeta^H y).  tau_out: host
 * complex128 [nrhs]. */
int hutchpp_project(mgmlmc_ctx* ctx, const mgmlmc_sketch* s, const double* zeta, const double* y,
                    int64_t n, int nrhs, double* tau_out);

/* Same projected samples as hutchpp_project, for callers that cannot allocate
 * device memory when they need them: a host framework that has reserved the
 * whole GPU for its own caching allocator, or a latency-critical loop that
 * forbids cudaMalloc/cudaFree (they synchronise the device) after start-up.
 * The paper has no counterpart; this is a deployment variant of the call above.
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library routine, and
 * no context is needed.  Partial sums go to a fixed file-scope device array of
 * about 4.3 MB that every GPU loading the library holds until exit; the first
 * call on a device (with that device current) looks up the array's device
 * address once per CUDA context, so make that first call before any stream
 * capture (and again first after a cudaDeviceReset).  Every call
 * overwrites the slots it later reads (no state carries over), but all calls
 * share the one array: calls that overlap on the GPU (other streams, other host
 * threads) race and give wrong results.
 *   stream   cudaStream_t for the two launches (asynchronous; NULL = legacy default)
 *   Q        device complex128 [d][n] (may be NULL when d == 0), d <= 32
 *   zeta, y  device complex128 [nrhs][n], nrhs <= 256
 *   tau_out  DEVICE complex128 [nrhs]: tau_r = zeta_r^H y_r - (Q^H zeta_r)^H (Q^H y_r)
 * Returns MGMLMC_ERR_INVALID_ARG for nrhs > 256, d > 32, negative sizes or null
 * pointers (nothing is launched), MGMLMC_ERR_CUDA if the address lookup or a
 * launch fails (an error left pending by earlier work on the calling thread is
 * picked up and reported here too), MGMLMC_OK otherwise (nrhs == 0 is a no-op).
 * The pointers themselves cannot be checked: shapes and devices are the
 * caller's responsibility (the Python binding checks them). */
int hutchpp_project_noalloc(void* stream, const double* Q, int d, const double* zeta, const double* y,
                            int64_t n, int nrhs, double* tau_out);

/* ---- learned preconditioner (library extension; the paper has no learned part) ---- */

/* A gauge-covariant convolutional network M ~ D^{-1} used as a correction after
 * the V-cycle inside FGMRES (solve_params.precond = 2):  z = V(v);  t = v - D z;
 * z += |t| M(t / |t|)  (the net sees unit-norm residuals, so train it on pairs
 * (r / |r|, e / |r|)).
 * Layer l:  z_k(x) = sum_d sum_c W[d][k][c] T_d(x) a_c(x + d)  over the 9 offsets
 * d = 3 (dt+1) + (dx+1) of the 3x3 neighbourhood, T_d(x) the parallel transporter
 * from x + d to x (links with the antiperiodic sign on time-boundary crossings,
 * diagonals the average of the two L-shaped paths); hidden layers apply
 * z max(0, |z| + b_k)/|z|, the last is linear.  Channels 2 -> C -> ... -> 2;
 * weights complex, used rounded to bfloat16, FP32 accumulation and FP32 master
 * weights; loss (1/nrhs) sum ||M(r) - e||^2 / ||e||^2 on (residual, error) pairs.
 * Flat parameter layout (floats): per layer W (9 * c_out * c_in complex,
 * index (d * c_out + k) * c_in + c, re/im interleaved), then b (c_out) for
 * hidden layers.  Fields: device complex64 [nrhs][site][2]. */
typedef struct mgmlmc_nn mgmlmc_nn;
int nn_create(mgmlmc_ctx* ctx, const double* U, int L, int layers, int channels, uint64_t seed, mgmlmc_nn** out);
void nn_destroy(mgmlmc_nn* nn);
int64_t nn_num_params(const mgmlmc_nn* nn);
int nn_set_params(mgmlmc_ctx* ctx, mgmlmc_nn* nn, const float* host_params);
int nn_get_params(mgmlmc_ctx* ctx, const mgmlmc_nn* nn, float* host_params);
int nn_forward(mgmlmc_ctx* ctx, mgmlmc_nn* nn, const void* r, void* y, int nrhs);
/* loss, and (host_grad != NULL) its gradient w.r.t. the bf16-rounded weights and the biases, flat layout */
int nn_loss_grad(mgmlmc_ctx* ctx, mgmlmc_nn* nn, const void* r, const void* e, int nrhs, double* loss,
                 float* host_grad);
/* one Adam step (beta 0.9 / 0.999, eps 1e-8) on the loss of (r, e); *loss = loss before the step */
int nn_train_step(mgmlmc_ctx* ctx, mgmlmc_nn* nn, const void* r, const void* e, int nrhs, double lr, double* loss);
/* use nn in the fine-level preconditioner of h (precond = 2); NULL detaches. nn must outlive the attachment. */
int mg_attach_nn(mgmlmc_ctx* ctx, mgmlmc_hier* h, mgmlmc_nn* nn);
/* Number format of the layers.  0: FP32 CUDA-core kernels (layer inputs FP32).  1 (the default where L is a
 * multiple of 16): tcgen05 tensor-core kernels with BF16 operands and FP32 accumulation: every layer input
 * (the residual included) is rounded to bfloat16, the channel mixing of each of the 9 offsets is one MMA whose
 * FP32 result is multiplied by the transporter in the epilogue (T_d(x) is a scalar per site and offset, so it
 * commutes with the mixing); in the backward pass the pre-activation gradients and, for the weight gradient,
 * the transported inputs T_d a are rounded to bfloat16 as well.  Returns MGMLMC_ERR_INVALID_ARG for format 1
 * on other lattices.  A tensor-core layer whose bounded wait expires makes nn_forward / nn_loss_grad /
 * nn_train_step return MGMLMC_ERR_TIMEOUT (inside FGMRES the hierarchy's tensor-core status reports it). */
int nn_set_format(mgmlmc_ctx* ctx, mgmlmc_nn* nn, int format);
int nn_get_format(const mgmlmc_nn* nn);
/* Rebinds nn to another gauge field U (device complex128 [L][L][2], any even L >= 4; a multiple of 16 in
 * format 1): the transporters are recomputed, the weights and the Adam state kept, so one network trains on
 * pairs from several lattices and serves any of them (the layers are local and gauge covariant).  Detach it
 * from hierarchies of the old lattice first. */
int nn_set_field(mgmlmc_ctx* ctx, mgmlmc_nn* nn, const double* U, int L);
/* Training pairs from the method's own fine-level solves (the learned correction's data): for the Rademacher
 * right-hand sides zeta_s of stream (seed, level 0, MGMLMC_PHASE_HARVEST, s), s = sample0 .. sample0+count-1,
 * with v = V(zeta) one FP32 V-cycle of h, r = zeta - D v and x = D^{-1} zeta by FP32 FGMRES (V-cycle
 * preconditioned) to relative residual tol:
 *   R[s] = r / ||r||,   E[s] = (x - v) / ||r||     (so D E = R up to the solver tolerance).
 * R, E: device complex64 [count][n_0], caller-owned; the call blocks until they are written.  Errors:
 * MGMLMC_ERR_INVALID_ARG (null / aliased pointers, count < 0, tol outside (0, 1)), MGMLMC_ERR_NOT_CONVERGED is
 * not raised (a solve that stops at the iteration limit still yields a pair), CUDA errors as elsewhere. */
int nn_harvest_pairs(mgmlmc_ctx* ctx, mgmlmc_hier* h, uint64_t seed, int64_t sample0, int count, double tol,
                     void* R, void* E);

/* ---- Algorithm 2 end to end --------------------------------------------- */

typedef struct {
  double eps;                       /* target relative 1-sigma accuracy */
  int d[MGMLMC_MAX_LEVELS];         /* deflation vectors per level difference, 0..64 (0 = plain MG-MLMC) */
  int k;                            /* block power sweeps (2) */
  int nrhs_max;                     /* largest batch of samples per level (256) */
  int nrhs_first;                   /* first batch per level (32) */
  int policy;                       /* mgmlmc_policy */
  int form;                         /* mgmlmc_form */
  uint64_t seed;
  double cost[MGMLMC_MAX_LEVELS];   /* C_l per sample (cost_mode 0) */
  int cost_mode;                    /* 0 = cost[], 1 = counted flops of each sample's solves */
  int min_samples;                  /* >= 2 */
  int64_t max_samples;              /* per level */
  solve_params solve;
  double* sample_out[MGMLMC_MAX_LEVELS]; /* optional host buffers, complex128 [sample_cap] */
  int64_t sample_cap;
  int noise;                        /* mgmlmc_noise of the sketch and stochastic vectors (Rademacher) */
  int weight;                       /* mgmlmc_weight: tr(D^{-1}) or tr(gamma5 D^{-1}) (plain) */
} est_params;

typedef struct {
  double tau[2];                    /* estimate of tr(D^{-1}) = sum_l (tau_l + tau_l^lr) + tau_L */
  double sigma;                     /* sqrt(sum_l V_l / N_l) */
  double tau_L[2];
  int nlev;
  int64_t N[MGMLMC_MAX_LEVELS];     /* samples used per level difference */
  int64_t computed[MGMLMC_MAX_LEVELS]; /* samples computed (>= N; batches overshoot) */
  double mean[MGMLMC_MAX_LEVELS][2];
  double V[MGMLMC_MAX_LEVELS];
  double C[MGMLMC_MAX_LEVELS];
  double tau_lr[MGMLMC_MAX_LEVELS][2];
  int64_t solves;                   /* linear solves (right-hand sides) issued */
  int64_t inner_iters;              /* total inner Krylov iterations */
  int steps;                        /* s at which Algorithm 2 stopped */
  double flops;                     /* counted operator flops of all solves (sketches included): sum over
                                       solves of (inner iterations + 1) x the nnz flops of the level's operator
                                       (8 flops per complex non-zero), the cost model of Section 4 */
} est_result;

int est_params_default(est_params* p);

/* MG-MLMC++ (Algorithm 2): per level difference the Hutch++ sketch (d_l, k),
 * tau_L from the coarsest dense inverse, then the stochastic loop.  Samples
 * are computed in batches on the GPU; the host replays Algorithm 2 sample by
 * sample (s = 1, 2, ...) on them, so the stopping decisions are those of the
 * per-sample algorithm and extra batch samples are discarded. */
int trace_estimate(mgmlmc_ctx* ctx, mgmlmc_hier* h, const est_params* p, est_result* r);

/* ---- plain Hutchinson (Algorithm 1) ------------------------------------- */

typedef struct {
  double eps;          /* target relative 1-sigma accuracy */
  int nrhs_first;      /* first batch of samples (32) */
  int nrhs_max;        /* largest batch (256) */
  uint64_t seed;       /* sample s uses the stream (seed, level 0, MGMLMC_PHASE_HUTCH, s) */
  int noise;           /* mgmlmc_noise */
  int weight;          /* mgmlmc_weight */
  int min_samples;     /* >= 2 */
  int64_t max_samples;
  solve_params solve;  /* solves on level 0 (e.g. precond = 0, m = 30: unpreconditioned GMRES(30)) */
  double* sample_out;  /* optional host buffer, complex128 [sample_cap] */
  int64_t sample_cap;
  const mgmlmc_sketch* deflate; /* NULL, or a deflation basis from deflation_basis: the samples become
                                   zeta^H (I - V V^H) D^{-1} zeta and the basis's direct part is added */
} hutch_params;

typedef struct {
  double tau[2];       /* estimate of tr(D^{-1}) (or tr(gamma5 D^{-1})) */
  double sigma;        /* sqrt(V / s) */
  int64_t N;           /* samples used (s at the stop) */
  int64_t computed;    /* samples computed (>= N) */
  int64_t solves;
  int64_t inner_iters;
  double tau_defl[2];  /* the deflation basis's direct part tr(V^H D^{-1} V) (0 without deflation) */
} hutch_result;

int hutch_params_default(hutch_params* p);

/* Algorithm 1 on the fine operator of h: tau_s = zeta_s^H D^{-1} zeta_s (or zeta_s^H gamma5 D^{-1} zeta_s),
 * stop once V/s <= (eps |tau|)^2.  Samples are solved in batches; the host replays the per-sample stop, so
 * N is that of the per-sample algorithm and surplus samples are discarded. */
int hutchinson_estimate(mgmlmc_ctx* ctx, mgmlmc_hier* h, const hutch_params* p, hutch_result* r);

/* Deflation basis of the exactly deflated Hutchinson estimator (Section 2, "Exact Deflation"; the paper's
 * comparator in Section 4): the right singular vectors of the fine operator D with the k smallest singular
 * values, i.e. the eigenvectors of the Hermitian gamma5 D with the smallest |mu|, approximated by `sweeps`
 * steps of the block power method on D^{-1} gamma5 (V <- CholeskyQR2(D^{-1} gamma5 V), k Rademacher start
 * vectors from the stream (seed, level 0, phase 4, samples 0..k-1)), solves with sp.  *out owns V (fine size,
 * [k][n_0]); tau_defl (host complex128) = tr(V^H D^{-1} V) = tr(Pi D^{-1}) for Pi = V V^H (k more solves; exact
 * for any orthonormal V, so the deflated estimator is unbiased however far the iteration converged);
 * residual (host, may be NULL) = ||Y - V V^H Y||_F / ||Y||_F for Y = D^{-1} gamma5 V (0 for an invariant
 * subspace).  1 <= k <= 64.  Use the basis with hutchinson_estimate (hutch_params.deflate). */
int deflation_basis(mgmlmc_ctx* ctx, mgmlmc_hier* h, int k, int sweeps, uint64_t seed, const solve_params* sp,
                    mgmlmc_sketch** out, double* tau_defl, double* residual);

/* The target-accuracy update of Algorithm 2 for one step (host only, no GPU):
 * active[l] (in/out, 0/1) becomes 0 when V[l]/N[l] <= rho_l^2 with
 * rho_l^2 = sqrt(C_l V_l)/sum_j sqrt(C_j V_j) (eps |tau|)^2 (optimal) or
 * (eps |tau|)^2/nd (uniform); nothing changes while some N[j] < 2. */
int mlmc_update_active(int nd, int* active, const double* V, const int64_t* N, const double* C,
                       double eps, double tau_abs, int policy, int min_samples);

#ifdef __cplusplus
}
#endif
#endif /* MGMLMC_H */
