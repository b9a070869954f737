/*
 * ecg.h -- C ABI of the GB300 (sm_103a) enlarged Conjugate Gradient library.
 *
 * Method: S. Moufawad, "Flexibly Enlarged Conjugate Gradient methods"
 * (arXiv 2305.19013).  The library solves A x = b for a sparse symmetric
 * positive definite A with the enlarged CG methods of its Sections 2-4:
 * SRE-CG2 (Algorithm 1), MSDO-CG (Algorithm 2), modified MSDO-CG
 * (Section 2.2), their truncated forms (Section 3; SRE-CG is SRE-CG2 with
 * trunc = 2) and the flexibly enlarged forms that halve the block width once
 * (Algorithms 3 and 4).  Every iteration runs on the GPU: the domain
 * splitting T^t(r) (eq. (Tt)), the product A W, CGS2 A-orthogonalisation
 * against the stored blocks, A-orthonormalisation (Pre-CholQR or A-CholQR)
 * with a t x t Cholesky factorisation in FP64, and the updates
 * x += W alpha, r -= A W alpha.  There is no CPU fallback: without a CUDA
 * device every call returns ECG_ECUDA.
 *
 * Conventions for every function below:
 *   - Blocks of w vectors of length n are row-major n x w arrays of double
 *     (entry (i, j) at [i*w + j]); small w x w matrices are row-major too.
 *   - Return value: ECG_OK (0) on success, ECG_ENOCONV (> 0) when the
 *     iteration limit was reached (the result is still valid), or a negative
 *     error code.  No C++ exception crosses this interface.
 *   - Thread safety: a context may be used by one host thread at a time.
 */
#ifndef ECG_H
#define ECG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ECG_OK 0
#define ECG_ENOCONV 1        /* k_max reached before the tolerance */
#define ECG_EINVAL (-1)      /* bad argument (sizes, partition, options) */
#define ECG_ENOMEM (-2)      /* a device or host allocation failed */
#define ECG_ECUDA (-3)       /* a CUDA runtime call failed, or no device */
#define ECG_EBREAKDOWN (-4)  /* a block became numerically rank deficient */
#define ECG_ENOTSPD (-5)     /* a diagonal entry of A is not positive */
#define ECG_ETIMEOUT (-6)    /* a bounded device-side wait ran out (batched solver) */

/* Generator of the new block at iteration k (Sections 2-3). */
#define ECG_SRE 0     /* SRE-CG2, Algorithm 1: W_k = A W_{k-1} */
#define ECG_MSDO 1    /* MSDO-CG, Algorithm 2: P_k = T(r_{k-1}) + P_{k-1} diag(beta_k) */
#define ECG_MODMSDO 2 /* modified MSDO-CG, Section 2.2: W_k = T(r_{k-1}) */

/* Arithmetic of the iteration. */
#define ECG_FP64 0  /* every step in FP64: the method as the paper states it */
#define ECG_MIXED 1 /* FP32 blocks, vectors and matrix values inside an FP64
                       iterative-refinement loop; t x t factorisations, alpha,
                       beta and the true residual stay FP64 (not in the paper) */

/* Self A-orthonormalisation of the block (Section 2.1, Section 5). */
#define ECG_PRE_CHOLQR 0 /* Euclidean CholQR, then A-CholQR (the paper's choice in Section 5) */
#define ECG_A_CHOLQR 1   /* A-CholQR alone */

/* Stopping rules (ecg_opts.stop_rule) */
#define ECG_STOP_R0 0 /* rho_k <= tol * ||b - A x_0||, the paper's test */
#define ECG_STOP_B 1  /* rho_k <= tol * ||b|| */

/* Preconditioner kinds (ecg_set_preconditioner) */
#define ECG_PREC_NONE 0  /* no preconditioner */
#define ECG_PREC_IC0 1   /* block Jacobi, IC(0) of every diagonal block */

typedef struct ecg_ctx ecg_ctx; /* opaque */

/* Sparse SPD matrix in CSR form, both triangles stored. */
typedef struct {
  int64_t n;             /* rows = columns */
  int64_t nnz;           /* stored entries, rowptr[n] */
  const int64_t* rowptr; /* n + 1 offsets, rowptr[0] = 0 */
  const int32_t* col;    /* nnz column indices in [0, n) */
  const double* val;     /* nnz values */
  int on_device;         /* 1: the three arrays are device pointers; 0: host */
} ecg_csr;

typedef struct {
  int variant;       /* ECG_SRE, ECG_MSDO or ECG_MODMSDO (default ECG_SRE) */
  int trunc;         /* 0: A-orthogonalise against every stored block (the
                        full method, trunc = k_max); >= 1: against the last
                        trunc blocks only (Section 3) */
  double switch_tol; /* > 0: flexible switch t -> t/2 once
                        |rho_k - rho_{k-1}| / rho_0 < switch_tol (Section 4.2);
                        requires even t.  0: never switch */
  int ortho;         /* ECG_PRE_CHOLQR (default) or ECG_A_CHOLQR */
  int check_every;   /* iterations issued between two host polls of the
                        device-side stop flag (default 16; >= 1) */
  int use_graph;     /* 1: replay a captured CUDA graph of check_every
                        iterations when the window size is fixed (default 1) */
  int precision;     /* ECG_FP64 (default) or ECG_MIXED */
  double inner_tol;  /* ECG_MIXED: relative residual reduction each FP32
                        inner solve aims for (default 1e-5; 0 = default).
                        An inner solve also ends after 400 iterations
                        without a 1% smaller residual (FP32 stalls near
                        its rounding times the conditioning); the FP64
                        refinement then starts the next one */
  int restart_every; /* Section 3, restarted methods: j >= 2 restarts at the
                        iterations k with k mod j == 1 (0: off) */
  double restart_tol;   /* > 0: restart when |rho_{k-1} - rho_{k-2}| / rho_c
                           < restart_tol, rho_c the residual norm at the
                           start of the current cycle (Section 3); 0: off */
  int restart_max;      /* restarts allowed by restart_tol (0: unlimited;
                           1: the "restarted once" runs of Tables 8, 9) */
  int restart_at_switch; /* 1: the flexible switch also restarts (the
                            restarted flexibly method, Tables 8, 9); needs
                            switch_tol > 0 */
  /* A restart discards the stored blocks and takes the next block from
     [T(r_{k-1})] with the width in force; x_{k-1} is kept and the stopping
     test keeps comparing with rho_0. */
  int stop_rule;        /* ECG_STOP_R0 (default): stop when rho_k <= tol rho_0
                           (Algorithm 1); ECG_STOP_B: when rho_k <= tol ||b||,
                           so that a good x_0 shortens the solve */
  int block_residual;   /* 1: the block-residual enlarged CG of Section 1:
                           R_0 = [T^t(r_0)], t x t coefficients
                           alpha_k = W_k^T R_{k-1}, R_k = R_{k-1} - V_k alpha_k,
                           x_k = x_0 + X_k 1 and rho_k = ||R_k 1||.  SRE-CG2
                           directions, FP64, no switch, restart or
                           preconditioner (ECG_EINVAL otherwise) */
  int tensor_cores;     /* 1 (default): the FP64 CGS products (W -= Q C,
                           C = V^T W) and the final transforms W R^{-1},
                           Y R^{-1} run on the tensor cores (exact digit
                           products, FP64 results) when the block width is 16
                           and the window has at most 32 columns; 2: also the
                           CGS coefficient Grams of the mixed method's FP32
                           inner solves; 0: CUDA-core FMAs throughout.  Not a
                           choice of the paper: all compute the same products
                           up to rounding */
  void* stream;      /* cudaStream_t for all work; NULL: a stream the
                        context creates */
} ecg_opts;

typedef struct {
  int iters;           /* iterations run (k - 1 at exit of the loop) */
  int switch_it;       /* last iteration with t vectors before the switch
                          (k_F of Section 4.1); 0 if no switch */
  int restarts;        /* restarts performed (#r of Tables 4, 5) */
  int status;          /* same value as the return code */
  int64_t mem_vectors; /* largest number of stored basis vectors, the "mem"
                          of the paper's Tables 4-9 */
  double relres;       /* rho_k / rho_0, recursively updated residual */
  double relres_true;  /* ||b - A x|| / ||b||, recomputed at exit */
  double device_ms;    /* device time of the solve (CUDA events) */
  const double* history; /* rho_0 .. rho_iters (iters + 1 values), host
                            memory owned by the context, valid until the
                            next ecg_solve or ecg_destroy */
} ecg_result;

/* Fill *opts with the defaults listed above. */
void ecg_default_opts(ecg_opts* opts);

/* Create a solver context for A with the subdomain map `partition` (n
 * entries, values in [0, t), every subdomain non-empty; the delta_i of
 * Section 1).  A and partition are copied (host or device pointers per
 * A->on_device); the caller may free them afterwards.  1 <= t <= 64.
 * Returns ECG_EINVAL for bad sizes, partition values, empty subdomains,
 * unsupported t, or switch_tol > 0 with odd t; ECG_ENOTSPD when a diagonal
 * entry is not positive; ECG_ENOMEM / ECG_ECUDA on device failures.  On
 * error *out is NULL. */
int ecg_create(const ecg_csr* A, const int32_t* partition, int t, const ecg_opts* opts,
               ecg_ctx** out);

/* Solve A x = b (Algorithms 1-4): stop when rho_k <= tol * rho_0 or when
 * k reaches maxit (the paper's k_max: at most maxit - 1 iterations run).
 * With ECG_MIXED, rho_k is the FP64 true residual b - A x_j after each
 * refinement step j, maxit bounds the inner iterations of all steps
 * together, and history holds the inner residual estimates scaled to the
 * outer residual, with the true residual at every refinement point.
 * b, x0 and x_out are n doubles each, all host or all device pointers (the
 * location is detected; host arrays are copied in and out inside the call).
 * x0 may be NULL (x0 = 0).  res may be NULL.  Returns ECG_OK,
 * ECG_ENOCONV (x_out holds the last iterate), ECG_EBREAKDOWN (x_out holds
 * the last iterate before the rank-deficient block), ECG_EINVAL, ECG_ENOMEM
 * (the stored blocks do not fit: use trunc) or ECG_ECUDA. */
int ecg_solve(ecg_ctx* ctx, const double* b, const double* x0, double* x_out, double tol,
              int maxit, ecg_result* res);

/* Block Jacobi preconditioning (Section 3 "Preconditioned versions",
 * Algorithm 5; the block Jacobi preconditioner of Section 5, eq. (cholprec)):
 * M = L L^T with L = diag(L_1, ..., L_nb), L_i the incomplete Cholesky factor
 * with zero fill (IC(0)) of the diagonal block A(I_i, I_i), I_i the rows
 * with pblock[i] == block (in increasing order).  Every later ecg_solve on
 * ctx runs the preconditioned method: the generated blocks become
 * L^{-T}[T(L^{-1} r)] = [T(M^{-1} r)] (splits), M^{-1} A W_{k-1} (SRE-CG2) and
 * [T(M^{-1} r)] + P_{k-1} diag(beta) with beta = -V_{k-1}^T M^{-1} r
 * (MSDO-CG), while alpha, x, r, the A-orthonormalisation and the stopping
 * test on ||r|| are unchanged.
 *   pblock: n int32 block ids in [0, nblocks), host or device pointer,
 *           copied; every block non-empty and inside one subdomain of the
 *           partition (so that the split commutes with M^{-1}).
 *   kind:   ECG_PREC_IC0, or ECG_PREC_NONE to remove the preconditioner
 *           (pblock and nblocks are then ignored).
 * The exact Cholesky factors of the paper's "Chol" variant are not offered:
 * their fill makes the substitutions sequential along each block.
 * Returns ECG_OK, ECG_EINVAL (bad ids, an empty block, a block across
 * subdomains, bad kind), ECG_ENOTSPD (an IC(0) pivot is not positive; the
 * context is left without a preconditioner), ECG_ENOMEM or ECG_ECUDA. */
int ecg_set_preconditioner(ecg_ctx* ctx, const int32_t* pblock, int nblocks, int kind);

/* sweeps damped Jacobi sweeps on A x = b in place, x <- x + omega D^{-1}
 * (b - A x), FP64 (b, x: n doubles, device pointers; 0 < omega < 2).  Not a
 * step of the paper's methods: it removes the high-frequency error of an
 * initial iterate proposed by the warm-start network (ecg_nn.h) before the
 * solve starts from it. */
int ecg_smooth(ecg_ctx* ctx, const double* b, double* x, int sweeps, double omega);

/* Release every resource of ctx (NULL is accepted). */
void ecg_destroy(ecg_ctx* ctx);

/* Static, human-readable text for a status code. */
const char* ecg_strerror(int code);

/* Per-kernel-class device timing.  ecg_profile_enable(ctx, 1) resets the
 * counters and, until disabled, brackets every kernel class of each
 * iteration with CUDA events on the context's stream (graph replay is off
 * while profiling).  ecg_profile_read fills the name, total milliseconds and
 * launch count of class `cls` and returns the number of classes (also when
 * cls is out of range, so cls = -1 queries the count). */
int ecg_profile_enable(ecg_ctx* ctx, int on);
int ecg_profile_read(ecg_ctx* ctx, int cls, const char** name, double* ms, long long* launches);

/* Measure this GPU's FP64 fused multiply-add rate: a kernel of 8 blocks
 * per SM x 256 threads, each running 8 independent FMA chains of `iters`
 * steps, timed with CUDA events after a warm-up launch, on the default
 * stream of the current device.  *tflops receives 2 x FMAs / seconds / 1e12.
 * The FP64 block kernels of the method are bound by this rate (not a step of
 * the paper's methods; the paper states no hardware).  Allocates and frees
 * a small device buffer.  Returns ECG_OK, ECG_EINVAL or ECG_ECUDA. */
int ecg_probe_fp64(int iters, double* tflops);

/* ----------------------------------------------------------------------
 * Step-level entry points.  Each runs one step of the iteration with the
 * same kernels ecg_solve uses, on the context's matrix, partition and
 * stream, and returns after the step has finished on the device.  All array
 * arguments are device pointers; arrays of block pointers are host arrays
 * holding device pointers.
 * ---------------------------------------------------------------------- */

/* W = [T^t(r)] (half = 0; W is n x t) or [T^{t/2}(r)] over the merged pairs
 * {2j, 2j+1} (half = 1; W is n x t/2): eq. (Tt) and Section 4. */
int ecg_op_split(ecg_ctx* ctx, const double* r, double* W, int half);

/* Y = A X for an n x w block, 1 <= w <= 64 (Algorithm 1 line 6). */
int ecg_op_spmm(ecg_ctx* ctx, const double* X, double* Y, int w);

/* out = M^{-1} in = L^{-T} L^{-1} in for an n x w block, 1 <= w <= 64, with
 * the preconditioner set by ecg_set_preconditioner (ECG_EINVAL without
 * one).  in and out must not overlap. */
int ecg_op_prec_apply(ecg_ctx* ctx, const double* in, double* out, int w);

/* C = [X_0 ... X_{m-1}]^T Y: the block inner products of Sections 2-3
 * (CGS coefficients (A Q)^T W, beta = V^T r, W^T r).  X_j is n x wx[j]
 * with 1 <= wx[j] <= 128, Y is n x wy with wy in {1,2,4,8,16,32,64}; C is
 * (sum wx) x wy.  1 <= m <= 1024. */
int ecg_op_tdot(ecg_ctx* ctx, int m, const double* const* X, const int* wx, const double* Y,
                int wy, double* C);

/* W -= [Q_0 ... Q_{m-1}] C: the CGS update of Sections 2.1 and 3 (each of
 * the two passes of CGS2 ends with it), for the n x w block W (updated in
 * place), m blocks Q_j of n x wq[j] (1 <= wq[j] <= 128, 1 <= m <= 1024)
 * and the (sum wq) x w row-major coefficients C (device memory).  With
 * tensor_cores on, w = 16 and sum wq <= 32 it runs the tensor-core form. */
int ecg_op_block_sub(ecg_ctx* ctx, int m, const double* const* Q, const int* wq, const double* C, double* W, int w);

/* Two passes of block classical Gram-Schmidt in the A-inner product of the
 * n x w block W against m A-orthonormal blocks Q_j (n x wq[j]) with
 * V_j = A Q_j: each pass computes C = V^T W, then W -= Q C (Section 2.1,
 * "CGS2").  W is updated in place. */
int ecg_op_cgs2(ecg_ctx* ctx, int m, const double* const* Q, const double* const* V,
                const int* wq, double* W, int w);

/* A-orthonormalise the n x w block W in place with the context's ortho mode
 * and write V = A W_k; W_k^T A W_k = I (Algorithm 1 lines 4 and 8).  Returns
 * ECG_EBREAKDOWN for a numerically dependent block. */
int ecg_op_a_orthonormalize(ecg_ctx* ctx, double* W, double* V, int w);

/* One update of Algorithm 1 lines 9-12 given a raw block W (n x w, already
 * A-orthogonal to the stored blocks): A-orthonormalise it (W and V = A W_k
 * written back), alpha = W_k^T r, x += W_k alpha, r -= V alpha, and
 * *rho = ||r||.  rho is a host pointer. */
int ecg_op_block_update(ecg_ctx* ctx, double* W, double* V, int w, double* x, double* r,
                        double* rho);

/* MSDO-CG generator (Algorithm 2 lines 6-7): P = [T(r)] + P_prev diag(beta),
 * beta = -V_prev^T r, with T = T^t when w == t and T^{t/2} when w == t/2. */
int ecg_op_msdo_generate(ecg_ctx* ctx, const double* r, const double* P_prev,
                         const double* V_prev, int w, double* P);

/* C = [X_0 ... X_{m-1}]^T Y like ecg_op_tdot, without a context and without
 * allocating any memory.  The paper has no counterpart to this call; it is
 * for callers that cannot allocate device memory when they need the
 * product: services that reserve the whole GPU for their own pool
 * allocator up front (so a library cudaMalloc would fail or fragment that
 * pool), and code on a latency-critical path that must not hit
 * cudaMalloc/cudaFree, which can block or synchronise the device.
 *
 * n rows (1 <= n < 2^31); 1 <= m <= 64 blocks X_j of n x wx[j] doubles,
 * 1 <= wx[j] <= 128 and sum wx <= 256; Y is n x wy with wy in
 * {1,2,4,8,16,32,64}; C is (sum wx) x wy.  X (a host array of device
 * pointers), Y and C: X_j, Y, C are device pointers on the current
 * device.  stream is a cudaStream_t (NULL: the default stream).  The call
 * waits for the stream and returns after C is written.  Sizes beyond these
 * limits return ECG_EINVAL.
 *
 * Memory: the partial sums (4 MiB), the launch state and the block list
 * live in static device arrays that every GPU loading this library holds
 * until the process exits.  The first call on each device looks up their
 * device addresses and raises the shared-memory limit of the kernels it
 * launches; make that first call before any stream capture.  All
 * calls on a device share the arrays, so calls that overlap on the GPU
 * (from two host threads or two streams at once) race and corrupt each
 * other's results: issue them one after another. */
int ecg_tdot_noalloc(int64_t n, int m, const double* const* X, const int* wx, const double* Y, int wy,
                     double* C, void* stream);


/* ----------------------------------------------------------------------
 * Batched solver.  Many independent systems A_s x_s = b_s of uneven size
 * are solved together by truncated SRE-CG2 (Algorithm 1 with the window of
 * Section 3: CGS2 against the last `trunc` blocks, then Pre-CholQR or
 * A-CholQR) in ONE persistent cooperative kernel per solve (FP64) or per
 * refinement round (mixed precision).  Each system gets a group of CTAs in
 * proportion to its rows; the groups iterate independently, synchronised
 * inside a group by bounded barriers.  The paper has no batched form: this
 * is the per-system method of Algorithm 1 run side by side, with iterates
 * equal (to rounding) to a separate solve of each system.  The matrices
 * are stored in SELL-C-sigma form with slice height C and sort window sigma
 * chosen by timing the product on the batch itself unless fixed in the
 * options.
 * ---------------------------------------------------------------------- */
typedef struct ecg_batch ecg_batch;

typedef struct {
  int trunc;           /* window blocks, 1..4 (default 2: SRE-CG) */
  int ortho;           /* ECG_PRE_CHOLQR (default) or ECG_A_CHOLQR */
  int precision;       /* ECG_MIXED (default: FP32 inner solves, FP64 refinement) or ECG_FP64 */
  double inner_tol;    /* mixed: lower bound of the inner relative tolerance (default 1e-5) */
  int slice_height;    /* SELL slice height C in {8, 16, 32}; 0: autotune (default) */
  int sort_window;     /* SELL sigma: rows sorted by length inside windows of sigma rows
                          (1: no sorting); 0: autotune (default) */
  int ctas_per_sm;     /* persistent CTAs per SM, 1..4 (0: as many as fit, at most 2) */
  double wait_limit_s; /* bound of every device-side barrier wait (default 1.0) */
  int debug_barrier_extra; /* testing only: > 0 makes every group barrier wait for that
                              many arrivals that never come, so the first wait runs
                              out after wait_limit_s and the solve returns
                              ECG_ETIMEOUT (default 0) */
  void* stream;        /* cudaStream_t; NULL: a stream the batch creates */
} ecg_batch_opts;

void ecg_batch_default_opts(ecg_batch_opts* opts);

/* Create a batch of nsys systems.  A[s] and partition[s] as in ecg_create
 * (host or device per A[s].on_device; copied).  All systems share t, which
 * must be 4 or 8.  nsys must not exceed the number of persistent CTAs
 * (ctas_per_sm x SMs).  Returns ECG_OK, ECG_EINVAL, ECG_ENOTSPD, ECG_ENOMEM
 * or ECG_ECUDA; on error *out is NULL. */
int ecg_batch_create(int nsys, const ecg_csr* A, const int32_t* const* partition, int t,
                     const ecg_batch_opts* opts, ecg_batch** out);

/* Solve every system: b[s], x0[s] (x0 may be NULL: all zero) and x_out[s]
 * are n_s doubles, all host or all device pointers.  tol and maxit as in
 * ecg_solve (FP64: rho_k <= tol rho_0 on the recursive residual; mixed:
 * ||b - A x|| <= tol ||b - A x_0|| on the FP64 residual after a refinement
 * round, maxit bounding the inner iterations of all rounds).  res (may be
 * NULL) receives nsys results; their history arrays belong to the batch and
 * stay valid until the next solve or destroy.  Returns ECG_OK when every
 * system converged, else the first non-OK status (ECG_ENOCONV,
 * ECG_EBREAKDOWN, ECG_ETIMEOUT), or ECG_EINVAL / ECG_ENOMEM / ECG_ECUDA. */
int ecg_batch_solve(ecg_batch* batch, const double* const* b, const double* const* x0, double* const* x_out,
                    double tol, int maxit, ecg_result* res);

/* The layout the batch runs with: SELL slice height and sort window, the
 * number of persistent CTAs, the autotuner's time of one product Y = A X
 * over the whole batch in ms (0 when the layout was fixed), and whether the
 * last solve replayed its rounds from a captured CUDA graph (1) or issued
 * them directly because the capture was refused (0).  Any output pointer
 * may be NULL. */
int ecg_batch_layout(const ecg_batch* batch, int* slice_height, int* sort_window, int* ctas,
                     double* spmm_ms, int* graph);

void ecg_batch_destroy(ecg_batch* batch);

#ifdef __cplusplus
}
#endif

#endif /* ECG_H */
