/*
 * ecg_oracle.c -- plain, slow, double-precision CPU oracle for the enlarged
 * Conjugate Gradient methods of S. Moufawad, "Flexibly Enlarged Conjugate
 * Gradient methods" (arXiv 2305.19013).
 *
 * TEST INFRASTRUCTURE.  This file exists to check the CUDA solver.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark load
 * it.  It shares no code, header, table or helper with the CUDA path; it
 * uses no BLAS and runs every loop in its obvious order.  It is compiled
 * with -ffp-contract=off so that x86 and Arm builds round identically.
 *
 * Threads.  The same source is built twice: plain (one thread) and with
 * -fopenmp, where loops whose iterations are independent (rows of a block,
 * diagonal blocks of the preconditioner, chunks of a sum) are shared out
 * among threads.  Every sum over rows is taken in fixed chunks of OR_CHUNK
 * consecutive rows: each chunk is summed over its rows in increasing order
 * and the chunk sums are then added in chunk order.  The order does not
 * depend on the number of threads, so both builds return the same bits.
 *
 * Conventions.  A block of w vectors of length n is a row-major n x w array
 * (entry (i, j) at [i*w + j]).  Small w x w matrices are row-major too.
 *
 * Readings of the paper taken here where it is silent or garbled (each is
 * repeated at the function that uses it):
 *   - CGS2 ("Algorithm 18" of the author's thesis, not reproduced in the
 *     paper, Section 2.1 and Section 5): block classical Gram-Schmidt in the
 *     A-inner product, two full passes, with C = (A Q)^T W read off the
 *     stored A Q blocks.
 *   - Pre-CholQR (Section 5; the paper cites it without its body): a
 *     Householder QR of the block, signs fixed so that diag(R) > 0, followed
 *     by A-CholQR of the orthonormal factor.  A-CholQR alone is the other
 *     option Section 2.1 names and is kept as a mode.
 *   - Breakdown (not discussed in the paper): a Cholesky pivot that is not
 *     larger than 1e-14 times the diagonal entry it started from, or is not
 *     finite, stops the solve with status BREAKDOWN and the current iterate.
 *   - The switch test uses |rho_k - rho_{k-1}| / rho_0 (Section 4.2 and the
 *     restart test of Section 3 write the absolute value; Algorithms 3 and 4
 *     drop it, which would trigger the switch at the first decrease).
 *   - Halving pairs 0-based subdomains {2j, 2j+1} into subdomain j
 *     (Section 4, the merged sets delta~_i = delta_{2i-1} U delta_{2i}).
 *   - The loop runs while rho_{k-1} > eps*rho_0 and k < k_max (Algorithm 1),
 *     so at most k_max - 1 iterations; "iters" is the number of loop bodies.
 *   - switch_it is the last iteration that used t vectors (k_F of
 *     Section 4.1), so that mem = t*switch_it + (t/2)*(iters - switch_it)
 *     as in Tables 6-9.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ENOCONV 1
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_EBREAKDOWN (-4)
#define OR_ENOTSPD (-5)

#define OR_BREAKDOWN_RATIO 1e-14

#ifdef _OPENMP
#include <omp.h>
#define OR_PAR_FOR _Pragma("omp parallel for schedule(static)")
#else
#define OR_PAR_FOR
#endif

/* rows per chunk of every sum over rows (see "Threads" above) */
#define OR_CHUNK 4096

/* Threads of the OpenMP build (no effect in the plain build); n < 1 keeps
 * the current setting.  Returns the number of threads in use. */
int or_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------ row sums */

/* out[q] = sum over rows i of chunk c that lie in [i0, n) of
 * A[i*lda + ja] * B[i*ldb + c0 + q], q < nc, rows in increasing order. */
static void or_chunk_dot(int64_t c, int64_t i0, int64_t n, const double* A, int64_t lda, int ja,
                         const double* B, int64_t ldb, int c0, int nc, double* out) {
  int64_t lo = c * OR_CHUNK, hi = lo + OR_CHUNK;
  if (lo < i0) lo = i0;
  if (hi > n) hi = n;
  for (int q = 0; q < nc; q++) out[q] = 0.0;
  for (int64_t i = lo; i < hi; i++) {
    const double a = A[i * lda + ja];
    for (int q = 0; q < nc; q++) out[q] += a * B[i * ldb + c0 + q];
  }
}

/* d[q] = sum_{i0 <= i < n} A[i*lda + ja] * B[i*ldb + c0 + q] for q < nc
 * (nc <= 64): a column of A against nc columns of B, summed chunk by chunk
 * (OR_CHUNK rows) and the chunk sums added in chunk order. */
static void or_col_dots(int64_t i0, int64_t n, const double* A, int64_t lda, int ja, const double* B,
                        int64_t ldb, int c0, int nc, double* d) {
  for (int q = 0; q < nc; q++) d[q] = 0.0;
  if (i0 >= n) return;
  const int64_t cf = i0 / OR_CHUNK, nch = (n + OR_CHUNK - 1) / OR_CHUNK - cf;
  double* part = (double*)malloc(sizeof(double) * (size_t)(nch * nc));
  if (part) {
    OR_PAR_FOR
    for (int64_t c = 0; c < nch; c++) or_chunk_dot(cf + c, i0, n, A, lda, ja, B, ldb, c0, nc, part + c * nc);
    for (int64_t c = 0; c < nch; c++)
      for (int q = 0; q < nc; q++) d[q] += part[c * nc + q];
    free(part);
  } else { /* same sums, one chunk at a time */
    double tmp[nc];
    for (int64_t c = 0; c < nch; c++) {
      or_chunk_dot(cf + c, i0, n, A, lda, ja, B, ldb, c0, nc, tmp);
      for (int q = 0; q < nc; q++) d[q] += tmp[q];
    }
  }
}

/* dst[0 .. count) = src[0 .. count) */
static void or_copy(int64_t count, double* dst, const double* src) {
  OR_PAR_FOR
  for (int64_t i = 0; i < count; i++) dst[i] = src[i];
}

/* sum_i u[i] v[i] over [0, n), chunk by chunk */
static double or_dot(int64_t n, const double* u, const double* v) {
  double s;
  or_col_dots(0, n, u, 1, 0, v, 1, 0, 1, &s);
  return s;
}

/* ---------------------------------------------------------------- products */

/* y = A x for A in CSR (Algorithm 1 line 1: r0 = b - A x0). */
void or_spmv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
             const double* x, double* y) {
  OR_PAR_FOR
  for (int64_t i = 0; i < n; i++) {
    double s = 0.0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) s += val[p] * x[col[p]];
    y[i] = s;
  }
}

/* Y = A X for an n x w block X (the product A W_{k-1} of Algorithm 1 line 6
 * and V_k = A P_k of Algorithm 2 line 9). */
void or_spmm(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, int w,
             const double* X, double* Y) {
  OR_PAR_FOR
  for (int64_t i = 0; i < n; i++) {
    for (int c = 0; c < w; c++) {
      double s = 0.0;
      for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) s += val[p] * X[(int64_t)col[p] * w + c];
      Y[i * w + c] = s;
    }
  }
}

/* W = [T^t(r)]: column j holds r restricted to subdomain delta_j, zero
 * elsewhere (Section 1, eq. (Tt)). */
void or_split(int64_t n, const int32_t* part, int t, const double* r, double* W) {
  OR_PAR_FOR
  for (int64_t i = 0; i < n; i++) {
    for (int j = 0; j < t; j++) W[i * t + j] = 0.0;
    W[i * t + part[i]] = r[i];
  }
}

/* W = [T^{t/2}(r)] over the merged subdomains {2j, 2j+1} (Section 4,
 * eq. (Tt)); W is n x t/2. */
void or_split_half(int64_t n, const int32_t* part, int t, const double* r, double* W) {
  int h = t / 2;
  OR_PAR_FOR
  for (int64_t i = 0; i < n; i++) {
    for (int j = 0; j < h; j++) W[i * h + j] = 0.0;
    W[i * h + part[i] / 2] = r[i];
  }
}

/* C = X^T Y (wx x wy) for n x wx X and n x wy Y: the block inner products
 * W^T r, P^T A P and (AQ)^T W of Sections 2-4. */
static void or_tdot_chunk(int64_t c, int64_t n, int wx, const double* X, int wy, const double* Y, double* P) {
  const int64_t lo = c * OR_CHUNK, hi = (lo + OR_CHUNK < n) ? lo + OR_CHUNK : n;
  for (int a = 0; a < wx * wy; a++) P[a] = 0.0;
  for (int64_t i = lo; i < hi; i++)
    for (int a = 0; a < wx; a++) {
      const double xa = X[i * wx + a];
      for (int b = 0; b < wy; b++) P[a * wy + b] += xa * Y[i * wy + b];
    }
}

void or_block_tdot(int64_t n, int wx, const double* X, int wy, const double* Y, double* C) {
  /* Entry (a, b) sums its products over the rows of each chunk of OR_CHUNK
   * rows in increasing order; the chunk sums are added in chunk order. */
  const int64_t nch = (n + OR_CHUNK - 1) / OR_CHUNK;
  const int e = wx * wy;
  for (int a = 0; a < e; a++) C[a] = 0.0;
  double* part = (double*)malloc(sizeof(double) * (size_t)(nch * e));
  if (part) {
    OR_PAR_FOR
    for (int64_t c = 0; c < nch; c++) or_tdot_chunk(c, n, wx, X, wy, Y, part + c * e);
    for (int64_t c = 0; c < nch; c++)
      for (int a = 0; a < e; a++) C[a] += part[c * e + a];
    free(part);
    return;
  }
  double* tmp = (double*)malloc(sizeof(double) * (size_t)e); /* same sums, one chunk at a time */
  if (!tmp) {
    for (int a = 0; a < e; a++) C[a] = NAN;
    return;
  }
  for (int64_t c = 0; c < nch; c++) {
    or_tdot_chunk(c, n, wx, X, wy, Y, tmp);
    for (int a = 0; a < e; a++) C[a] += tmp[a];
  }
  free(tmp);
}

/* W -= Q C for n x wq Q, wq x w C and n x w W (the CGS update). */
void or_block_sub(int64_t n, int wq, const double* Q, int w, const double* C, double* W) {
  OR_PAR_FOR
  for (int64_t i = 0; i < n; i++)
    for (int b = 0; b < w; b++) {
      double s = 0.0;
      for (int a = 0; a < wq; a++) s += Q[i * wq + a] * C[a * w + b];
      W[i * w + b] -= s;
    }
}

/* X <- X R^{-1} for upper-triangular R, one row at a time. */
void or_right_trsm(int64_t n, int w, const double* R, double* X) {
  OR_PAR_FOR
  for (int64_t i = 0; i < n; i++) {
    double* x = X + i * w;
    for (int j = 0; j < w; j++) {
      double s = x[j];
      for (int a = 0; a < j; a++) s -= x[a] * R[a * w + j];
      x[j] = s / R[j * w + j];
    }
  }
}

/* -------------------------------------------------------------- small dense */

/* Cholesky G = R^T R, R upper triangular with positive diagonal; only the
 * upper triangle of G is read.  Returns 0, or j+1 when pivot j fails the
 * breakdown test (pivot <= 1e-14 * G_jj, or not finite). */
int or_cholesky(int w, const double* G, double* R) {
  for (int i = 0; i < w * w; i++) R[i] = 0.0;
  for (int j = 0; j < w; j++) {
    double d = G[j * w + j];
    for (int k = 0; k < j; k++) d -= R[k * w + j] * R[k * w + j];
    if (!(d > OR_BREAKDOWN_RATIO * G[j * w + j]) || !isfinite(d)) return j + 1;
    double rjj = sqrt(d);
    R[j * w + j] = rjj;
    for (int i = j + 1; i < w; i++) {
      double s = G[j * w + i];
      for (int k = 0; k < j; k++) s -= R[k * w + j] * R[k * w + i];
      R[j * w + i] = s / rjj;
    }
  }
  return 0;
}

/* Thin Householder QR of the n x w block W (n >= w): W = Q R with Q n x w,
 * Q^T Q = I, R upper triangular with nonnegative diagonal.  Returns 0, or
 * j+1 when column j is numerically dependent on the columns before it
 * (R_jj^2 <= 1e-14 ||w_j||^2), mirroring the Cholesky test. */
int or_householder_qr(int64_t n, int w, const double* W, double* Q, double* R) {
  double* Wc = (double*)malloc(sizeof(double) * (size_t)(n * w));
  double* Vh = (double*)malloc(sizeof(double) * (size_t)(n * w)); /* Householder vectors, v_j at Vh + j n */
  double* beta = (double*)malloc(sizeof(double) * (size_t)w);
  double* cn2 = (double*)malloc(sizeof(double) * (size_t)w);
  double* d = (double*)malloc(sizeof(double) * (size_t)w);
  if (!Wc || !Vh || !beta || !cn2 || !d) {
    free(Wc); free(Vh); free(beta); free(cn2); free(d);
    return -1;
  }
  or_copy(n * w, Wc, W);
  for (int j = 0; j < w; j++) or_col_dots(0, n, W, w, j, W, w, j, 1, &cn2[j]);
  for (int j = 0; j < w; j++) {
    /* Householder vector for Wc[j:, j]. */
    double nx2;
    or_col_dots(j, n, Wc, w, j, Wc, w, j, 1, &nx2);
    double nx = sqrt(nx2);
    double x0 = Wc[(int64_t)j * w + j];
    double alpha = (x0 >= 0.0) ? -nx : nx;
    OR_PAR_FOR
    for (int64_t i = 0; i < n; i++) Vh[j * n + i] = (i >= j) ? Wc[i * w + j] : 0.0;
    Vh[j * n + j] -= alpha;
    double vn2;
    or_col_dots(j, n, Vh + j * n, 1, 0, Vh + j * n, 1, 0, 1, &vn2);
    beta[j] = (vn2 > 0.0) ? 2.0 / vn2 : 0.0;
    /* Apply H_j = I - beta v v^T to Wc[j:, j:]: d_c = beta v^T Wc[j:, c]
     * for every column c >= j, then Wc[j:, c] -= d_c v (each column's
     * update reads only that column). */
    or_col_dots(j, n, Vh + j * n, 1, 0, Wc, w, j, w - j, d);
    for (int c = j; c < w; c++) d[c - j] *= beta[j];
    OR_PAR_FOR
    for (int64_t i = j; i < n; i++)
      for (int c = j; c < w; c++) Wc[i * w + c] -= d[c - j] * Vh[j * n + i];
  }
  for (int a = 0; a < w; a++)
    for (int b = 0; b < w; b++) R[a * w + b] = (b >= a) ? Wc[(int64_t)a * w + b] : 0.0;
  /* Q = H_0 ... H_{w-1} [I; 0]. */
  OR_PAR_FOR
  for (int64_t i = 0; i < n; i++)
    for (int c = 0; c < w; c++) Q[i * w + c] = (i == c) ? 1.0 : 0.0;
  for (int j = w - 1; j >= 0; j--) {
    or_col_dots(j, n, Vh + j * n, 1, 0, Q, w, 0, w, d);
    for (int c = 0; c < w; c++) d[c] *= beta[j];
    OR_PAR_FOR
    for (int64_t i = j; i < n; i++)
      for (int c = 0; c < w; c++) Q[i * w + c] -= d[c] * Vh[j * n + i];
  }
  /* Make diag(R) nonnegative. */
  for (int j = 0; j < w; j++) {
    if (R[j * w + j] < 0.0) {
      for (int b = 0; b < w; b++) R[j * w + b] = -R[j * w + b];
      OR_PAR_FOR
      for (int64_t i = 0; i < n; i++) Q[i * w + j] = -Q[i * w + j];
    }
  }
  int status = 0;
  for (int j = 0; j < w; j++) {
    double rjj = R[j * w + j];
    if (!(rjj * rjj > OR_BREAKDOWN_RATIO * cn2[j]) || !isfinite(rjj)) {
      status = j + 1;
      break;
    }
  }
  free(Wc); free(Vh); free(beta); free(cn2); free(d);
  return status;
}

/* Dense SPD solve by Cholesky for the small agreement checks: A x = b with A
 * an n x n row-major matrix.  Returns 0, or 1 if a pivot is not positive. */
int or_dense_spd_solve(int n, const double* A, const double* b, double* x) {
  double* L = (double*)calloc((size_t)n * n, sizeof(double));
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  if (!L || !y) { free(L); free(y); return -1; }
  for (int j = 0; j < n; j++) {
    double d = A[j * n + j];
    for (int k = 0; k < j; k++) d -= L[j * n + k] * L[j * n + k];
    if (!(d > 0.0)) { free(L); free(y); return 1; }
    L[j * n + j] = sqrt(d);
    for (int i = j + 1; i < n; i++) {
      double s = A[i * n + j];
      for (int k = 0; k < j; k++) s -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = s / L[j * n + j];
    }
  }
  for (int i = 0; i < n; i++) {
    double s = b[i];
    for (int k = 0; k < i; k++) s -= L[i * n + k] * y[k];
    y[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; i--) {
    double s = y[i];
    for (int k = i + 1; k < n; k++) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
  free(L); free(y);
  return 0;
}

/* ------------------------------------------------------ A-orthonormalisation */

/* A-orthonormalise the n x w block W in place ("A-orthonormalize W_k",
 * Algorithm 1 lines 4 and 8).  On return W holds W_k with W_k^T A W_k = I and
 * V holds A W_k.  mode 0: Pre-CholQR (Householder QR W = Q_e R_e, then
 * A-CholQR of Q_e: Q_e^T A Q_e = S^T S, W_k = Q_e S^{-1}, A W_k =
 * (A Q_e) S^{-1}).  mode 1: A-CholQR (W^T A W = R^T R, W_k = W R^{-1}).
 * mode 2: Pre-CholQR with CholQR as the Euclidean step (W^T W = R_e^T R_e,
 * Q_e = W R_e^{-1}, then the A-CholQR of Q_e as in mode 0); Section 5 cites
 * Pre-CholQR without its body, and this is the reading the GPU follows.  In
 * exact arithmetic modes 0 and 2 give the same Q_e (the thin QR with a
 * positive diagonal is unique); in floating point CholQR's Q_e loses
 * orthogonality like eps kappa(W)^2, Householder's like eps.
 * Returns 0 or OR_EBREAKDOWN. */
int or_a_orthonormalize(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                        int w, int mode, double* W, double* V) {
  double* G = (double*)malloc(sizeof(double) * (size_t)(w * w));
  double* R = (double*)malloc(sizeof(double) * (size_t)(w * w));
  double* Qe = NULL;
  int status = OR_OK;
  if (!G || !R) { free(G); free(R); return OR_ENOMEM; }
  if (mode == 0) {
    Qe = (double*)malloc(sizeof(double) * (size_t)(n * w));
    if (!Qe) { free(G); free(R); return OR_ENOMEM; }
    int qs = or_householder_qr(n, w, W, Qe, R);
    if (qs < 0) { status = OR_ENOMEM; goto done; }
    if (qs > 0) { status = OR_EBREAKDOWN; goto done; }
    or_copy(n * w, W, Qe);
  } else if (mode == 2) {
    or_block_tdot(n, w, W, w, W, G);
    if (or_cholesky(w, G, R) != 0) { status = OR_EBREAKDOWN; goto done; }
    or_right_trsm(n, w, R, W);
  }
  or_spmm(n, rowptr, col, val, w, W, V);
  or_block_tdot(n, w, W, w, V, G);
  if (or_cholesky(w, G, R) != 0) { status = OR_EBREAKDOWN; goto done; }
  or_right_trsm(n, w, R, W);
  or_right_trsm(n, w, R, V);
done:
  free(G); free(R); free(Qe);
  return status;
}

/* Two passes of block classical Gram-Schmidt in the A-inner product of W
 * (n x w) against the m stored blocks Q_j (n x wq[j]) with V_j = A Q_j
 * ("A-orthonormalize W_k against Q", Algorithm 1 line 7; CGS2 per Sections
 * 2.1 and 5).  Each pass computes every coefficient block C_j = V_j^T W from
 * the same W, then subtracts sum_j Q_j C_j. */
int or_cgs2(int64_t n, int m, const double* const* Q, const double* const* V, const int* wq, int w,
            double* W) {
  int tot = 0;
  for (int j = 0; j < m; j++) tot += wq[j];
  double* C = (double*)malloc(sizeof(double) * (size_t)((tot > 0 ? tot : 1) * w));
  if (!C) return OR_ENOMEM;
  for (int pass = 0; pass < 2; pass++) {
    int off = 0;
    for (int j = 0; j < m; j++) {
      or_block_tdot(n, wq[j], V[j], w, W, C + (size_t)off * w);
      off += wq[j];
    }
    off = 0;
    for (int j = 0; j < m; j++) {
      or_block_sub(n, wq[j], Q[j], w, C + (size_t)off * w, W);
      off += wq[j];
    }
  }
  free(C);
  return OR_OK;
}

/* ----------------------------------------------------------------- solvers */

typedef struct {
  int iters;            /* loop bodies executed (k - 1 at exit) */
  int switch_it;        /* k_F: last iteration with t vectors; 0 if no switch */
  int status;           /* OR_OK, OR_ENOCONV, OR_EBREAKDOWN, OR_EINVAL, ... */
  int64_t mem_vectors;  /* largest number of stored basis vectors */
  double relres;        /* rho_k / rho_0 (recursively updated residual) */
  double relres_true;   /* ||b - A x|| / ||b|| */
  int restarts;         /* restarts performed (Section 3) */
} or_result;

/* Restart controls of Section 3 (all zero: no restart).  every = j >= 2
 * restarts at the iterations k with k mod j == 1; tol > 0 restarts when
 * |rho_{k-1} - rho_{k-2}| / rho_c < tol, rho_c the residual norm at the
 * start of the current cycle (rho_0 for the first cycle; at most max_count
 * times when max_count > 0); at_switch = 1 restarts at the flexible switch
 * (the "restarted flexibly" variant of Tables 8 and 9).  Reading: Section 3
 * writes ||r_0|| in the restart test; taken literally it holds at every
 * iteration once rho_k < tol * rho_0, which contradicts the 1 to 59
 * restarts of Tables 4 and 5, so ||r_0|| is read as the initial residual of
 * the restarted cycle.  A restart discards the
 * stored blocks and takes the new block from [T(r_{k-1})], as at k = 1, with
 * the width in force (t, or t/2 after the switch); the stopping test keeps
 * comparing with rho_0. */
typedef struct {
  int every;
  double tol;
  int max_count;
  int at_switch;
} or_restart;

/* ---------------------------------------------------- block-Jacobi factor */

/* Block-Jacobi preconditioner M = L L^T with L = diag(L_1, ..., L_nb), L_i
 * the lower-triangular factor of the diagonal block A_i = A(I_i, I_i) of
 * the rows I_i of block i (Section 3 "Preconditioned versions", and the
 * block Jacobi preconditioner of eq. (cholprec) in Section 5).  kind 0:
 * the exact Cholesky factor of A_i; kind 1: the incomplete Cholesky factor
 * with zero fill (IC(0)), which keeps the pattern of the lower triangle of
 * A_i and matches A_i = L_i L_i^T on that pattern.  Both are computed by the
 * same row-by-row Cholesky recurrence, on the full lower triangle for kind 0
 * and on the pattern of A_i for kind 1.  Inside a block the rows keep
 * increasing global order.
 *
 * Storage: position p = bptr[i] + (local index) enumerates the rows block
 * by block; row p of L holds its entries in increasing local column order
 * with the diagonal last. */
typedef struct {
  int64_t n;
  int nb;
  int kind;
  int64_t* bptr;  /* nb + 1 */
  int64_t* rows;  /* n: global row of position p */
  int64_t* pos;   /* n: position of global row i */
  int32_t* blk;   /* n: block of position p */
  int64_t* lptr;  /* n + 1 */
  int32_t* lcol;  /* local column */
  double* lval;
} or_prec;

void or_prec_free(or_prec* pc) {
  if (!pc) return;
  free(pc->bptr); free(pc->rows); free(pc->pos); free(pc->blk);
  free(pc->lptr); free(pc->lcol); free(pc->lval);
  free(pc);
}

/* Entry (i, j) of A with global indices (0 when absent). */
static double or_a_entry(const int64_t* rowptr, const int32_t* col, const double* val, int64_t i,
                         int64_t j) {
  double s = 0.0;
  for (int64_t q = rowptr[i]; q < rowptr[i + 1]; q++) if (col[q] == j) s += val[q];
  return s;
}

/* Builds the factor.  pblock[i] in [0, nb) is the block of row i; every
 * block must be non-empty.  Returns OR_ENOTSPD when a pivot is not positive
 * (IC(0) can break down on matrices that are not M-matrices). */
int or_prec_setup(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                  const int32_t* pblock, int nb, int kind, or_prec** out) {
  *out = NULL;
  if (n <= 0 || nb < 1 || (kind != 0 && kind != 1)) return OR_EINVAL;
  or_prec* pc = (or_prec*)calloc(1, sizeof(or_prec));
  if (!pc) return OR_ENOMEM;
  pc->n = n;
  pc->nb = nb;
  pc->kind = kind;
  pc->bptr = (int64_t*)calloc((size_t)nb + 1, sizeof(int64_t));
  pc->rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  pc->pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  pc->blk = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  pc->lptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!pc->bptr || !pc->rows || !pc->pos || !pc->blk || !pc->lptr) { or_prec_free(pc); return OR_ENOMEM; }
  for (int64_t i = 0; i < n; i++) {
    if (pblock[i] < 0 || pblock[i] >= nb) { or_prec_free(pc); return OR_EINVAL; }
    pc->bptr[pblock[i] + 1]++;
  }
  for (int b = 0; b < nb; b++) {
    if (pc->bptr[b + 1] == 0) { or_prec_free(pc); return OR_EINVAL; }
    pc->bptr[b + 1] += pc->bptr[b];
  }
  {
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nb);
    if (!fill) { or_prec_free(pc); return OR_ENOMEM; }
    for (int b = 0; b < nb; b++) fill[b] = pc->bptr[b];
    for (int64_t i = 0; i < n; i++) { /* increasing i keeps each block sorted */
      int64_t p = fill[pblock[i]]++;
      pc->rows[p] = i;
      pc->pos[i] = p;
      pc->blk[p] = pblock[i];
    }
    free(fill);
  }
  /* pattern: local columns j <= i of the lower triangle (full for kind 0);
   * lptr[p + 1] first holds the count of row p */
  OR_PAR_FOR
  for (int64_t p = 0; p < n; p++) {
    const int b = pc->blk[p];
    const int64_t li = p - pc->bptr[b];
    int64_t cnt = 0;
    if (kind == 0) {
      cnt = li + 1;
    } else {
      const int64_t i = pc->rows[p];
      for (int64_t q = rowptr[i]; q < rowptr[i + 1]; q++) {
        const int64_t j = col[q];
        if (j == i || pblock[j] != b || pc->pos[j] >= p) continue;
        /* count each distinct column once */
        int seen = 0;
        for (int64_t q2 = rowptr[i]; q2 < q; q2++) if (col[q2] == j) seen = 1;
        if (!seen) cnt++;
      }
      cnt += 1; /* diagonal */
    }
    pc->lptr[p + 1] = cnt;
  }
  for (int64_t p = 0; p < n; p++) pc->lptr[p + 1] += pc->lptr[p];
  const int64_t nnz = pc->lptr[n];
  pc->lcol = (int32_t*)malloc(sizeof(int32_t) * (size_t)nnz);
  pc->lval = (double*)malloc(sizeof(double) * (size_t)nnz);
  if (!pc->lcol || !pc->lval) { or_prec_free(pc); return OR_ENOMEM; }
  OR_PAR_FOR
  for (int64_t p = 0; p < n; p++) {
    const int b = pc->blk[p];
    const int64_t li = p - pc->bptr[b];
    const int64_t i = pc->rows[p];
    int64_t e = pc->lptr[p];
    if (kind == 0) {
      for (int64_t lj = 0; lj <= li; lj++) pc->lcol[e++] = (int32_t)lj;
    } else {
      for (int64_t q = rowptr[i]; q < rowptr[i + 1]; q++) {
        const int64_t j = col[q];
        if (j == i || pblock[j] != b || pc->pos[j] >= p) continue;
        const int32_t lj = (int32_t)(pc->pos[j] - pc->bptr[b]);
        int seen = 0;
        for (int64_t e2 = pc->lptr[p]; e2 < e; e2++) if (pc->lcol[e2] == lj) seen = 1;
        if (seen) continue;
        /* insertion in increasing column order */
        int64_t at = e;
        while (at > pc->lptr[p] && pc->lcol[at - 1] > lj) { pc->lcol[at] = pc->lcol[at - 1]; at--; }
        pc->lcol[at] = lj;
        e++;
      }
      pc->lcol[e++] = (int32_t)li;
    }
  }
  /* Row-by-row Cholesky on the pattern:
   *   l_ij = (a_ij - sum_{k < j} l_ik l_jk) / l_jj   for j < i in the pattern,
   *   l_ii = sqrt(a_ii - sum_{k < i} l_ik^2),
   * the sums running over the columns k present in both rows.  A row only
   * reads rows of its own block, so the blocks are independent. */
  int notspd = 0;
  OR_PAR_FOR
  for (int bb = 0; bb < nb; bb++)
  for (int64_t p = pc->bptr[bb]; p < pc->bptr[bb + 1]; p++) {
    const int b = bb;
    const int64_t i = pc->rows[p];
    const int64_t e0 = pc->lptr[p], e1 = pc->lptr[p + 1];
    for (int64_t e = e0; e < e1 - 1; e++) {
      const int64_t pj = pc->bptr[b] + pc->lcol[e];
      double s = or_a_entry(rowptr, col, val, i, pc->rows[pj]);
      /* merge row i's entries before e with row j's off-diagonal entries */
      int64_t a = e0, c = pc->lptr[pj];
      const int64_t cend = pc->lptr[pj + 1] - 1;
      while (a < e && c < cend) {
        if (pc->lcol[a] == pc->lcol[c]) { s -= pc->lval[a] * pc->lval[c]; a++; c++; }
        else if (pc->lcol[a] < pc->lcol[c]) a++;
        else c++;
      }
      pc->lval[e] = s / pc->lval[pc->lptr[pj + 1] - 1];
    }
    double d = or_a_entry(rowptr, col, val, i, i);
    for (int64_t e = e0; e < e1 - 1; e++) d -= pc->lval[e] * pc->lval[e];
    if (!(d > 0.0)) {
      /* a failed pivot ends this block; the factor is discarded below */
#ifdef _OPENMP
#pragma omp atomic write
#endif
      notspd = 1;
      break;
    }
    pc->lval[e1 - 1] = sqrt(d);
  }
  if (notspd) { or_prec_free(pc); return OR_ENOTSPD; }
  *out = pc;
  return OR_OK;
}

int64_t or_prec_nnz(const or_prec* pc) { return pc->lptr[pc->n]; }

/* The factor in global coordinates: entry q is L[I[q], J[q]] = V[q]. */
void or_prec_export(const or_prec* pc, int64_t* I, int64_t* J, double* V) {
  for (int64_t p = 0; p < pc->n; p++) {
    const int b = pc->blk[p];
    for (int64_t e = pc->lptr[p]; e < pc->lptr[p + 1]; e++) {
      I[e] = pc->rows[p];
      J[e] = pc->rows[pc->bptr[b] + pc->lcol[e]];
      V[e] = pc->lval[e];
    }
  }
}

/* X <- L^{-1} X for an n x w block (forward substitution in each block;
 * the blocks are independent). */
void or_prec_lsolve(const or_prec* pc, int w, double* X) {
  OR_PAR_FOR
  for (int b = 0; b < pc->nb; b++)
  for (int64_t p = pc->bptr[b]; p < pc->bptr[b + 1]; p++) {
    const int64_t i = pc->rows[p];
    const int64_t e1 = pc->lptr[p + 1];
    for (int c = 0; c < w; c++) {
      double s = X[i * w + c];
      for (int64_t e = pc->lptr[p]; e < e1 - 1; e++)
        s -= pc->lval[e] * X[pc->rows[pc->bptr[b] + pc->lcol[e]] * w + c];
      X[i * w + c] = s / pc->lval[e1 - 1];
    }
  }
}

/* X <- L^{-T} X for an n x w block (backward substitution in each block,
 * by columns of L: solve for the last unknown, then remove it). */
void or_prec_ltsolve(const or_prec* pc, int w, double* X) {
  OR_PAR_FOR
  for (int b = 0; b < pc->nb; b++)
  for (int64_t p = pc->bptr[b + 1] - 1; p >= pc->bptr[b]; p--) {
    const int64_t i = pc->rows[p];
    const int64_t e1 = pc->lptr[p + 1];
    for (int c = 0; c < w; c++) {
      const double z = X[i * w + c] / pc->lval[e1 - 1];
      X[i * w + c] = z;
      for (int64_t e = pc->lptr[p]; e < e1 - 1; e++)
        X[pc->rows[pc->bptr[b] + pc->lcol[e]] * w + c] -= pc->lval[e] * z;
    }
  }
}

/* X <- M^{-1} X = L^{-T} L^{-1} X. */
void or_prec_apply(const or_prec* pc, int w, double* X) {
  or_prec_lsolve(pc, w, X);
  or_prec_ltsolve(pc, w, X);
}

/* W = L^{-T} [T(L^{-1} r)]: the preconditioned split of Algorithm 5 and eq.
 * (zsre2), taken literally (half = 1: the t/2 split). */
static void or_prec_split(const or_prec* pc, int64_t n, const int32_t* part, int t, int half,
                          const double* r, double* tmp, double* W) {
  memcpy(tmp, r, sizeof(double) * (size_t)n);
  or_prec_lsolve(pc, 1, tmp);
  if (half) or_split_half(n, part, t, tmp, W);
  else or_split(n, part, t, tmp, W);
  or_prec_ltsolve(pc, half ? t / 2 : t, W);
}

static double or_norm2(int64_t n, const double* v) { return sqrt(or_dot(n, v, v)); }

/* The MSDO-CG direction of Algorithm 2 (lines 6-7): on entry P holds the
 * split [T(r_{k-1})] (n x w); on return beta = -V_{k-1}^T z (w entries) and
 * P = [T(r_{k-1})] + P_{k-1} diag(beta).  z is r_{k-1}, or M^{-1} r_{k-1} in
 * the preconditioned form of Algorithm 5.  Reading: eq. (pk) prints
 * P_{k-1}^t A r where Algorithm 2 writes V_{k-1}^T r; with V_{k-1} = A P_{k-1}
 * both are the same vector, computed here from the stored V_{k-1}. */
void or_msdo_direction(int64_t n, int w, const double* Pprev, const double* Vprev, const double* z,
                       double* beta, double* P) {
  or_block_tdot(n, w, Vprev, 1, z, beta);
  for (int j = 0; j < w; j++) beta[j] = -beta[j];
  OR_PAR_FOR
  for (int64_t i = 0; i < n; i++)
    for (int j = 0; j < w; j++) P[i * w + j] += Pprev[i * w + j] * beta[j];
}

/* Enlarged CG.  variant 0: SRE-CG2 (Algorithm 1; W_k = A W_{k-1}); 1: MSDO-CG
 * (Algorithm 2; P_k = T(r_{k-1}) + P_{k-1} diag(beta_k), beta_k =
 * -V_{k-1}^T r_{k-1}); 2: modified MSDO-CG (Section 2.2; W_k = T(r_{k-1})).
 * trunc == 0 orthonormalises against every stored block; trunc >= 1 against
 * the last trunc blocks only (Section 3; trunc = 2 on variant 0 is SRE-CG).
 * switch_tol > 0 enables the flexible halving of Algorithms 3 and 4.
 * ortho: 0 Pre-CholQR, 1 A-CholQR, 2 Pre-CholQR with a CholQR Euclidean
 * step (or_a_orthonormalize).  k_max follows Algorithm 1 (at most
 * k_max - 1 iterations).  history (length k_max, may be NULL) receives rho_k
 * for k = 0..iters.  xhist (n * (k_max - 1), may be NULL) receives x_k after
 * iteration k at offset (k-1)*n.  basis (may be NULL) receives every W_k
 * in order, block after block (n * sum of widths entries, capacity
 * basis_cap doubles); widths (k_max entries, may be NULL) their widths.
 * pc (may be NULL) is a block-Jacobi preconditioner M = L L^T: the
 * generated blocks become those of Section 3 "Preconditioned versions"
 * (eq. (zsre2), (zmsd2), Algorithm 5): every [T(r)] is replaced by
 * L^{-T}[T(L^{-1} r)], W_k = A W_{k-1} by M^{-1} A W_{k-1}, and beta_k =
 * -V_{k-1}^T (M^{-1} r_{k-1}); alpha_k, x_k, r_k and the A-orthonormalisation
 * are unchanged, and rho_k stays the norm of the unpreconditioned
 * residual. */
int or_ecg_solve(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                 const int32_t* part, int t, int variant, int trunc, double switch_tol, int ortho,
                 const double* b, const double* x0, double eps, int kmax, double* x,
                 double* history, double* xhist, double* basis, int64_t basis_cap, int* widths,
                 const or_restart* rs, const or_prec* pc, or_result* res) {
  memset(res, 0, sizeof(*res));
  or_restart rsz;
  memset(&rsz, 0, sizeof(rsz));
  if (!rs) rs = &rsz;
  if (n <= 0 || t < 1 || variant < 0 || variant > 2 || trunc < 0 || ortho < 0 || ortho > 2 ||
      !(eps >= 0.0) || (switch_tol > 0.0 && (t % 2 != 0)) || rs->every == 1 || rs->every < 0 ||
      !(rs->tol >= 0.0) || rs->max_count < 0 || (rs->at_switch && !(switch_tol > 0.0))) {
    res->status = OR_EINVAL;
    return OR_EINVAL;
  }
  {
    /* Every subdomain must be non-empty and every id in [0, t). */
    int* cnt = (int*)calloc((size_t)t, sizeof(int));
    if (!cnt) { res->status = OR_ENOMEM; return OR_ENOMEM; }
    int bad = 0;
    for (int64_t i = 0; i < n; i++) {
      if (part[i] < 0 || part[i] >= t) { bad = 1; break; }
      cnt[part[i]]++;
    }
    for (int j = 0; j < t && !bad; j++) if (cnt[j] == 0) bad = 1;
    free(cnt);
    if (bad) { res->status = OR_EINVAL; return OR_EINVAL; }
  }
  for (int64_t i = 0; i < n; i++) {
    double d = 0.0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) if (col[p] == i) d += val[p];
    if (!(d > 0.0)) { res->status = OR_ENOTSPD; return OR_ENOTSPD; }
  }

  int cap = (trunc == 0) ? (kmax > 1 ? kmax : 1) : trunc; /* blocks kept in Q */
  double** Qb = (double**)calloc((size_t)cap, sizeof(double*));
  double** Vb = (double**)calloc((size_t)cap, sizeof(double*));
  int* wq = (int*)calloc((size_t)cap, sizeof(int));
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* tmp = (double*)malloc(sizeof(double) * (size_t)n);
  double* z = (double*)malloc(sizeof(double) * (size_t)n); /* M^{-1} r_{k-1} */
  double* W = (double*)malloc(sizeof(double) * (size_t)(n * t));
  double* Vn = (double*)malloc(sizeof(double) * (size_t)(n * t));
  double* Pprev = (double*)malloc(sizeof(double) * (size_t)(n * t)); /* P_{k-1} */
  double* Vprev = (double*)malloc(sizeof(double) * (size_t)(n * t)); /* V_{k-1} = A P_{k-1} */
  double* alpha = (double*)malloc(sizeof(double) * (size_t)t);
  double* beta = (double*)malloc(sizeof(double) * (size_t)t);
  const double** qs = (const double**)calloc((size_t)cap, sizeof(double*));
  const double** vs = (const double**)calloc((size_t)cap, sizeof(double*));
  int* ws = (int*)calloc((size_t)cap, sizeof(int));
  double rho0 = 0.0;
  int64_t mem = 0;
  int status = OR_ENOCONV;
  int k = 1;
  if (!Qb || !Vb || !wq || !r || !tmp || !z || !W || !Vn || !Pprev || !Vprev || !alpha || !beta || !qs ||
      !vs || !ws) {
    status = OR_ENOMEM;
    goto out;
  }

  /* Algorithm 1 line 1: r0 = b - A x0, rho0 = ||r0||. */
  if (x0) memcpy(x, x0, sizeof(double) * (size_t)n);
  else memset(x, 0, sizeof(double) * (size_t)n);
  or_spmv(n, rowptr, col, val, x, tmp);
  OR_PAR_FOR
  for (int64_t i = 0; i < n; i++) r[i] = b[i] - tmp[i];
  rho0 = or_norm2(n, r);
  double rho_prev = rho0;
  double tol1 = 1.0;
  double rtol1 = 1.0;        /* |rho_{k-1} - rho_{k-2}| / rho_c */
  double rho_cycle = rho0;   /* residual norm at the start of the cycle */
  int counter = 0;
  int width = t;      /* width of the block generated this iteration */
  int wprev = t;      /* width of W_{k-1} / P_{k-1} */
  int nq = 0;         /* blocks currently in Q */
  int head = 0;       /* ring position of the oldest block */
  int64_t basis_used = 0;
  if (history) history[0] = rho0;

  while (rho_prev > eps * rho0 && k < kmax) {
    /* ---- generate the raw block (Algorithms 1-4, lines 3-11) ---- */
    int do_switch = (k > 1 && switch_tol > 0.0 && tol1 < switch_tol && counter == 0);
    int do_restart = 0;
    if (k > 1) {
      if (rs->every >= 2 && k % rs->every == 1) do_restart = 1;
      if (rs->tol > 0.0 && rtol1 < rs->tol && (rs->max_count == 0 || res->restarts < rs->max_count))
        do_restart = 1;
      if (do_switch && rs->at_switch) do_restart = 1;
    }
    if (do_restart) { /* Section 3: discard Q, start again from x_{k-1} */
      nq = 0;
      head = 0;
      res->restarts++;
      rho_cycle = rho_prev;
    }
    if (k == 1) {
      width = t;
      /* W_1 = [T^t(r_0)], or L^{-T}[T^t(L^{-1} r_0)] */
      if (pc) or_prec_split(pc, n, part, t, 0, r, tmp, W);
      else or_split(n, part, t, r, W);
    } else if (do_switch) {
      width = t / 2;
      /* W_k = [T^{t/2}(r_{k-1})], or L^{-T}[T^{t/2}(L^{-1} r_{k-1})] */
      if (pc) or_prec_split(pc, n, part, t, 1, r, tmp, W);
      else or_split_half(n, part, t, r, W);
      counter = 1;
      res->switch_it = k - 1;
    } else if (do_restart) {
      width = wprev; /* [T(r_{k-1})] with the width in force */
      if (pc) or_prec_split(pc, n, part, t, width != t, r, tmp, W);
      else if (width == t) or_split(n, part, t, r, W);
      else or_split_half(n, part, t, r, W);
    } else {
      width = wprev;
      if (variant == 0) {
        or_copy(n * width, W, Vprev); /* W_k = A W_{k-1} */
        if (pc) or_prec_apply(pc, width, W);                     /* M^{-1} A W_{k-1} */
      } else {
        if (pc) or_prec_split(pc, n, part, t, width != t, r, tmp, W);
        else if (width == t) or_split(n, part, t, r, W);
        else or_split_half(n, part, t, r, W);
        if (variant == 1) {
          /* beta_k = -V_{k-1}^T r_{k-1} (-V_{k-1}^T M^{-1} r_{k-1} when
           * preconditioned); P_k = T(r_{k-1}) + P_{k-1} diag(beta_k). */
          memcpy(z, r, sizeof(double) * (size_t)n);
          if (pc) or_prec_apply(pc, 1, z);
          or_msdo_direction(n, width, Pprev, Vprev, z, beta, W);
        }
      }
    }

    /* ---- A-orthonormalise against Q (CGS2), then itself ---- */
    int64_t stored = width;
    if (k > 1 && nq > 0) {
      int m = nq;
      for (int j = 0; j < m; j++) {
        int slot = (head + j) % cap;
        qs[j] = Qb[slot];
        vs[j] = Vb[slot];
        ws[j] = wq[slot];
        stored += wq[slot];
      }
      int cs = or_cgs2(n, m, qs, vs, ws, width, W);
      if (cs != OR_OK) { status = cs; goto out; }
    }
    if (stored > mem) mem = stored;
    int st = or_a_orthonormalize(n, rowptr, col, val, width, ortho, W, Vn);
    if (st != OR_OK) { status = st; goto out; }

    /* ---- push (W_k, V_k) into Q, dropping the oldest beyond trunc ---- */
    {
      int slot;
      if (nq < cap) {
        slot = (head + nq) % cap;
        nq++;
      } else {
        slot = head;
        head = (head + 1) % cap;
      }
      if (!Qb[slot]) {
        Qb[slot] = (double*)malloc(sizeof(double) * (size_t)(n * t));
        Vb[slot] = (double*)malloc(sizeof(double) * (size_t)(n * t));
        if (!Qb[slot] || !Vb[slot]) { status = OR_ENOMEM; goto out; }
      }
      or_copy(n * width, Qb[slot], W);
      or_copy(n * width, Vb[slot], Vn);
      wq[slot] = width;
    }
    if (basis && basis_used + n * width <= basis_cap) {
      or_copy(n * width, basis + basis_used, W);
      basis_used += n * width;
    }
    if (widths) widths[k - 1] = width;

    /* ---- alpha_k = W_k^T r_{k-1}; x_k, r_k, rho_k (lines 12-15) ---- */
    or_block_tdot(n, width, W, 1, r, alpha);
    OR_PAR_FOR
    for (int64_t i = 0; i < n; i++) {
      double sx = 0.0, sr = 0.0;
      for (int j = 0; j < width; j++) {
        sx += W[i * width + j] * alpha[j];
        sr += Vn[i * width + j] * alpha[j];
      }
      x[i] += sx;
      r[i] -= sr;
    }
    double rho = or_norm2(n, r);
    tol1 = fabs(rho - rho_prev) / rho0;
    rtol1 = fabs(rho - rho_prev) / rho_cycle;
    rho_prev = rho;
    if (history) history[k] = rho;
    if (xhist) memcpy(xhist + (int64_t)(k - 1) * n, x, sizeof(double) * (size_t)n);
    or_copy(n * width, Pprev, W);
    or_copy(n * width, Vprev, Vn);
    wprev = width;
    k++;
  }
  if (status == OR_ENOCONV && rho_prev <= eps * rho0) status = OR_OK;

out:
  res->iters = k - 1;
  res->status = status;
  res->mem_vectors = mem;
  if (r && tmp) {
    double rr = or_norm2(n, r);
    res->relres = (rho0 > 0.0) ? rr / rho0 : rr;
    or_spmv(n, rowptr, col, val, x, tmp);
    OR_PAR_FOR
    for (int64_t i = 0; i < n; i++) tmp[i] = b[i] - tmp[i];
    double nb = or_norm2(n, b);
    res->relres_true = (nb > 0.0) ? or_norm2(n, tmp) / nb : or_norm2(n, tmp);
  }
  if (Qb) for (int j = 0; j < cap; j++) free(Qb[j]);
  if (Vb) for (int j = 0; j < cap; j++) free(Vb[j]);
  free(Qb); free(Vb); free(wq); free(r); free(tmp); free(z); free(W); free(Vn); free(Pprev); free(Vprev);
  free(alpha); free(beta); free(qs); free(vs); free(ws);
  return status;
}

/* Block-residual enlarged CG, the block CG method based on SRE-CG that the
 * paper mentions in Section 1 (one system solved as t right-hand sides):
 * R_0 = [T^t(r_0)], X_0 = 0 (n x t); each iteration takes the SRE-CG
 * direction block (W_1 = R_0, W_k = A W_{k-1}, A-orthonormalised by CGS2
 * against the last trunc blocks (all for trunc = 0) and then against
 * itself), and updates every column of the block residual with its own
 * coefficients:
 *   alpha_k = W_k^T R_{k-1} (t x t),  X_k = X_{k-1} + W_k alpha_k,
 *   R_k = R_{k-1} - A W_k alpha_k.
 * The solution of A x = b is x_k = x_0 + X_k 1, the sum of the columns
 * (A X_k 1 = R_0 1 - R_k 1 = r_0 - R_k 1), and rho_k = ||R_k 1||.
 * Readings: the paper gives only that sentence; the direction blocks,
 * orthonormalisation and loop bound are those of Algorithm 1, and the
 * stopping test is the paper's rho_k <= eps rho_0 on the summed residual.
 * history (k_max entries, may be NULL) receives rho_k; xhist (may be NULL)
 * x_k after iteration k at (k-1)*n; Xout (n x t, may be NULL) the final X. */
int or_becg_solve(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                  const int32_t* part, int t, int trunc, int ortho, const double* b, const double* x0,
                  double eps, int kmax, double* x, double* history, double* xhist, double* Xout,
                  or_result* res) {
  memset(res, 0, sizeof(*res));
  if (n <= 0 || t < 1 || trunc < 0 || ortho < 0 || ortho > 2 || !(eps >= 0.0)) {
    res->status = OR_EINVAL;
    return OR_EINVAL;
  }
  for (int64_t i = 0; i < n; i++)
    if (part[i] < 0 || part[i] >= t) { res->status = OR_EINVAL; return OR_EINVAL; }
  const int cap = (trunc == 0) ? (kmax > 1 ? kmax : 1) : trunc;
  double** Qb = (double**)calloc((size_t)cap, sizeof(double*));
  double** Vb = (double**)calloc((size_t)cap, sizeof(double*));
  const double** qs = (const double**)calloc((size_t)cap, sizeof(double*));
  const double** vs = (const double**)calloc((size_t)cap, sizeof(double*));
  int* ws = (int*)calloc((size_t)cap, sizeof(int));
  double* R = (double*)malloc(sizeof(double) * (size_t)(n * t));
  double* X = (double*)calloc((size_t)(n * t), sizeof(double));
  double* W = (double*)malloc(sizeof(double) * (size_t)(n * t));
  double* Vn = (double*)malloc(sizeof(double) * (size_t)(n * t));
  double* Vprev = (double*)malloc(sizeof(double) * (size_t)(n * t));
  double* alpha = (double*)malloc(sizeof(double) * (size_t)(t * t));
  double* tmp = (double*)malloc(sizeof(double) * (size_t)n);
  int status = OR_ENOCONV, k = 1, nq = 0, head = 0;
  double rho0 = 0.0, rho_prev = 0.0;
  if (!Qb || !Vb || !qs || !vs || !ws || !R || !X || !W || !Vn || !Vprev || !alpha || !tmp) {
    status = OR_ENOMEM;
    goto out;
  }
  if (x0) memcpy(x, x0, sizeof(double) * (size_t)n);
  else memset(x, 0, sizeof(double) * (size_t)n);
  or_spmv(n, rowptr, col, val, x, tmp);
  for (int64_t i = 0; i < n; i++) tmp[i] = b[i] - tmp[i];
  rho0 = or_norm2(n, tmp);
  rho_prev = rho0;
  if (history) history[0] = rho0;
  or_split(n, part, t, tmp, R); /* R_0 = [T^t(r_0)] */
  while (rho_prev > eps * rho0 && k < kmax) {
    if (k == 1) or_copy(n * t, W, R); /* W_1 = R_0 */
    else or_copy(n * t, W, Vprev);    /* W_k = A W_{k-1} */
    if (k > 1 && nq > 0) {
      for (int j = 0; j < nq; j++) {
        const int slot = (head + j) % cap;
        qs[j] = Qb[slot];
        vs[j] = Vb[slot];
        ws[j] = t;
      }
      const int cs = or_cgs2(n, nq, qs, vs, ws, t, W);
      if (cs != OR_OK) { status = cs; goto out; }
    }
    {
      const int st = or_a_orthonormalize(n, rowptr, col, val, t, ortho, W, Vn);
      if (st != OR_OK) { status = st; goto out; }
    }
    {
      int slot;
      if (nq < cap) { slot = (head + nq) % cap; nq++; }
      else { slot = head; head = (head + 1) % cap; }
      if (!Qb[slot]) {
        Qb[slot] = (double*)malloc(sizeof(double) * (size_t)(n * t));
        Vb[slot] = (double*)malloc(sizeof(double) * (size_t)(n * t));
        if (!Qb[slot] || !Vb[slot]) { status = OR_ENOMEM; goto out; }
      }
      or_copy(n * t, Qb[slot], W);
      or_copy(n * t, Vb[slot], Vn);
    }
    /* alpha_k = W_k^T R_{k-1}; X += W alpha; R -= V alpha */
    or_block_tdot(n, t, W, t, R, alpha);
    for (int64_t i = 0; i < n; i++)
      for (int c = 0; c < t; c++) {
        double sx = 0.0, sr = 0.0;
        for (int a = 0; a < t; a++) {
          sx += W[i * t + a] * alpha[a * t + c];
          sr += Vn[i * t + a] * alpha[a * t + c];
        }
        X[i * t + c] += sx;
        R[i * t + c] -= sr;
      }
    for (int64_t i = 0; i < n; i++) {
      double sr = 0.0, sx = 0.0;
      for (int c = 0; c < t; c++) {
        sr += R[i * t + c];
        sx += X[i * t + c];
      }
      tmp[i] = sr;
      x[i] = (x0 ? x0[i] : 0.0) + sx;
    }
    const double rho = or_norm2(n, tmp);
    rho_prev = rho;
    if (history) history[k] = rho;
    if (xhist) memcpy(xhist + (int64_t)(k - 1) * n, x, sizeof(double) * (size_t)n);
    or_copy(n * t, Vprev, Vn);
    k++;
  }
  if (status == OR_ENOCONV && rho_prev <= eps * rho0) status = OR_OK;
out:
  res->iters = k - 1;
  res->status = status;
  res->mem_vectors = (int64_t)t * (nq + 3);
  if (tmp && X) {
    res->relres = (rho0 > 0.0) ? rho_prev / rho0 : rho_prev;
    or_spmv(n, rowptr, col, val, x, tmp);
    for (int64_t i = 0; i < n; i++) tmp[i] = b[i] - tmp[i];
    const double nb = or_norm2(n, b);
    res->relres_true = (nb > 0.0) ? or_norm2(n, tmp) / nb : or_norm2(n, tmp);
    if (Xout) or_copy(n * t, Xout, X);
  }
  if (Qb) for (int j = 0; j < cap; j++) free(Qb[j]);
  if (Vb) for (int j = 0; j < cap; j++) free(Vb[j]);
  free(Qb); free(Vb); free(qs); free(vs); free(ws); free(R); free(X); free(W); free(Vn); free(Vprev);
  free(alpha); free(tmp);
  return status;
}

/* Classical CG (Hestenes-Stiefel), the method of Section 1 that the enlarged
 * methods generalise.  Same loop convention as or_ecg_solve: at most
 * k_max - 1 iterations, stop when ||r_k|| <= eps ||r_0||. */
int or_cg_solve(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                const double* b, const double* x0, double eps, int kmax, double* x,
                double* history, double* xhist, or_result* res) {
  memset(res, 0, sizeof(*res));
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* p = (double*)malloc(sizeof(double) * (size_t)n);
  double* q = (double*)malloc(sizeof(double) * (size_t)n);
  if (!r || !p || !q) { free(r); free(p); free(q); res->status = OR_ENOMEM; return OR_ENOMEM; }
  if (x0) memcpy(x, x0, sizeof(double) * (size_t)n);
  else memset(x, 0, sizeof(double) * (size_t)n);
  or_spmv(n, rowptr, col, val, x, q);
  for (int64_t i = 0; i < n; i++) { r[i] = b[i] - q[i]; p[i] = r[i]; }
  double rr = or_dot(n, r, r);
  double rho0 = sqrt(rr), rho = rho0;
  if (history) history[0] = rho0;
  int k = 1;
  while (rho > eps * rho0 && k < kmax) {
    or_spmv(n, rowptr, col, val, p, q);
    double pq = or_dot(n, p, q);
    double a = rr / pq;
    for (int64_t i = 0; i < n; i++) { x[i] += a * p[i]; r[i] -= a * q[i]; }
    double rr_new = or_dot(n, r, r);
    double bcoef = rr_new / rr;
    for (int64_t i = 0; i < n; i++) p[i] = r[i] + bcoef * p[i];
    rr = rr_new;
    rho = sqrt(rr);
    if (history) history[k] = rho;
    if (xhist) memcpy(xhist + (int64_t)(k - 1) * n, x, sizeof(double) * (size_t)n);
    k++;
  }
  res->iters = k - 1;
  res->status = (rho <= eps * rho0) ? OR_OK : OR_ENOCONV;
  res->relres = rho0 > 0.0 ? rho / rho0 : rho;
  or_spmv(n, rowptr, col, val, x, q);
  double nb = or_norm2(n, b);
  for (int64_t i = 0; i < n; i++) q[i] = b[i] - q[i];
  res->relres_true = nb > 0.0 ? or_norm2(n, q) / nb : or_norm2(n, q);
  free(r); free(p); free(q);
  return res->status;
}

/* The paper's memory count (Tables 6-9): number of stored basis vectors of a
 * flexible run, t per iteration up to switch_it, t/2 afterwards; t * iters
 * without a switch. */
int64_t or_mem_flexible(int t, int iters, int switch_it) {
  if (switch_it <= 0) return (int64_t)t * iters;
  return (int64_t)t * switch_it + (int64_t)(t / 2) * (iters - switch_it);
}
