// ecg_kernels.cuh -- sm_103a kernels of the enlarged CG iteration (FP64).
//
// Method: S. Moufawad, "Flexibly Enlarged Conjugate Gradient methods"
// (arXiv 2305.19013), Algorithms 1-4.  One iteration k is the kernel chain
//
//   k_generate      raw block X: [T^t(r)], [T^{t/2}(r)], A W_{k-1} or the
//                   MSDO direction T(r) + P_{k-1} diag(beta)   (eq. (Tt), Alg. 1-4)
//   2 x (k_tdot_window + k_reduce_C + k_update)
//                   CGS2 against the stored window: C = V^T X, X -= Q C
//   k_gram_self + k_small_e   (Pre-CholQR only) X^T X = R_e^T R_e, R_e^{-1}
//   k_spmm_gram     Y = A X, G = q^T (A q), g = q^T r with q = X R_e^{-1}
//   k_small_a       G = S^T S, R^{-1} = R_e^{-1} S^{-1}, alpha = S^{-T} g
//   k_final         W_k = X R^{-1}, V_k = Y R^{-1} into the window slot,
//                   x += W_k alpha, r -= V_k alpha, partial ||r||^2 (and the
//                   MSDO beta = -V_k^T r_k partials)
//   k_finish        rho_k, history, switch and stop decisions, window push
//
// All iteration state lives in device memory (DevState), so the same launch
// sequence serves every iteration and can be captured in a CUDA graph.
// Every kernel first checks the state and returns at once when the solve
// has stopped or when the current block width differs from its template
// width W (which happens right after the flexible switch, until the host
// moves to the t/2 kernels).
//
// GB300 has about 1.2 TFLOP/s of FP64 against 6.7 TB/s of HBM, so every
// n x t block pass here is bound by FP64 FMA issue, not by memory.  The
// kernels therefore stage row tiles in shared memory and give each thread
// distinct output entries, so that every DFMA issued is a useful one
// (symmetric Grams compute their upper triangle only).  Reductions over
// rows are two-stage and fixed-order: each CTA writes its partial sums and
// a second kernel adds them in CTA order, so repeated solves are bitwise
// identical.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ecg {

constexpr int kThreads = 256;
constexpr int kChunk = 64;  // window columns per CGS chunk
constexpr double kBreakdownRatio = 1e-14;

enum Gen { GEN_SPLIT = 0, GEN_SRE = 1, GEN_MSDO = 2 };
enum Status { ST_OK = 0, ST_ENOCONV = 1, ST_EBREAKDOWN = -4 };

struct BlockDesc {
  double* W;  // A-orthonormal block W_j (n x w)
  double* V;  // A W_j (n x w)
  int w;      // width
  int off;    // first column of this block in the concatenated window
  int slot;   // storage slot index
  int pad;
};

struct DevState {
  int k;          // iteration about to run (1-based)
  int width;      // width of the block built in iteration k
  int gen;        // Gen of iteration k
  int stop;       // nonzero once the loop has ended
  int status;     // final status when stop != 0
  int counter;    // 1 after the flexible switch
  int switch_it;  // k_F
  int nq;         // blocks in the window
  int kmax;
  int iters;      // iterations completed
  int variant;    // 0 SRE, 1 MSDO, 2 modified MSDO
  int cap;        // window capacity (blocks)
  int t;
  int next_slot;  // storage slot for the block of iteration k
  long long mem;  // largest number of stored basis vectors
  double eps, switch_tol;
  double rho0, rho_prev, tol1, rho;
};

// Offsets of the small matrices inside KP::small (t <= 64).
constexpr int kSmallG = 0;                 // reduced Gram (upper) / scratch
constexpr int kSmallRe = kSmallG + 4096;   // R_e^{-1}
constexpr int kSmallRi = kSmallRe + 4096;  // R^{-1} = R_e^{-1} S^{-1}
constexpr int kSmallAl = kSmallRi + 4096;  // alpha
constexpr int kSmallBe = kSmallAl + 64;    // beta
constexpr int kSmallSize = kSmallBe + 64;

struct KP {
  int n, t;
  const int* rowptr;
  const int* col;
  const double* val;
  const int* part;
  double* X;  // raw block of the iteration (n x W)
  double* Y;  // A X (n x W)
  double* x;
  double* r;
  const double* b;
  DevState* st;
  BlockDesc* desc;   // window, oldest first
  double* slotW;     // window storage, slot s at slotW + s * slot_stride
  double* slotV;
  long long slot_stride;
  double* C;         // CGS coefficients, (window columns) x W
  double* part_buf;  // per-CTA partial sums
  double* small;     // small matrices, see kSmall*
  double* history;   // rho_k, k = 0..kmax-1
  double* rho_part;  // per-CTA partial ||r||^2
  double* beta_part; // per-CTA partial V^T r (64 per CTA)
  int want_beta;     // accumulate beta partials in k_final (MSDO-CG)
};

__device__ __forceinline__ bool skip(const DevState* st, int w) {
  return st->stop != 0 || st->width != w;
}

template <int W>
struct Tile {
  // rows per shared-memory tile
  static constexpr int R = (W >= 64) ? 16 : 32;
};

__device__ __forceinline__ void cta_rows(int n, int& r0, int& r1) {
  long long per = ((long long)n + gridDim.x - 1) / gridDim.x;
  long long b = per * blockIdx.x;
  long long e = b + per;
  r0 = (int)(b < n ? b : n);
  r1 = (int)(e < n ? e : n);
}

// Fixed-order block reduction of one double per thread; result in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sbuf) {
  sbuf[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sbuf[threadIdx.x] += sbuf[threadIdx.x + s];
    __syncthreads();
  }
  double out = sbuf[0];
  __syncthreads();
  return out;
}

// Upper-triangle entry e -> (a, b), a <= b, row-major over a.
__device__ __forceinline__ void upper_ab(int e, int w, int& a, int& b) {
  int aa = 0;
  int rowlen = w;
  while (e >= rowlen) {
    e -= rowlen;
    aa++;
    rowlen--;
  }
  a = aa;
  b = aa + e;
}

// y = x U for one row x and an upper-triangular W x W matrix U, for the
// column pair (b1, b2) = (bp, W-1-bp): y1 = sum_{a<=b1} x_a U_{a,b1} and
// y2 = sum_{a<=b2} x_a U_{a,b2}.  Every pair costs W+1 FMAs per input row, so
// all lanes of a warp run the same trip count (one column per lane would
// leave lane b idle for W-1-b of the W steps).  Two rows (x, z) share U.
template <int W>
__device__ __forceinline__ void tri_pair2(const double* x, const double* z, const double* U, int bp,
                                          double& x1, double& x2, double& z1, double& z2) {
  const int b1 = bp, b2 = W - 1 - bp;
  double sx1 = 0.0, sx2 = 0.0, sz1 = 0.0, sz2 = 0.0;
#pragma unroll 4
  for (int j = 0; j <= W; j++) {
    const bool first = (j <= b1);
    const int a = first ? j : j - b1 - 1;
    const double u = U[a * W + (first ? b1 : b2)];
    const double vx = fma(x[a], u, first ? sx1 : sx2);
    const double vz = fma(z[a], u, first ? sz1 : sz2);
    if (first) {
      sx1 = vx;
      sz1 = vz;
    } else {
      sx2 = vx;
      sz2 = vz;
    }
  }
  x1 = sx1;
  x2 = sx2;
  z1 = sz1;
  z2 = sz2;
}

// Sum of in[c * stride + e] over c < count for every e < nent, written to
// out[e] via `store(e, sum)`: one warp per entry, lanes over c (lane l takes
// c = l, l+32, ...), then a fixed shuffle tree, so the result does not
// depend on timing.  All threads of the CTA must call it.
template <typename Store>
__device__ __forceinline__ void cta_reduce_partials(const double* in, long long stride, int count, int nent,
                                                    Store store) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int e = warp; e < nent; e += nw) {
    double s = 0.0;
    for (int c = lane; c < count; c += 32) s += in[(long long)c * stride + e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) store(e, s);
  }
}

// ----------------------------------------------------------------- setup

// r = b - A x (or r = b when x is null); per-CTA partial ||r||^2 and ||b||^2.
__global__ void __launch_bounds__(kThreads) k_residual(KP P, const double* x, double* rout,
                                                        double* part_rr, double* part_bb) {
  __shared__ double sbuf[kThreads];
  int r0, r1;
  cta_rows(P.n, r0, r1);
  double rr = 0.0, bb = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    double y = 0.0;
    if (x) {
      for (int p = P.rowptr[i]; p < P.rowptr[i + 1]; p++) y += P.val[p] * x[P.col[p]];
    }
    double bi = P.b[i];
    double ri = bi - y;
    if (rout) rout[i] = ri;
    rr += ri * ri;
    bb += bi * bi;
  }
  rr = block_sum(rr, sbuf);
  bb = block_sum(bb, sbuf);
  if (threadIdx.x == 0) {
    part_rr[blockIdx.x] = rr;
    if (part_bb) part_bb[blockIdx.x] = bb;
  }
}

// Algorithm 1 line 1: rho_0 and the loop state for k = 1.
__global__ void k_start(KP P, int nparts) {
  __shared__ double sbuf[kThreads];
  double s = 0.0;
  for (int c = threadIdx.x; c < nparts; c += blockDim.x) s += P.rho_part[c];
  s = block_sum(s, sbuf);
  if (threadIdx.x == 0) {
    DevState* st = P.st;
    double rho0 = sqrt(s);
    st->rho0 = rho0;
    st->rho_prev = rho0;
    st->rho = rho0;
    st->tol1 = 1.0;
    st->k = 1;
    st->width = st->t;
    st->gen = GEN_SPLIT;
    st->counter = 0;
    st->switch_it = 0;
    st->nq = 0;
    st->iters = 0;
    st->next_slot = 0;
    st->mem = 0;
    st->stop = 0;
    st->status = ST_ENOCONV;
    P.history[0] = rho0;
    if (!(rho0 > st->eps * rho0)) {
      st->stop = 1;
      st->status = ST_OK;
    } else if (1 >= st->kmax) {
      st->stop = 1;
      st->status = ST_ENOCONV;
    }
  }
}

// ------------------------------------------------------------ generation

// Raw block of iteration k (Algorithms 1-4, lines 3-11).
template <int W>
__global__ void __launch_bounds__(kThreads) k_generate(KP P, int gw) {
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  const int gen = st->gen;
  const bool half = (W != P.t);  // after the switch: [T^{t/2}(r)]
  const long long total = (long long)P.n * W;
  const BlockDesc* last = (st->nq > 0) ? &P.desc[st->nq - 1] : nullptr;
  const double* vprev = last ? last->V : nullptr;
  const double* pprev = last ? last->W : nullptr;
  const double* beta = P.small + kSmallBe;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / W);
    int j = (int)(e % W);
    double v;
    if (gen == GEN_SRE) {
      v = vprev[e];  // W_k = A W_{k-1}
    } else {
      int pj = half ? (P.part[i] >> 1) : P.part[i];
      v = (j == pj) ? P.r[i] : 0.0;
      if (gen == GEN_MSDO) v += pprev[e] * beta[j];
    }
    P.X[e] = v;
  }
}

// ------------------------------------------------------------------ CGS2

// Partial sums of C = [V_0 .. V_{nq-1}]^T B over this CTA's rows, for the 64
// window columns of chunk blockIdx.y.  B is n x WB (P.X).
template <int WB>
__global__ void __launch_bounds__(kThreads) k_tdot_window(KP P, int gw, const double* B) {
  constexpr int R = Tile<WB>::R;
  constexpr int EPT = (kChunk * WB + kThreads - 1) / kThreads;
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  const int nq = st->nq;
  if (nq <= 0) return;
  const BlockDesc* D = P.desc;
  const int wtot = D[nq - 1].off + D[nq - 1].w;
  const int c0 = blockIdx.y * kChunk;
  if (c0 >= wtot) return;
  const int ncol = min(kChunk, wtot - c0);
  __shared__ const double* cptr[kChunk];
  __shared__ int cstr[kChunk];
  extern __shared__ double smem[];
  double* sA = smem;             // R x kChunk
  double* sB = sA + R * kChunk;  // R x WB
  if (threadIdx.x < ncol) {
    int cg = c0 + threadIdx.x;
    int lo = 0, hi = nq - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (D[mid].off <= cg) lo = mid;
      else hi = mid - 1;
    }
    cptr[threadIdx.x] = D[lo].V + (cg - D[lo].off);
    cstr[threadIdx.x] = D[lo].w;
  }
  const int E = ncol * WB;
  double acc[EPT];
#pragma unroll
  for (int q = 0; q < EPT; q++) acc[q] = 0.0;
  int r0, r1;
  cta_rows(P.n, r0, r1);
  __syncthreads();
  for (int row0 = r0; row0 < r1; row0 += R) {
    const int nr = min(R, r1 - row0);
    for (int idx = threadIdx.x; idx < R * ncol; idx += blockDim.x) {
      int r = idx / ncol, cc = idx - r * ncol;
      sA[r * kChunk + cc] = (r < nr) ? cptr[cc][(long long)(row0 + r) * cstr[cc]] : 0.0;
    }
    for (int idx = threadIdx.x; idx < R * WB; idx += blockDim.x) {
      int r = idx / WB;
      sB[idx] = (r < nr) ? B[(long long)row0 * WB + idx] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < EPT; q++) {
      int e = threadIdx.x + q * kThreads;
      if (e < E) {
        int a = e / WB, bb = e - a * WB;
        double s = acc[q];
        for (int r = 0; r < nr; r++) s = fma(sA[r * kChunk + a], sB[r * WB + bb], s);
        acc[q] = s;
      }
    }
    __syncthreads();
  }
  double* out = P.part_buf + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * (kChunk * WB);
#pragma unroll
  for (int q = 0; q < EPT; q++) {
    int e = threadIdx.x + q * kThreads;
    if (e < E) out[e] = acc[q];
  }
}

// C[c0 + a][b] = sum over the gxw row-CTAs of the chunk partials (CTA order).
template <int WB>
__global__ void __launch_bounds__(kThreads) k_reduce_C(KP P, int gw, int gxw, double* Cout) {
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  const int nq = st->nq;
  if (nq <= 0) return;
  const int wtot = P.desc[nq - 1].off + P.desc[nq - 1].w;
  const int c0 = blockIdx.y * kChunk;
  if (c0 >= wtot) return;
  const int ncol = min(kChunk, wtot - c0);
  // one warp per entry, lanes over the row-CTAs, fixed shuffle tree
  const int lane = threadIdx.x & 31;
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e >= ncol * WB) return;
  const double* in = P.part_buf + (long long)blockIdx.y * gxw * (kChunk * WB) + e;
  double s = 0.0;
  for (int c = lane; c < gxw; c += 32) s += in[(long long)c * (kChunk * WB)];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) Cout[(long long)c0 * WB + e] = s;
}

// X -= [Q_0 .. Q_{nq-1}] C over the whole window (CGS update).
template <int W>
__global__ void __launch_bounds__(kThreads) k_update(KP P, int gw, double* Xio, const double* Cin) {
  constexpr int R = Tile<W>::R;
  constexpr int EPT = (R * W + kThreads - 1) / kThreads;
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  const int nq = st->nq;
  if (nq <= 0) return;
  const BlockDesc* D = P.desc;
  const int wtot = D[nq - 1].off + D[nq - 1].w;
  const int nch = (wtot + kChunk - 1) / kChunk;
  __shared__ const double* cptr[kChunk];
  __shared__ int cstr[kChunk];
  extern __shared__ double smem[];
  double* sQ = smem;                 // R x kChunk
  double* sC = sQ + R * kChunk;      // kChunk x W
  int r0, r1;
  cta_rows(P.n, r0, r1);
  for (int row0 = r0; row0 < r1; row0 += R) {
    const int nr = min(R, r1 - row0);
    double acc[EPT];
#pragma unroll
    for (int q = 0; q < EPT; q++) {
      int e = threadIdx.x + q * kThreads;
      int r = e / W;
      acc[q] = (e < R * W && r < nr) ? Xio[(long long)row0 * W + e] : 0.0;
    }
    for (int ch = 0; ch < nch; ch++) {
      const int c0 = ch * kChunk;
      const int ncol = min(kChunk, wtot - c0);
      __syncthreads();
      if (threadIdx.x < ncol) {
        int cg = c0 + threadIdx.x;
        int lo = 0, hi = nq - 1;
        while (lo < hi) {
          int mid = (lo + hi + 1) >> 1;
          if (D[mid].off <= cg) lo = mid;
          else hi = mid - 1;
        }
        cptr[threadIdx.x] = D[lo].W + (cg - D[lo].off);
        cstr[threadIdx.x] = D[lo].w;
      }
      for (int idx = threadIdx.x; idx < ncol * W; idx += blockDim.x)
        sC[idx] = Cin[(long long)c0 * W + idx];
      __syncthreads();
      for (int idx = threadIdx.x; idx < R * ncol; idx += blockDim.x) {
        int r = idx / ncol, cc = idx - r * ncol;
        sQ[r * kChunk + cc] = (r < nr) ? cptr[cc][(long long)(row0 + r) * cstr[cc]] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < EPT; q++) {
        int e = threadIdx.x + q * kThreads;
        if (e < R * W) {
          int r = e / W, bb = e - r * W;
          double s = acc[q];
          for (int a = 0; a < ncol; a++) s = fma(-sQ[r * kChunk + a], sC[a * W + bb], s);
          acc[q] = s;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < EPT; q++) {
      int e = threadIdx.x + q * kThreads;
      int r = e / W;
      if (e < R * W && r < nr) Xio[(long long)row0 * W + e] = acc[q];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------- orthonormalisation

// Partial upper-triangle Gram X^T X (Euclidean step of Pre-CholQR).
template <int W>
__global__ void __launch_bounds__(kThreads) k_gram_self(KP P, int gw, const double* Xin) {
  constexpr int R = Tile<W>::R;
  constexpr int E = W * (W + 1) / 2;
  constexpr int EPT = (E + kThreads - 1) / kThreads;
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  __shared__ double sB[R * W];
  int ea[EPT], eb[EPT];
#pragma unroll
  for (int q = 0; q < EPT; q++) {
    int e = threadIdx.x + q * kThreads;
    if (e < E) upper_ab(e, W, ea[q], eb[q]);
    else ea[q] = eb[q] = 0;
  }
  double acc[EPT];
#pragma unroll
  for (int q = 0; q < EPT; q++) acc[q] = 0.0;
  int r0, r1;
  cta_rows(P.n, r0, r1);
  for (int row0 = r0; row0 < r1; row0 += R) {
    const int nr = min(R, r1 - row0);
    for (int idx = threadIdx.x; idx < R * W; idx += blockDim.x)
      sB[idx] = (idx / W < nr) ? Xin[(long long)row0 * W + idx] : 0.0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < EPT; q++) {
      if (threadIdx.x + q * kThreads < E) {
        double s = acc[q];
        for (int r = 0; r < nr; r++) s = fma(sB[r * W + ea[q]], sB[r * W + eb[q]], s);
        acc[q] = s;
      }
    }
    __syncthreads();
  }
  double* out = P.part_buf + (long long)blockIdx.x * E;
#pragma unroll
  for (int q = 0; q < EPT; q++) {
    int e = threadIdx.x + q * kThreads;
    if (e < E) out[e] = acc[q];
  }
}

// Cholesky G = R^T R of the W x W matrix in sG (full symmetric storage) into
// sR (upper), with the pivot test pivot <= 1e-14 * G_jj.  Returns false on
// breakdown.  sG is destroyed.  All threads of the CTA must call it.
template <int W>
__device__ bool cta_cholesky(double* sG, double* sR, double* sD, int* sflag) {
  for (int i = threadIdx.x; i < W * W; i += blockDim.x) sR[i] = 0.0;
  for (int i = threadIdx.x; i < W; i += blockDim.x) sD[i] = sG[i * W + i];
  if (threadIdx.x == 0) *sflag = 0;
  __syncthreads();
  for (int j = 0; j < W; j++) {
    if (threadIdx.x == 0) {
      double d = sG[j * W + j];
      if (!(d > kBreakdownRatio * sD[j]) || !isfinite(d)) *sflag = 1;
      else sR[j * W + j] = sqrt(d);
    }
    __syncthreads();
    if (*sflag) return false;
    const double rjj = sR[j * W + j];
    for (int i = j + 1 + threadIdx.x; i < W; i += blockDim.x) sR[j * W + i] = sG[j * W + i] / rjj;
    __syncthreads();
    const int m = W - j - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      int i = j + 1 + idx / m, l = j + 1 + idx % m;
      if (l >= i) sG[i * W + l] = fma(-sR[j * W + i], sR[j * W + l], sG[i * W + l]);
    }
    __syncthreads();
  }
  return true;
}

// Inverse of the upper-triangular sR into sRi (upper), one column per thread.
template <int W>
__device__ void cta_triu_inverse(const double* sR, double* sRi) {
  for (int i = threadIdx.x; i < W * W; i += blockDim.x) sRi[i] = 0.0;
  __syncthreads();
  if (threadIdx.x < W) {
    const int c = threadIdx.x;
    for (int i = c; i >= 0; i--) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int l = i + 1; l <= c; l++) s = fma(-sR[i * W + l], sRi[l * W + c], s);
      sRi[i * W + c] = s / sR[i * W + i];
    }
  }
  __syncthreads();
}

// Euclidean step of Pre-CholQR: reduce X^T X, factor, store R_e^{-1}.
template <int W>
__global__ void __launch_bounds__(kThreads) k_small_e(KP P, int gw, int gx) {
  constexpr int E = W * (W + 1) / 2;
  DevState* st = P.st;
  if (skip(st, gw)) return;
  extern __shared__ double smem[];
  double* sG = smem;
  double* sR = sG + W * W;
  double* sRi = sR + W * W;
  double* sD = sRi + W * W;
  __shared__ int sflag;
  cta_reduce_partials(P.part_buf, E, gx, E, [&](int e, double s) {
    int a, b;
    upper_ab(e, W, a, b);
    sG[a * W + b] = s;
    sG[b * W + a] = s;
  });
  __syncthreads();
  if (!cta_cholesky<W>(sG, sR, sD, &sflag)) {
    if (threadIdx.x == 0) {
      st->stop = 1;
      st->status = ST_EBREAKDOWN;
    }
    return;
  }
  cta_triu_inverse<W>(sR, sRi);
  for (int i = threadIdx.x; i < W * W; i += blockDim.x) P.small[kSmallRe + i] = sRi[i];
}

// Y = A X; with GRAM, per-CTA partials of G = q^T (A q) (upper) and
// g = q^T r, q = X R_e^{-1} when PRE (else q = X).
template <int W, bool GRAM, bool PRE>
__global__ void __launch_bounds__(kThreads) k_spmm_gram(KP P, int gw, const double* Xin, double* Yout) {
  constexpr int R = Tile<W>::R;
  constexpr int E = W * (W + 1) / 2;
  constexpr int EPT = (E + kThreads - 1) / kThreads;
  constexpr int EPT2 = (R * W + kThreads - 1) / kThreads;
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  extern __shared__ double smem[];
  double* sX = smem;              // R x W
  double* sY = sX + R * W;        // R x W
  double* sQ = sY + R * W;        // R x W (PRE)
  double* sV = sQ + R * W;        // R x W (PRE)
  double* sRe = sV + R * W;       // W x W (PRE)
  double* sr = sRe + W * W;       // R
  int ea[EPT], eb[EPT];
  double acc[EPT];
  double accg = 0.0;
  if (GRAM) {
#pragma unroll
    for (int q = 0; q < EPT; q++) {
      int e = threadIdx.x + q * kThreads;
      if (e < E) upper_ab(e, W, ea[q], eb[q]);
      else ea[q] = eb[q] = 0;
      acc[q] = 0.0;
    }
    if (PRE) {
      for (int i = threadIdx.x; i < W * W; i += blockDim.x) sRe[i] = P.small[kSmallRe + i];
    }
  }
  int r0, r1;
  cta_rows(P.n, r0, r1);
  for (int row0 = r0; row0 < r1; row0 += R) {
    const int nr = min(R, r1 - row0);
#pragma unroll
    for (int q = 0; q < EPT2; q++) {
      int idx = threadIdx.x + q * kThreads;
      if (idx < R * W) {
        int r = idx / W, bb = idx - r * W;
        double y = 0.0, xv = 0.0;
        if (r < nr) {
          const int i = row0 + r;
          const int pe = P.rowptr[i + 1];
          for (int p = P.rowptr[i]; p < pe; p++) y = fma(P.val[p], Xin[(long long)P.col[p] * W + bb], y);
          Yout[(long long)i * W + bb] = y;
          xv = Xin[(long long)i * W + bb];
        }
        sY[idx] = y;
        sX[idx] = xv;
      }
    }
    if (GRAM) {
      for (int r = threadIdx.x; r < R; r += blockDim.x) sr[r] = (r < nr) ? P.r[row0 + r] : 0.0;
      __syncthreads();
      const double* q_ = sX;
      const double* v_ = sY;
      if (PRE) {
        if (W == 1) {
          for (int r = threadIdx.x; r < R; r += blockDim.x) {
            sQ[r] = sX[r] * sRe[0];
            sV[r] = sY[r] * sRe[0];
          }
        } else {
          constexpr int H = (W > 1) ? W / 2 : 1;
          for (int idx = threadIdx.x; idx < R * H; idx += blockDim.x) {
            const int r = idx / H, bp = idx - r * H;
            double q1, q2, v1, v2;
            tri_pair2<W>(sX + r * W, sY + r * W, sRe, bp, q1, q2, v1, v2);
            sQ[r * W + bp] = q1;
            sQ[r * W + W - 1 - bp] = q2;
            sV[r * W + bp] = v1;
            sV[r * W + W - 1 - bp] = v2;
          }
        }
        __syncthreads();
        q_ = sQ;
        v_ = sV;
      }
      #pragma unroll
      for (int q = 0; q < EPT; q++) {
        if (threadIdx.x + q * kThreads < E) {
          double s = acc[q];
          for (int r = 0; r < nr; r++) s = fma(q_[r * W + ea[q]], v_[r * W + eb[q]], s);
          acc[q] = s;
        }
      }
      if (threadIdx.x < W) {
        double s = accg;
        for (int r = 0; r < nr; r++) s = fma(q_[r * W + threadIdx.x], sr[r], s);
        accg = s;
      }
      __syncthreads();
    }
  }
  if (GRAM) {
    double* out = P.part_buf + (long long)blockIdx.x * (E + W);
#pragma unroll
    for (int q = 0; q < EPT; q++) {
      int e = threadIdx.x + q * kThreads;
      if (e < E) out[e] = acc[q];
    }
    if (threadIdx.x < W) out[E + threadIdx.x] = accg;
  }
}

// A-CholQR step: reduce G and g, G = S^T S, R^{-1} = [R_e^{-1}] S^{-1},
// alpha = S^{-T} g (= W_k^T r_{k-1}).
template <int W, bool PRE>
__global__ void __launch_bounds__(kThreads) k_small_a(KP P, int gw, int gx) {
  constexpr int E = W * (W + 1) / 2;
  DevState* st = P.st;
  if (skip(st, gw)) return;
  extern __shared__ double smem[];
  double* sG = smem;
  double* sR = sG + W * W;
  double* sSi = sR + W * W;
  double* sD = sSi + W * W;
  double* sg = sD + W;
  __shared__ int sflag;
  cta_reduce_partials(P.part_buf, E + W, gx, E + W, [&](int e, double s) {
    if (e < E) {
      int a, b;
      upper_ab(e, W, a, b);
      sG[a * W + b] = s;
      sG[b * W + a] = s;
    } else {
      sg[e - E] = s;
    }
  });
  __syncthreads();
  if (!cta_cholesky<W>(sG, sR, sD, &sflag)) {
    if (threadIdx.x == 0) {
      st->stop = 1;
      st->status = ST_EBREAKDOWN;
    }
    return;
  }
  cta_triu_inverse<W>(sR, sSi);
  for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
    int a = e / W, b = e % W;
    double s = 0.0;
    if (a <= b) {
      if (PRE) {
        for (int l = a; l <= b; l++) s = fma(P.small[kSmallRe + a * W + l], sSi[l * W + b], s);
      } else {
        s = sSi[e];
      }
    }
    P.small[kSmallRi + e] = s;
  }
  if (threadIdx.x < W) {
    const int b = threadIdx.x;
    double s = 0.0;
    for (int a = 0; a <= b; a++) s = fma(sSi[a * W + b], sg[a], s);
    P.small[kSmallAl + b] = s;
  }
}

// W_k = X R^{-1}, V_k = Y R^{-1} (written to Wout / Vout), x += W_k alpha,
// r -= V_k alpha; per-CTA ||r_k||^2 and, for MSDO-CG, V_k^T r_k partials.
template <int W>
__global__ void __launch_bounds__(kThreads) k_final(KP P, int gw, const double* Xin, const double* Yin,
                                                     double* Wout, double* Vout, double* xio, double* rio) {
  constexpr int R = Tile<W>::R;
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  if (Wout == nullptr) {  // the solver's window slot
    const long long s = st->next_slot;
    Wout = P.slotW + s * P.slot_stride;
    Vout = P.slotV + s * P.slot_stride;
  }
  extern __shared__ double smem[];
  double* sX = smem;            // R x W
  double* sY = sX + R * W;      // R x W
  double* sWa = sY + R * W;     // R x W
  double* sVa = sWa + R * W;    // R x W
  double* sVk = sVa + R * W;    // R x W
  double* sRi = sVk + R * W;    // W x W
  double* sal = sRi + W * W;    // W
  double* srn = sal + W;        // R
  double* sbuf = srn + R;       // kThreads
  for (int i = threadIdx.x; i < W * W; i += blockDim.x) sRi[i] = P.small[kSmallRi + i];
  for (int i = threadIdx.x; i < W; i += blockDim.x) sal[i] = P.small[kSmallAl + i];
  double rho_acc = 0.0, beta_acc = 0.0;
  int r0, r1;
  cta_rows(P.n, r0, r1);
  for (int row0 = r0; row0 < r1; row0 += R) {
    const int nr = min(R, r1 - row0);
    for (int idx = threadIdx.x; idx < R * W; idx += blockDim.x) {
      bool in = idx / W < nr;
      sX[idx] = in ? Xin[(long long)row0 * W + idx] : 0.0;
      sY[idx] = in ? Yin[(long long)row0 * W + idx] : 0.0;
    }
    __syncthreads();
    if (W == 1) {
      for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const double wk = sX[r] * sRi[0], vk = sY[r] * sRi[0];
        if (r < nr) {
          Wout[row0 + r] = wk;
          Vout[row0 + r] = vk;
        }
        sWa[r] = wk * sal[0];
        sVa[r] = vk * sal[0];
        sVk[r] = vk;
      }
    } else {
      constexpr int H = (W > 1) ? W / 2 : 1;
      for (int idx = threadIdx.x; idx < R * H; idx += blockDim.x) {
        const int r = idx / H, bp = idx - r * H;
        double w1, w2, v1, v2;
        tri_pair2<W>(sX + r * W, sY + r * W, sRi, bp, w1, w2, v1, v2);
        const int b1 = bp, b2 = W - 1 - bp;
        if (r < nr) {
          const long long o = (long long)(row0 + r) * W;
          Wout[o + b1] = w1;
          Wout[o + b2] = w2;
          Vout[o + b1] = v1;
          Vout[o + b2] = v2;
        }
        sWa[r * W + b1] = w1 * sal[b1];
        sWa[r * W + b2] = w2 * sal[b2];
        sVa[r * W + b1] = v1 * sal[b1];
        sVa[r * W + b2] = v2 * sal[b2];
        sVk[r * W + b1] = v1;
        sVk[r * W + b2] = v2;
      }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      double rn = 0.0;
      if (r < nr) {
        double dx = 0.0, dr = 0.0;
        for (int bb = 0; bb < W; bb++) {
          dx += sWa[r * W + bb];
          dr += sVa[r * W + bb];
        }
        const int i = row0 + r;
        xio[i] += dx;
        rn = rio[i] - dr;
        rio[i] = rn;
        rho_acc = fma(rn, rn, rho_acc);
      }
      srn[r] = rn;
    }
    __syncthreads();
    if (P.want_beta && threadIdx.x < W) {
      double s = beta_acc;
      for (int r = 0; r < nr; r++) s = fma(sVk[r * W + threadIdx.x], srn[r], s);
      beta_acc = s;
    }
    __syncthreads();
  }
  double tot = block_sum(rho_acc, sbuf);
  if (threadIdx.x == 0) P.rho_part[blockIdx.x] = tot;
  if (P.want_beta && threadIdx.x < W) P.beta_part[(long long)blockIdx.x * 64 + threadIdx.x] = beta_acc;
}

// End of iteration k: rho_k, tol1, window push, stop and switch tests.
__global__ void k_finish(KP P, int gw, int gx) {
  __shared__ double sbuf[kThreads];
  DevState* st = P.st;
  if (skip(st, gw)) return;
  double s = 0.0;
  for (int c = threadIdx.x; c < gx; c += blockDim.x) s += P.rho_part[c];
  s = block_sum(s, sbuf);
  const int W = st->width;
  if (P.want_beta && threadIdx.x < W) {
    double bsum = 0.0;
    for (int c = 0; c < gx; c++) bsum += P.beta_part[(long long)c * 64 + threadIdx.x];
    P.small[kSmallBe + threadIdx.x] = -bsum;  // beta_{k+1} = -V_k^T r_k
  }
  if (threadIdx.x != 0) return;
  const int k = st->k;
  const double rho = sqrt(s);
  st->rho = rho;
  P.history[k] = rho;
  st->tol1 = fabs(rho - st->rho_prev) / st->rho0;
  st->rho_prev = rho;
  st->iters = k;
  // memory count: the window used this iteration plus the new block
  long long stored = W;
  for (int j = 0; j < st->nq; j++) stored += P.desc[j].w;
  if (stored > st->mem) st->mem = stored;
  // push (W_k, V_k), dropping the oldest block beyond the capacity
  BlockDesc nb;
  nb.slot = st->next_slot;
  nb.W = P.slotW + (long long)nb.slot * P.slot_stride;
  nb.V = P.slotV + (long long)nb.slot * P.slot_stride;
  nb.w = W;
  nb.pad = 0;
  if (st->nq < st->cap) {
    nb.off = (st->nq > 0) ? P.desc[st->nq - 1].off + P.desc[st->nq - 1].w : 0;
    P.desc[st->nq] = nb;
    st->nq++;
  } else {
    for (int j = 0; j + 1 < st->nq; j++) P.desc[j] = P.desc[j + 1];
    int off = 0;
    for (int j = 0; j + 1 < st->nq; j++) {
      P.desc[j].off = off;
      off += P.desc[j].w;
    }
    nb.off = off;
    P.desc[st->nq - 1] = nb;
  }
  st->next_slot = (st->nq < st->cap) ? st->nq : P.desc[0].slot;
  const int knext = k + 1;
  st->k = knext;
  if (!(rho > st->eps * st->rho0)) {
    st->stop = 1;
    st->status = ST_OK;
  } else if (knext >= st->kmax) {
    st->stop = 1;
    st->status = ST_ENOCONV;
  } else if (st->switch_tol > 0.0 && st->counter == 0 && st->tol1 < st->switch_tol) {
    st->gen = GEN_SPLIT;  // W_k = [T^{t/2}(r_{k-1})]
    st->width = W / 2;
    st->counter = 1;
    st->switch_it = k;
  } else {
    st->gen = (st->variant == 0) ? GEN_SRE : (st->variant == 1 ? GEN_MSDO : GEN_SPLIT);
  }
}

// rho = ||r|| from the per-CTA partials (step-level block update).
__global__ void k_rho_only(KP P, int gx) {
  __shared__ double sbuf[kThreads];
  double s = 0.0;
  for (int c = threadIdx.x; c < gx; c += blockDim.x) s += P.rho_part[c];
  s = block_sum(s, sbuf);
  if (threadIdx.x == 0) P.st->rho = sqrt(s);
}

// dst[i] = -src[i], i < w (beta = -V^T r for the step-level MSDO generator).
__global__ void k_neg_copy(const double* src, double* dst, int w) {
  if ((int)threadIdx.x < w) dst[threadIdx.x] = -src[threadIdx.x];
}

}  // namespace ecg
