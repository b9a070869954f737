// ecg_kernels.cuh -- sm_103a kernels of the enlarged CG iteration.
//
// Method: S. Moufawad, "Flexibly Enlarged Conjugate Gradient methods"
// (arXiv 2305.19013), Algorithms 1-5.  One iteration k is the kernel chain
//
//   [k_prec_solve (+ k_reduce_partials)]   block Jacobi preconditioned forms
//                   only (Section 3, Alg. 5): X = M^{-1} V_{k-1}, or
//                   z = M^{-1} r_{k-1} and the MSDO beta = -V_{k-1}^T z
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
// The block kernels are templates on the scalar type T of the n x t blocks,
// the vectors x, r, b and the matrix values: double for the FP64 method,
// float for the inner solves of the mixed-precision method.  Everything
// small stays FP64 in both: per-CTA partial sums, the t x t Gram matrices,
// their Cholesky factors and inverses, alpha, beta and the residual norms.
//
// GB300 has about 1.2 TFLOP/s of FP64 against 6.7 TB/s of HBM, so with
// T = double every n x t block pass is bound by FP64 FMA issue, not by
// memory.  The kernels therefore stage row tiles in shared memory and give
// each thread distinct output entries, so that every FMA issued is a useful
// one (symmetric Grams compute their upper triangle only).  With T = float
// the same passes are bound by HBM.  Reductions over rows are two-stage and
// fixed-order: each CTA writes its partial sums and a second kernel adds
// them in CTA order, so repeated solves are bitwise identical.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ecg {

constexpr int kThreads = 256;
constexpr int kChunk = 64;  // window columns per CGS chunk

enum Gen { GEN_SPLIT = 0, GEN_SRE = 1, GEN_MSDO = 2 };
enum Status { ST_OK = 0, ST_ENOCONV = 1, ST_ECUDA = -3, ST_EBREAKDOWN = -4 };

struct BlockDesc {
  void* W;  // A-orthonormal block W_j (n x w, scalar type of the solve)
  void* V;  // A W_j (n x w)
  int w;    // width
  int off;  // first column of this block in the concatenated window
  int slot; // storage slot index
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
  int hist_off;   // history index of rho_0 for this solve
  int restarts;   // restarts performed (Section 3)
  int restart_every;      // j >= 2: restart at k with k mod j == 1 (0: off)
  int restart_max;        // restarts allowed by restart_tol (0: unlimited)
  int restart_at_switch;  // 1: the flexible switch also restarts
  int fault;              // 1: a bounded wait on a bulk copy ran out
  int stag_iters;         // > 0: end the solve when rho_k has not fallen below
                          // 0.99 rho_best for this many iterations (the FP32
                          // rounds of mixed precision; the refinement goes on)
  int best_k;             // iteration of rho_best
  double restart_tol;     // > 0: restart when rtol1 < restart_tol
  double rho_cycle;       // residual norm at the start of the current cycle
  double rtol1;           // |rho_k - rho_{k-1}| / rho_cycle
  long long mem;  // largest number of stored basis vectors
  double eps, switch_tol;
  double breakdown_ratio;  // Cholesky pivot test: pivot > ratio * diagonal
  double rho0, rho_prev, tol1, rho;
  double rho_best;        // smallest rho_k so far, up to 1% (stag_iters)
};

// Offsets of the small matrices inside KP::small (t <= 64).
constexpr int kSmallG = 0;                 // reduced Gram (upper) / scratch
constexpr int kSmallRe = kSmallG + 4096;   // R_e^{-1}
constexpr int kSmallRi = kSmallRe + 4096;  // R^{-1} = R_e^{-1} S^{-1}
constexpr int kSmallAl = kSmallRi + 4096;  // alpha
constexpr int kSmallBe = kSmallAl + 64;    // beta
constexpr int kSmallAb = kSmallBe + 64;    // block-residual alpha (t x t)
constexpr int kSmallSize = kSmallAb + 4096;

struct KP {
  int n, t;
  const int* rowptr;
  const int* col;
  const double* val;   // matrix values, FP64
  const float* valf;   // matrix values rounded to FP32 (mixed precision)
  const int* part;
  void* X;  // raw block of the iteration (n x W)
  void* Y;  // A X (n x W)
  void* x;
  void* r;
  const void* b;
  DevState* st;
  BlockDesc* desc;   // window, oldest first
  void* slotW;       // window storage, slot s at slotW + s * slot_stride elements
  void* slotV;
  long long slot_stride;
  double* C;         // CGS coefficients, (window columns) x W
  double* part_buf;  // per-CTA partial sums
  double* small;     // small matrices, see kSmall*
  double* history;   // rho_k at history[hist_off + k]
  double* rho_part;  // per-CTA partial ||r||^2
  double* beta_part; // per-CTA partial V^T r (64 per CTA)
  int want_beta;     // accumulate beta partials in k_final (MSDO-CG)
  int prec;          // 1: block Jacobi preconditioned generators (z = M^{-1} r)
  void* z;           // M^{-1} r_{k-1} (n), written by k_prec_solve
  int block;         // 1: block-residual mode (k_final leaves x, r alone)
  double* Rb;        // block residual R_k (n x t), block-residual mode
  int wcap;          // most window columns a CGS chunk can hold (<= kChunk);
                     // the CGS kernels' shared memory is sized by it
  int sre_src;       // 1: an SRE block is read from V_{k-1} where it is
                     // used (k_generate skips the copy into X, the first
                     // CGS pass reads V_{k-1} and writes X)
};

// Block Jacobi preconditioner M = L L^T, L = diag(L_1 .. L_nb), L_i the
// IC(0) factor of the diagonal block of A on the rows of block i.  Rows
// keep their global numbering; inside a block they are taken in increasing
// order, so L's entries in row i are the columns j < i of A's row i that
// belong to the same block.  The substitutions run level by level: a row's
// forward level is one more than the largest level of the rows its L entries
// reference, its backward level likewise over the entries of L^T.
//
// Each substitution is stored in level order ("positions" q): position q
// holds row rows[q], its cnt[q] <= K off-diagonal entries at col/val[q*K ..]
// (ELL, padded) and the reciprocal pivot diag[q] = 1 / l_ii, so a row's data
// needs no indirection through the row index and no division.
struct PrecSweep {
  const int* blk;   // nb + 1: block b's levels are [blk[b], blk[b+1])
  const int* lev;   // level l's positions are [lev[l], lev[l+1])
  const int* rows;  // row of each position
  const int* cnt;   // entries of each position
  const int* col;   // q * K + k: column (global row) of entry k
  const void* val;  // q * K + k: value (T)
  const void* diag; // q: l_ii (T)
  const int* dep;   // q * K + k: index of entry k's row inside the previous
                    // level (level-local mode), else nullptr
  int K;
  // chunks of consecutive levels inside a block (chunked level-local
  // mode): chunk j starts at level cpos[j] and position cq[j] and ends where
  // chunk j + 1 starts; block b's chunks are [cblk[b], cblk[b+1])
  const int* cpos;
  const int* cq;
  const int* cblk;
};
struct PrecP {
  int nb;
  int local;         // 1: every entry references the previous level (both
                     // sweeps), whose values the solve keeps in shared memory
  int maxw;          // rows of the widest level (level-local mode)
  int qc;            // > 0: chunked level-local mode, at most qc positions
                     // (and kChunkLevels levels) per chunk
  PrecSweep f;       // forward: y = L^{-1} x, entries l_ij, j < i
  PrecSweep b;       // backward: z = L^{-T} y, entries l_ji, j > i
  double* part;      // nb x W partial -V_{k-1}^T z (MSDO-CG)
};

template <typename T>
__device__ __forceinline__ const T* values(const KP& P);
template <>
__device__ __forceinline__ const double* values<double>(const KP& P) {
  return P.val;
}
template <>
__device__ __forceinline__ const float* values<float>(const KP& P) {
  return P.valf;
}

// Sum over the rows of one CTA.  FP64 accumulates one FMA chain across all
// tiles.  FP32 sums each row tile in FP32 and adds the tile sums into an
// FP32 (hi, lo) pair with an exact two-sum, so the long accumulation over a
// CTA's rows loses no more than one FP32 rounding per tile.
template <typename T>
struct RowAcc;
template <>
struct RowAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ double begin() const { return s; }
  __device__ __forceinline__ void end(double v) { s = v; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct RowAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ float begin() const { return 0.f; }
  __device__ __forceinline__ void end(float v) {
    const float s = hi + v;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (v - bp);
    hi = s;
    lo += err;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ bool skip(const DevState* st, int w) {
  return st->stop != 0 || st->width != w;
}

template <int W>
struct Tile {
  // rows per shared-memory tile
  static constexpr int R = (W >= 64) ? 16 : 32;
};

// Rows per tile of the CGS coefficients: FP32 tiles are 128 rows, so that
// the per-tile waits and barriers are paid over enough rows to keep HBM
// busy (FP64 is bound by its FMA rate at 32 rows).
template <typename T, int WB>
struct TdotTile {
  static constexpr int R = (sizeof(T) == 4 && WB % 4 == 0) ? 128 : Tile<WB>::R;
};

// Rows per tile of the CGS update: FP32 threads own 2 rows x 4 columns, so
// a tile of 2048 / W rows (at most 128) occupies all 256 threads.
template <typename T, int W>
struct UpdTile {
  static constexpr int R = (sizeof(T) == 4) ? ((2048 / W) < 128 ? (2048 / W) : 128) : Tile<W>::R;
};
// Stages of the CGS update: two in both precisions.  FP64 is bound by its
// FMA rate; FP32 by shared-memory reads, and with two stages four CTAs fit
// an SM.
template <typename T>
struct UpdStages {
  static constexpr int S = 2;
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
template <typename T, int W>
__device__ __forceinline__ void tri_pair2(const T* x, const T* z, const T* U, int bp, T& x1, T& x2, T& z1,
                                          T& z2) {
  const int b1 = bp, b2 = W - 1 - bp;
  T sx1 = 0, sx2 = 0, sz1 = 0, sz2 = 0;
#pragma unroll 4
  for (int j = 0; j <= W; j++) {
    const bool first = (j <= b1);
    const int a = first ? j : j - b1 - 1;
    const T u = U[a * W + (first ? b1 : b2)];
    const T vx = fma(x[a], u, first ? sx1 : sx2);
    const T vz = fma(z[a], u, first ? sz1 : sz2);
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

// y = x U for one row x and an upper-triangular W x W matrix U, for the
// column pair (bp, W-1-bp), as in tri_pair2 for a single row.
template <typename T, int W>
__device__ __forceinline__ void tri_pair1(const T* x, const T* U, int bp, T& x1, T& x2) {
  const int b1 = bp, b2 = W - 1 - bp;
  T s1 = 0, s2 = 0;
#pragma unroll 4
  for (int j = 0; j <= W; j++) {
    const bool first = (j <= b1);
    const int a = first ? j : j - b1 - 1;
    const T v = fma(x[a], U[a * W + (first ? b1 : b2)], first ? s1 : s2);
    if (first) s1 = v;
    else s2 = v;
  }
  x1 = s1;
  x2 = s2;
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

// Sum of the per-CTA partials in[c * nent + e], c < count, into out[e], one
// warp per entry across as many CTAs as needed (lanes split c; each lane
// keeps 8 loads in flight; a fixed shuffle tree adds the lanes, so the result
// is the same on every run).  Turns the ~600-deep dependent load chain a
// single CTA would walk into a few memory round trips.
__device__ __forceinline__ double warp_sum_partials(const double* in, long long stride, int count, int lane) {
  double s = 0.0;
  for (int c0 = lane; c0 < count; c0 += 32 * 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const int c = c0 + 32 * u;
      v[u] = (c < count) ? in[(long long)c * stride] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; u++) s += v[u];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

__global__ void __launch_bounds__(kThreads) k_reduce_partials(const DevState* st, int gw, const double* in,
                                                               int count, int nent, double* out) {
  if (skip(st, gw)) return;
  const int lane = threadIdx.x & 31;
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e >= nent) return;
  const double s = warp_sum_partials(in + e, nent, count, lane);
  if (lane == 0) out[e] = s;
}


// ------------------------------------------------------ bulk tile pipeline
//
// A row tile of a row-major n x w block is one contiguous range, so one bulk
// copy (cp.async.bulk, executed by the TMA engine) moves a block's tile into
// shared memory.  Thread 0 issues the copies of the next S = Stages<T>::S tiles ahead;
// an mbarrier per stage counts the bytes that have landed, and every thread
// waits on it with a bounded number of polls (a wait that runs out marks
// DevState::fault, waits boundedly for the copies already issued, and the
// CTA returns).  Usable when each block row is a multiple of 16 bytes and
// every base is 16-byte aligned (FP64 w >= 2, FP32 w >= 4); otherwise the
// kernels fall back to loads through registers.
template <typename T>
struct Stages {
  // the FP64 kernels are FMA-bound and need little prefetch; the FP32 ones
  // are bound by HBM and keep three tiles in flight
  static constexpr int S = (sizeof(T) == 8) ? 2 : 3;
};
// a wait for one tile gives up after kWaitNs of wall time (the copies take
// microseconds) or kWaitPolls polls, whichever comes first
constexpr unsigned long long kWaitNs = 1000000000ull;
constexpr long long kWaitPolls = 1LL << 26;
constexpr int kMaxStreams = 16;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// dynamic shared memory of this launch (bytes)
__device__ __forceinline__ uint32_t dyn_smem_bytes() {
  uint32_t v;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
  return v;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

struct BulkStream {
  const unsigned char* base;  // block base address
  int row_bytes;              // bytes of one block row
  int dst_off;                // byte offset of this block's tile inside a stage
};

// The tiles [r0 + i R, min(r0 + (i+1) R, r1)) of up to kMaxStreams blocks.
// Every thread of the CTA makes the same add() calls, so ns and stage_bytes
// agree across the CTA; the stream table itself lives in shared memory and
// is written and read by thread 0 alone.
template <int S>
struct BulkTiles {
  BulkStream* st;        // kMaxStreams entries in shared memory
  int ns = 0;
  uint64_t* bar;         // S mbarriers
  unsigned char* stage;  // S stages of stage_bytes
  int stage_bytes = 0;
  int r0 = 0, r1 = 0, R = 0, ntiles = 0;

  __device__ bool add(const void* base, int row_bytes) {
    if (ns >= kMaxStreams || (row_bytes & 15) || (((uintptr_t)base) & 15)) return false;
    if (threadIdx.x == 0) {
      st[ns].base = (const unsigned char*)base;
      st[ns].row_bytes = row_bytes;
      st[ns].dst_off = stage_bytes;
    }
    stage_bytes += R * row_bytes;
    ns++;
    return true;
  }
  __device__ int rows(int i) const { return min(R, r1 - (r0 + i * R)); }
  // thread 0 only
  __device__ void issue(int i) {
    const int row0 = r0 + i * R, nr = rows(i), s = i % S;
    uint32_t tx = 0;
    for (int j = 0; j < ns; j++) tx += (uint32_t)(nr * st[j].row_bytes);
    mbar_expect_tx(&bar[s], tx);
    unsigned char* dst = stage + (long long)s * stage_bytes;
    for (int j = 0; j < ns; j++)
      bulk_g2s(dst + st[j].dst_off, st[j].base + (long long)row0 * st[j].row_bytes, (uint32_t)(nr * st[j].row_bytes),
               &bar[s]);
  }
  __device__ bool wait(int i) {
    const uint32_t parity = (uint32_t)((i / S) & 1);
    if (mbar_try_wait(&bar[i % S], parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long p = 0; p < kWaitPolls; p += 64) {
      for (int q = 0; q < 64; q++)
        if (mbar_try_wait(&bar[i % S], parity)) return true;
      if (global_ns() - t0 > kWaitNs) return false;
    }
    return false;
  }
  __device__ unsigned char* tile(int i) const { return stage + (long long)(i % S) * stage_bytes; }
  // all threads: barriers ready and the first S tiles in flight
  __device__ void start() {
    if (threadIdx.x == 0) {
      for (int s = 0; s < S; s++) mbar_init(&bar[s], 1);
      mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int i = 0; i < min(S, ntiles); i++) issue(i);
  }
  // thread 0, once every thread is done reading tile i (after a barrier):
  // refill its stage with tile i+S
  __device__ void refill(int i) {
    if (threadIdx.x == 0 && i + S < ntiles) {
      fence_proxy_async();
      issue(i + S);
    }
  }
  // all threads, after tile i was consumed
  __device__ void next(int i) {
    __syncthreads();
    refill(i);
  }
  // all threads: wait for tile i; false (uniform over the CTA) after a
  // bounded wait ran out, with the copies already issued drained (bounded)
  __device__ bool ready(int i, DevState* st_) {
    const bool ok = __syncthreads_and(wait(i));
    if (ok) return true;
    if (threadIdx.x == 0) {
      st_->fault = 1;
      st_->status = ST_ECUDA;
      st_->stop = 1;
      for (int j = i; j < min(i + S, ntiles); j++) wait(j);
    }
    __syncthreads();
    return false;
  }
};

// Dynamic shared memory of the tile kernels (bytes), for both the bulk-copy
// pipeline and the fallback through registers.
// The CGS kernels are sized by wcap, the most window columns a chunk can
// hold (min(kChunk, stored blocks x t)): k_tdot_window needs the bulk
// stages of wcap + W columns, FP32's row-slice sums (kThreads x 16
// doubles) and the register path's R x (kChunk + W) tile; k_update needs
// wcap x W coefficients and then the bulk stages or the register path's
// R x wcap tile.
template <typename T, int W>
constexpr size_t smem_tdot(int wcap = kChunk) {
  constexpr size_t R = TdotTile<T, W>::R;
  const size_t bulk = sizeof(T) * Stages<T>::S * R * (size_t)(wcap + W);
  const size_t red = sizeof(T) == 4 ? (size_t)kThreads * 16 * 8 : 0;
  const size_t reg = sizeof(T) * R * (kChunk + W);
  const size_t m = bulk > red ? bulk : red;
  return 64 + (m > reg ? m : reg);
}
template <typename T, int W>
constexpr size_t smem_update(int wcap = kChunk) {
  constexpr size_t R = UpdTile<T, W>::R;
  const size_t cc = (size_t)(wcap < kChunk ? wcap : kChunk);
  const size_t coef = (sizeof(T) * cc * W + 15) & ~(size_t)15;
  const size_t bulk = 64 + sizeof(T) * UpdStages<T>::S * R * (cc + W);
  const size_t reg = sizeof(T) * R * cc;
  return coef + (bulk > reg ? bulk : reg);
}
template <typename T, int W>
constexpr size_t smem_gram_self() {
  // FP32 (W 4, 8, 16): kThreads-row stages, then 16 x kThreads doubles
  if constexpr (sizeof(T) == 4 && (W == 4 || W == 8 || W == 16)) {
    constexpr size_t st = sizeof(float) * Stages<float>::S * kThreads * W, red = sizeof(double) * 16 * kThreads;
    return 64 + (st > red ? st : red);
  }
  return 64 + sizeof(T) * Stages<T>::S * Tile<W>::R * W;
}
template <typename T, int W>
constexpr size_t smem_final_scalar() {
  return sizeof(double) * kThreads + 64 +
         sizeof(T) * ((2 * Stages<T>::S + 3) * Tile<W>::R * W + W * W + W + Tile<W>::R);
}
constexpr int kFinStages = 2;  // stages of the FP32 row-per-thread k_final
template <int W>
constexpr size_t smem_final_f32() {
  return sizeof(double) * kThreads + 64 + sizeof(float) * ((size_t)kFinStages * 2 * kThreads * W + W * W + W) +
         sizeof(float) * kThreads + sizeof(double) * kThreads;
}
template <typename T, int W>
constexpr size_t smem_final() {
  return (sizeof(T) == 4 && (W == 4 || W == 8 || W == 16) && smem_final_f32<W>() > smem_final_scalar<T, W>())
             ? smem_final_f32<W>()
             : smem_final_scalar<T, W>();
}

// Row ranges aligned to the tile height, so that all but the last tile of
// the last CTA are full.
__device__ __forceinline__ void cta_rows_aligned(int n, int R, int& r0, int& r1) {
  long long per = ((long long)n + gridDim.x - 1) / gridDim.x;
  per = ((per + R - 1) / R) * R;
  long long b = per * blockIdx.x;
  long long e = b + per;
  r0 = (int)(b < n ? b : n);
  r1 = (int)(e < n ? e : n);
}

// ----------------------------------------------------------------- setup

// r = b - A x (or r = b when x is null); per-CTA partial ||r||^2 and ||b||^2
// (each row's square in FP64).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_residual(KP P, const T* x, T* rout, const T* b, double* part_rr,
                                                        double* part_bb) {
  __shared__ double sbuf[kThreads];
  const T* val = values<T>(P);
  int r0, r1;
  cta_rows(P.n, r0, r1);
  double rr = 0.0, bb = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    T y = 0;
    if (x) {
      for (int p = P.rowptr[i]; p < P.rowptr[i + 1]; p++) y += val[p] * x[P.col[p]];
    }
    const T bi = b[i];
    const T ri = bi - y;
    if (rout) rout[i] = ri;
    rr += (double)ri * (double)ri;
    bb += (double)bi * (double)bi;
  }
  rr = block_sum(rr, sbuf);
  bb = block_sum(bb, sbuf);
  if (threadIdx.x == 0) {
    part_rr[blockIdx.x] = rr;
    if (part_bb) part_bb[blockIdx.x] = bb;
  }
}

// Algorithm 1 line 1: rho_0 and the loop state for k = 1.
// With part_bb (the stopping rule rho_k <= tol ||b||) the tolerance is
// rescaled to the test rho_k <= eps rho_0 the loop uses.
__global__ void k_start(KP P, int nparts, const double* part_bb) {
  __shared__ double sbuf[kThreads];
  double s = 0.0, sb = 0.0;
  for (int c = threadIdx.x; c < nparts; c += blockDim.x) {
    s += P.rho_part[c];
    if (part_bb) sb += part_bb[c];
  }
  s = block_sum(s, sbuf);
  if (part_bb) sb = block_sum(sb, sbuf);
  if (threadIdx.x == 0) {
    DevState* st = P.st;
    double rho0 = sqrt(s);
    if (part_bb && rho0 > 0.0) st->eps = st->eps * sqrt(sb) / rho0;
    st->rho0 = rho0;
    st->rho_prev = rho0;
    st->rho = rho0;
    st->tol1 = 1.0;
    st->rtol1 = 1.0;
    st->rho_cycle = rho0;
    st->k = 1;
    st->width = st->t;
    st->gen = GEN_SPLIT;
    st->counter = 0;
    st->switch_it = 0;
    st->nq = 0;
    st->iters = 0;
    st->next_slot = 0;
    st->mem = 0;
    st->restarts = 0;
    st->stop = 0;
    st->status = ST_ENOCONV;
    P.history[st->hist_off] = rho0;
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
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) k_generate(KP P, int gw) {
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  const int gen = st->gen;
  const bool half = (W != P.t);  // after the switch: [T^{t/2}(r)]
  const long long total = (long long)P.n * W;
  const BlockDesc* last = (st->nq > 0) ? &P.desc[st->nq - 1] : nullptr;
  const T* vprev = last ? (const T*)last->V : nullptr;
  const T* pprev = last ? (const T*)last->W : nullptr;
  const double* beta = P.small + kSmallBe;
  // preconditioned: k_prec_solve wrote X = M^{-1} V_{k-1}, or z = M^{-1} r;
  // with sre_src the first CGS pass reads V_{k-1} itself
  if ((P.prec || P.sre_src) && gen == GEN_SRE) return;
  const T* r = (const T*)(P.prec ? P.z : P.r);
  T* X = (T*)P.X;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / W);
    int j = (int)(e % W);
    T v;
    if (gen == GEN_SRE) {
      v = vprev[e];  // W_k = A W_{k-1}
    } else {
      int pj = half ? (P.part[i] >> 1) : P.part[i];
      v = (j == pj) ? r[i] : T(0);
      if (gen == GEN_MSDO) v += pprev[e] * (T)beta[j];
    }
    X[e] = v;
  }
}

// ------------------------------------------------------------------ CGS2

// Partial sums of C = [V_0 .. V_{nq-1}]^T B over this CTA's rows, for the 64
// window columns of chunk blockIdx.y.  B is n x WB.
template <typename T, int WB>
__global__ void __launch_bounds__(kThreads) k_tdot_window(KP P, int gw, const T* B) {
  constexpr int R = TdotTile<T, WB>::R;
  constexpr int EPT = (kChunk * WB + kThreads - 1) / kThreads;
  constexpr int S = Stages<T>::S;
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  const int nq = st->nq;
  if (nq <= 0) return;
  const BlockDesc* D = P.desc;
  const int wtot = D[nq - 1].off + D[nq - 1].w;
  const int c0 = blockIdx.y * kChunk;
  if (c0 >= wtot) return;
  // the SRE block A W_{k-1} = V_{k-1}, not copied into X
  if (P.sre_src && !P.prec && st->gen == GEN_SRE) B = (const T*)D[nq - 1].V;
  const int ncol = min(kChunk, wtot - c0);
  __shared__ const T* cptr[kChunk];
  __shared__ int cstr[kChunk];
  __shared__ int cofs[kChunk];  // pipelined: element offset of (row 0, column) in a stage
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int E = ncol * WB;
  RowAcc<T> acc[EPT];
  // blocks of this chunk
  auto find = [&](int cg) {
    int lo = 0, hi = nq - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (D[mid].off <= cg) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  };
  const int jlo = find(c0), jhi = find(c0 + ncol - 1);
  __shared__ BulkStream sst[kMaxStreams];
  BulkTiles<S> bt;
  bt.st = sst;
  bt.bar = (uint64_t*)smem_raw;
  bt.stage = smem_raw + 64;
  bt.R = R;
  int span = 0;
  bool bulk = (jhi - jlo + 2 <= kMaxStreams);
  for (int j = jlo; j <= jhi && bulk; j++) {
    span += D[j].w;
    bulk = bt.add(D[j].V, D[j].w * (int)sizeof(T));
  }
  bulk = bulk && span <= kChunk && bt.add(B, WB * (int)sizeof(T));
  bulk = bulk && 64u + (uint32_t)S * (uint32_t)bt.stage_bytes <= dyn_smem_bytes();
  if (bulk) {
    cta_rows_aligned(P.n, R, bt.r0, bt.r1);
    bt.ntiles = (bt.r1 - bt.r0 + R - 1) / R;
    // block j's tile starts R * (D[j].off - D[jlo].off) elements into a stage
    if (threadIdx.x < ncol) {
      const int cg = c0 + threadIdx.x;
      const int j = find(cg);
      cofs[threadIdx.x] = R * (D[j].off - D[jlo].off) + (cg - D[j].off);
      cstr[threadIdx.x] = D[j].w;
    }
    const int bofs = R * span;
    if constexpr (sizeof(T) == 4 && WB % 4 == 0) {
      // FP32: each thread owns a 4 x 4 block of C and a slice of every
      // tile's rows, reading 4 + 4 values (two 16-byte loads) per 16 FMAs;
      // the slices are summed in shared memory at the end.  Needs every
      // block width and the chunk a multiple of 4.
      constexpr int BB = WB / 4;
      bool w4 = (ncol % 4 == 0);
      // widths multiple of 4 make every offset one too, so a thread's four
      // columns lie in one block and start on a 16-byte boundary
      for (int j = jlo; j <= jhi; j++) w4 = w4 && (D[j].w % 4 == 0);
      const int EB = (ncol / 4) * BB;
      if (w4 && EB <= kThreads && 64u + kThreads * 16u * 8u <= dyn_smem_bytes()) {
        const int RS = kThreads / EB;
        const int eb = threadIdx.x % EB, rs = threadIdx.x / EB;
        const bool active = rs < RS;
        const int a0 = (eb / BB) * 4, b0 = (eb % BB) * 4;
        RowAcc<float> ra[16];
        bt.start();
        for (int i = 0; i < bt.ntiles; i++) {
          if (!bt.ready(i, (DevState*)st)) return;
          const float* stg = (const float*)bt.tile(i);
          const int nr = bt.rows(i);
          if (active) {
            const float* sa = stg + cofs[a0];
            const int sd = cstr[a0];
            const float* sB = stg + bofs + b0;
            float sv[16];
#pragma unroll
            for (int k = 0; k < 16; k++) sv[k] = 0.f;
            for (int r = rs; r < nr; r += RS) {
              const float4 av = *reinterpret_cast<const float4*>(sa + r * sd);
              const float4 bv = *reinterpret_cast<const float4*>(sB + r * WB);
              const float ax[4] = {av.x, av.y, av.z, av.w}, bx[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
              for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 4; v++) sv[u * 4 + v] = fmaf(ax[u], bx[v], sv[u * 4 + v]);
            }
#pragma unroll
            for (int k = 0; k < 16; k++) ra[k].end(sv[k]);
          }
          bt.next(i);
        }
        // sum the row slices (the stages are free now)
        double* red = reinterpret_cast<double*>(smem_raw + 64);
        __syncthreads();
        if (active)
#pragma unroll
          for (int k = 0; k < 16; k++) red[(rs * EB + eb) * 16 + k] = ra[k].value();
        __syncthreads();
        double* out = P.part_buf + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * (kChunk * WB);
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
          const int a = e / WB, b = e - a * WB;
          const int ebe = (a / 4) * BB + b / 4, k = (a % 4) * 4 + (b % 4);
          double sum = 0.0;
          for (int q = 0; q < RS; q++) sum += red[(q * EB + ebe) * 16 + k];
          out[e] = sum;
        }
        return;
      }
    }
    bt.start();  // includes a __syncthreads, so cofs/cstr are visible
    for (int i = 0; i < bt.ntiles; i++) {
      if (!bt.ready(i, (DevState*)st)) return;
      const T* stg = (const T*)bt.tile(i);
      const int nr = bt.rows(i);
      const T* sB = stg + bofs;
#pragma unroll
      for (int q = 0; q < EPT; q++) {
        int e = threadIdx.x + q * kThreads;
        if (e < E) {
          const int a = e / WB, bb = e - a * WB;
          const T* sa = stg + cofs[a];
          const int sd = cstr[a];
          T s = acc[q].begin();
          for (int r = 0; r < nr; r++) s = fma(sa[r * sd], sB[r * WB + bb], s);
          acc[q].end(s);
        }
      }
      bt.next(i);
    }
  } else {
    T* sA = (T*)smem_raw;          // R x kChunk
    T* sBt = sA + R * kChunk;      // R x WB
    if (threadIdx.x < ncol) {
      int cg = c0 + threadIdx.x;
      int lo = find(cg);
      cptr[threadIdx.x] = (const T*)D[lo].V + (cg - D[lo].off);
      cstr[threadIdx.x] = D[lo].w;
    }
    int r0, r1;
    cta_rows(P.n, r0, r1);
    __syncthreads();
    for (int row0 = r0; row0 < r1; row0 += R) {
      const int nr = min(R, r1 - row0);
      for (int idx = threadIdx.x; idx < R * ncol; idx += blockDim.x) {
        int r = idx / ncol, cc = idx - r * ncol;
        sA[r * kChunk + cc] = (r < nr) ? cptr[cc][(long long)(row0 + r) * cstr[cc]] : T(0);
      }
      for (int idx = threadIdx.x; idx < R * WB; idx += blockDim.x) {
        int r = idx / WB;
        sBt[idx] = (r < nr) ? B[(long long)row0 * WB + idx] : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < EPT; q++) {
        int e = threadIdx.x + q * kThreads;
        if (e < E) {
          int a = e / WB, bb = e - a * WB;
          T s = acc[q].begin();
          for (int r = 0; r < nr; r++) s = fma(sA[r * kChunk + a], sBt[r * WB + bb], s);
          acc[q].end(s);
        }
      }
      __syncthreads();
    }
  }
  double* out = P.part_buf + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * (kChunk * WB);
#pragma unroll
  for (int q = 0; q < EPT; q++) {
    int e = threadIdx.x + q * kThreads;
    if (e < E) out[e] = acc[q].value();
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
  const double s = warp_sum_partials(in, kChunk * WB, gxw, lane);
  if (lane == 0) Cout[(long long)c0 * WB + e] = s;
}

// X -= [Q_0 .. Q_{nq-1}] C over the whole window (CGS update).  A window of
// at most kChunk columns (the truncated methods) takes the bulk-copy
// pipeline, the X tile riding in the same stage as the window's tiles.
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) k_update(KP P, int gw, T* Xio, const double* Cin) {
  constexpr int R = UpdTile<T, W>::R;
  constexpr int EPT = (R * W + kThreads - 1) / kThreads;
  constexpr int S = UpdStages<T>::S;
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  const int nq = st->nq;
  if (nq <= 0) return;
  const BlockDesc* D = P.desc;
  const int wtot = D[nq - 1].off + D[nq - 1].w;
  // the block is read from Xsrc and written to Xio: V_{k-1} on the first
  // pass of an SRE iteration whose generator skipped the copy, else X
  const T* Xsrc = (P.sre_src && !P.prec && st->gen == GEN_SRE) ? (const T*)D[nq - 1].V : Xio;
  // window columns per pass: the launch's shared memory holds ccap x W
  // coefficients and ccap window columns of a tile
  const int ccap = min(kChunk, P.wcap);
  const int nch = (wtot + ccap - 1) / ccap;
  __shared__ const T* cptr[kChunk];
  __shared__ int cstr[kChunk];
  __shared__ int cofs[kChunk];  // pipelined: element offset of (row 0, column) in a stage
  __shared__ BulkStream sst[kMaxStreams];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sC = (T*)smem_raw;  // ccap x W
  unsigned char* rest = smem_raw + ((sizeof(T) * ccap * W + 15) & ~(size_t)15);
  BulkTiles<S> bt;
  bt.st = sst;
  bt.bar = (uint64_t*)rest;
  bt.stage = rest + 64;
  bt.R = R;
  bool bulk = (nch == 1 && nq + 1 <= kMaxStreams);
  for (int j = 0; j < nq && bulk; j++) bulk = bt.add(D[j].W, D[j].w * (int)sizeof(T));
  bulk = bulk && bt.add(Xsrc, W * (int)sizeof(T));
  bulk = bulk && (uint32_t)(rest - smem_raw) + 64u + (uint32_t)S * (uint32_t)bt.stage_bytes <= dyn_smem_bytes();
  if (bulk) {
    if (threadIdx.x < wtot) {
      const int cg = threadIdx.x;
      int lo = 0, hi = nq - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (D[mid].off <= cg) lo = mid;
        else hi = mid - 1;
      }
      cofs[cg] = R * D[lo].off + (cg - D[lo].off);
      cstr[cg] = D[lo].w;
    }
    for (int idx = threadIdx.x; idx < wtot * W; idx += blockDim.x) sC[idx] = (T)Cin[idx];
    cta_rows_aligned(P.n, R, bt.r0, bt.r1);
    bt.ntiles = (bt.r1 - bt.r0 + R - 1) / R;
    const int xofs = R * wtot;
    if constexpr (sizeof(T) == 4 && W % 4 == 0) {
      // FP32: each thread owns 2 rows x 4 columns of the tile and reads, per
      // 4 window columns, 2 + 4 16-byte vectors for 32 FMAs.  Its rows are
      // rp and rp + R/2, so that the eight threads of a quarter-warp read
      // two consecutive rows (different bank groups).  Needs every block
      // width a multiple of 4.
      bool w4 = true;
      for (int j = 0; j < nq; j++) w4 = w4 && (D[j].w % 4 == 0);
      if (w4) {
        constexpr int CG = W / 4;
        const int cg = threadIdx.x % CG, rp = threadIdx.x / CG;
        constexpr int HALF = R / 2;
        const int b0 = cg * 4, rl0 = rp;
        const bool active = rp < HALF;
        bt.start();
        for (int i = 0; i < bt.ntiles; i++) {
          if (!bt.ready(i, (DevState*)st)) return;
          const float* stg = (const float*)bt.tile(i);
          const int row0 = bt.r0 + i * R, nr = bt.rows(i);
          float acc[2][4];
          if (active) {
#pragma unroll
            for (int u = 0; u < 2; u++) {
              const float4 xv = *reinterpret_cast<const float4*>(stg + xofs + (rl0 + u * HALF) * W + b0);
              acc[u][0] = xv.x;
              acc[u][1] = xv.y;
              acc[u][2] = xv.z;
              acc[u][3] = xv.w;
            }
            for (int a = 0; a < wtot; a += 4) {
              const float* qa = stg + cofs[a];
              const int sd = cstr[a];
              float4 qv[2];
#pragma unroll
              for (int u = 0; u < 2; u++) qv[u] = *reinterpret_cast<const float4*>(qa + (rl0 + u * HALF) * sd);
#pragma unroll
              for (int k = 0; k < 4; k++) {
                const float4 cv = *reinterpret_cast<const float4*>(&sC[(a + k) * W + b0]);
#pragma unroll
                for (int u = 0; u < 2; u++) {
                  const float q = (k == 0) ? qv[u].x : (k == 1) ? qv[u].y : (k == 2) ? qv[u].z : qv[u].w;
                  acc[u][0] = fmaf(-q, cv.x, acc[u][0]);
                  acc[u][1] = fmaf(-q, cv.y, acc[u][1]);
                  acc[u][2] = fmaf(-q, cv.z, acc[u][2]);
                  acc[u][3] = fmaf(-q, cv.w, acc[u][3]);
                }
              }
            }
          }
          __syncthreads();
          bt.refill(i);
          if (active)
#pragma unroll
            for (int u = 0; u < 2; u++)
              if (rl0 + u * HALF < nr)
                *reinterpret_cast<float4*>(&Xio[(long long)(row0 + rl0 + u * HALF) * W + b0]) =
                    make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
        }
        return;
      }
    }
    bt.start();
    for (int i = 0; i < bt.ntiles; i++) {
      if (!bt.ready(i, (DevState*)st)) return;
      const T* stg = (const T*)bt.tile(i);
      const int row0 = bt.r0 + i * R, nr = bt.rows(i);
      T acc[EPT];
#pragma unroll
      for (int q = 0; q < EPT; q++) {
        const int e = threadIdx.x + q * kThreads;
        if (e < R * W) {
          const int r = e / W, bb = e - r * W;
          T sacc = stg[xofs + e];
          for (int a = 0; a < wtot; a++) sacc = fma(-stg[cofs[a] + r * cstr[a]], sC[a * W + bb], sacc);
          acc[q] = sacc;
        }
      }
      __syncthreads();
      bt.refill(i);
#pragma unroll
      for (int q = 0; q < EPT; q++) {
        const int e = threadIdx.x + q * kThreads;
        if (e < R * W && e / W < nr) Xio[(long long)row0 * W + e] = acc[q];
      }
    }
    return;
  }
  T* sQ = (T*)rest;  // R x ccap
  int r0, r1;
  cta_rows(P.n, r0, r1);
  for (int row0 = r0; row0 < r1; row0 += R) {
    const int nr = min(R, r1 - row0);
    T acc[EPT];
#pragma unroll
    for (int q = 0; q < EPT; q++) {
      int e = threadIdx.x + q * kThreads;
      int r = e / W;
      acc[q] = (e < R * W && r < nr) ? Xsrc[(long long)row0 * W + e] : T(0);
    }
    for (int ch = 0; ch < nch; ch++) {
      const int c0 = ch * ccap;
      const int ncol = min(ccap, wtot - c0);
      __syncthreads();
      if (threadIdx.x < ncol) {
        int cg = c0 + threadIdx.x;
        int lo = 0, hi = nq - 1;
        while (lo < hi) {
          int mid = (lo + hi + 1) >> 1;
          if (D[mid].off <= cg) lo = mid;
          else hi = mid - 1;
        }
        cptr[threadIdx.x] = (const T*)D[lo].W + (cg - D[lo].off);
        cstr[threadIdx.x] = D[lo].w;
      }
      for (int idx = threadIdx.x; idx < ncol * W; idx += blockDim.x) sC[idx] = (T)Cin[(long long)c0 * W + idx];
      __syncthreads();
      for (int idx = threadIdx.x; idx < R * ncol; idx += blockDim.x) {
        int r = idx / ncol, cc = idx - r * ncol;
        sQ[r * ccap + cc] = (r < nr) ? cptr[cc][(long long)(row0 + r) * cstr[cc]] : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < EPT; q++) {
        int e = threadIdx.x + q * kThreads;
        if (e < R * W) {
          int r = e / W, bb = e - r * W;
          T s = acc[q];
          for (int a = 0; a < ncol; a++) s = fma(-sQ[r * ccap + a], sC[a * W + bb], s);
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

// ------------------------------------------- FP32 register-blocked forms
// FP32 spends two shared-memory reads per FMA in the scalar forms above, so
// its tile kernels are bound by those reads rather than by HBM.  For block
// widths 4, 8 and 16 the kernels below give each thread whole rows or 4 x 4
// blocks, with 16-byte shared-memory reads.

// FP32 block widths with a register-blocked spmm_gram / final.
template <typename T, int W>
struct F32Rows {
  static constexpr bool on = sizeof(T) == 4 && (W == 4 || W == 8 || W == 16);
};

// Row stride (floats) of the FP32 spmm_gram tiles: W columns plus one
// 16-byte chunk, which holds (r_i, 0, 0, 0) in the Y rows so that
// g = q^T r comes out of the same 4 x 4 blocks as G.  For W = 8 and 16 the
// stride is an odd number of 16-byte chunks, so that eight consecutive rows
// read at the same column land in eight different bank groups.
template <int W>
struct PadStride {
  static constexpr int SP = W + 4;
};

// u-th component of a float4 (u a compile-time constant after unrolling).
__device__ __forceinline__ float f4c(const float4& v, int u) {
  return u == 0 ? v.x : (u == 1 ? v.y : (u == 2 ? v.z : v.w));
}
__device__ __forceinline__ void f4fma(float4& acc, float a, const float4& b) {
  acc.x = fmaf(a, b.x, acc.x);
  acc.y = fmaf(a, b.y, acc.y);
  acc.z = fmaf(a, b.z, acc.z);
  acc.w = fmaf(a, b.w, acc.w);
}

// acc[c] = (x U)[4c .. 4c+3] for one row x (W floats, 16-byte aligned) and
// the upper-triangular W x W matrix U (row-major, zeros below the
// diagonal): chunk m of x meets only column chunks c >= m.
template <int W>
__device__ __forceinline__ void tri_row4(const float* x, const float* U, float4 (&acc)[W / 4]) {
  constexpr int C4 = W / 4;
#pragma unroll
  for (int c = 0; c < C4; c++) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int m = 0; m < C4; m++) {
    const float4 xa = *reinterpret_cast<const float4*>(x + 4 * m);
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const float xl = f4c(xa, u);
      const float4* Ul = reinterpret_cast<const float4*>(U + (4 * m + u) * W);
#pragma unroll
      for (int c = m; c < C4; c++) f4fma(acc[c], xl, Ul[c]);
    }
  }
}

// k_gram_self for FP32 and W in {4, 8, 16}: tiles of kThreads rows through
// the bulk-copy pipeline; each thread owns a 4 x 4 block (ab <= bb) of
// X^T X and a slice of every tile's rows (16-byte shared-memory reads, 16
// FMAs per pair), FP32 per tile and compensated across tiles.  The slices
// are summed in the freed stages at the end.  Returns false, before
// touching shared memory, when X is not 16-byte aligned.
template <int W>
__device__ __forceinline__ bool gram_self_f32(const KP& P, const DevState* st, const float* Xin) {
  constexpr int R = kThreads, C4 = W / 4, EU = C4 * (C4 + 1) / 2, RS = kThreads / EU, E = W * (W + 1) / 2;
  constexpr int S = Stages<float>::S;
  if (((uintptr_t)Xin & 15) != 0) return false;
  __shared__ BulkStream sst[kMaxStreams];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BulkTiles<S> bt;
  bt.st = sst;
  bt.bar = (uint64_t*)smem_raw;
  bt.stage = smem_raw + 64;
  bt.R = R;
  bt.add(Xin, W * (int)sizeof(float));
  cta_rows_aligned(P.n, R, bt.r0, bt.r1);
  bt.ntiles = (bt.r1 - bt.r0 + R - 1) / R;
  const int eb = threadIdx.x % EU, rs = threadIdx.x / EU;
  const bool active = rs < RS;
  int ab, bb;
  upper_ab(eb, C4, ab, bb);
  RowAcc<float> ra[16];
  bt.start();
  for (int i = 0; i < bt.ntiles; i++) {
    if (!bt.ready(i, (DevState*)st)) return true;
    const float4* t4 = reinterpret_cast<const float4*>(bt.tile(i));
    const int nr = bt.rows(i);
    if (active) {
      float sv[16];
#pragma unroll
      for (int k = 0; k < 16; k++) sv[k] = 0.f;
      for (int r = rs; r < nr; r += RS) {
        const float4 qa = t4[r * C4 + ab];
        const float4 qb = t4[r * C4 + bb];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const float qu = f4c(qa, u);
          sv[u * 4 + 0] = fmaf(qu, qb.x, sv[u * 4 + 0]);
          sv[u * 4 + 1] = fmaf(qu, qb.y, sv[u * 4 + 1]);
          sv[u * 4 + 2] = fmaf(qu, qb.z, sv[u * 4 + 2]);
          sv[u * 4 + 3] = fmaf(qu, qb.w, sv[u * 4 + 3]);
        }
      }
#pragma unroll
      for (int k = 0; k < 16; k++) ra[k].end(sv[k]);
    }
    bt.next(i);
  }
  double* red = reinterpret_cast<double*>(smem_raw + 64);  // [16][kThreads]
  __syncthreads();
  if (active)
#pragma unroll
    for (int k = 0; k < 16; k++) red[k * kThreads + threadIdx.x] = ra[k].value();
  __syncthreads();
  double* out = P.part_buf + (long long)blockIdx.x * E;
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    int a, b;
    upper_ab(e, W, a, b);
    const int ba = a / 4, bq = b / 4;
    const int ebe = ba * C4 - ba * (ba - 1) / 2 + (bq - ba), k = (a % 4) * 4 + (b % 4);
    double sum = 0.0;
    for (int q = 0; q < RS; q++) sum += red[k * kThreads + q * EU + ebe];
    out[e] = sum;
  }
  return true;
}

// Partial upper-triangle Gram X^T X (Euclidean step of Pre-CholQR).
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) k_gram_self(KP P, int gw, const T* Xin) {
  constexpr int R = Tile<W>::R;
  constexpr int E = W * (W + 1) / 2;
  constexpr int EPT = (E + kThreads - 1) / kThreads;
  constexpr int S = Stages<T>::S;
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  if constexpr (F32Rows<T, W>::on) {
    if (gram_self_f32<W>(P, st, (const float*)Xin)) return;
  }
  __shared__ BulkStream sst[kMaxStreams];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int ea[EPT], eb[EPT];
#pragma unroll
  for (int q = 0; q < EPT; q++) {
    int e = threadIdx.x + q * kThreads;
    if (e < E) upper_ab(e, W, ea[q], eb[q]);
    else ea[q] = eb[q] = 0;
  }
  RowAcc<T> acc[EPT];
  auto accumulate = [&](const T* sB, int nr) {
#pragma unroll
    for (int q = 0; q < EPT; q++) {
      if (threadIdx.x + q * kThreads < E) {
        T s = acc[q].begin();
        for (int r = 0; r < nr; r++) s = fma(sB[r * W + ea[q]], sB[r * W + eb[q]], s);
        acc[q].end(s);
      }
    }
  };
  BulkTiles<S> bt;
  bt.st = sst;
  bt.bar = (uint64_t*)smem_raw;
  bt.stage = smem_raw + 64;
  bt.R = R;
  if (bt.add(Xin, W * (int)sizeof(T))) {
    cta_rows_aligned(P.n, R, bt.r0, bt.r1);
    bt.ntiles = (bt.r1 - bt.r0 + R - 1) / R;
    bt.start();
    for (int i = 0; i < bt.ntiles; i++) {
      if (!bt.ready(i, (DevState*)st)) return;
      accumulate((const T*)bt.tile(i), bt.rows(i));
      bt.next(i);
    }
  } else {
    T* sB = (T*)smem_raw;  // R x W
    int r0, r1;
    cta_rows(P.n, r0, r1);
    for (int row0 = r0; row0 < r1; row0 += R) {
      const int nr = min(R, r1 - row0);
      for (int idx = threadIdx.x; idx < R * W; idx += blockDim.x)
        sB[idx] = (idx / W < nr) ? Xin[(long long)row0 * W + idx] : T(0);
      __syncthreads();
      accumulate(sB, nr);
      __syncthreads();
    }
  }
  double* out = P.part_buf + (long long)blockIdx.x * E;
#pragma unroll
  for (int q = 0; q < EPT; q++) {
    int e = threadIdx.x + q * kThreads;
    if (e < E) out[e] = acc[q].value();
  }
}

// 1/sqrt(d) for a positive normal d: an FP32 estimate refined by two steps
// of Newton's method for f(y) = y^{-2} - d, y <- y + y (1 - d y^2) / 2.
// Each step squares the relative error (about 1e-7 for the estimate), so
// two end at FP64 rounding.  On this GPU an FP64 square root and division
// are long chains of FP64 instructions, and the factorisations below are
// latency-bound on them.  Outside the FP32 exponent range the plain
// quotient is taken.
__device__ __forceinline__ double rsqrt_newton(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double y = (double)rsqrtf((float)d);
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const double e = fma(-d * y, y, 1.0);
    y = fma(0.5 * y, e, y);
  }
  return y;
}

// 1/d for a positive normal d: the hardware's FP32 reciprocal estimate of
// d's significand (relative error below 2^-22), rescaled by d's exponent
// with integer arithmetic, then one third-order Newton-Raphson step
// y <- y (1 + e + e^2), e = 1 - d y, which cubes the relative error.  Three
// dependent FP64 FMAs instead of a division: the pivots of the
// factorisation below form a serial chain of them.  Exponents at the ends
// of the range take the plain quotient.
__device__ __forceinline__ double recip_pos(double d) {
  const long long b = __double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e < 2 || e > 2044) return 1.0 / d;
  const uint32_t fb = (127u << 23) | (uint32_t)((b >> 29) & 0x7FFFFF);  // d's significand in [1, 2)
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(__uint_as_float(fb)));
  const uint32_t yb = __float_as_uint(yf);
  const long long ye = (long long)((yb >> 23) & 0xFF) - 127 + 1023 - (e - 1023);
  const double y0 = __longlong_as_double((ye << 52) | ((long long)(yb & 0x7FFFFF) << 29));
  const double r = fma(-d, y0, 1.0);
  const double p = fma(r, r, r);
  return fma(y0, p, y0);
}

// The breakdown test of a pivot: d > thr (thr = ratio x the original
// diagonal entry, >= 0) and d finite and positive.  Positive doubles order
// like their bit patterns, so the test is integer compares.
__device__ __forceinline__ bool pivot_ok(double d, double thr) {
  const long long b = __double_as_longlong(d), t = __double_as_longlong(thr);
  return b > 0 && b > t && ((b >> 52) & 0x7FF) != 0x7FF;
}

// R^{-1} for the Cholesky factor R (G = R^T R, R upper with positive
// diagonal) of the W x W Gram in sA (full symmetric storage; overwritten by
// R^{-1}, zeros below the diagonal), by way of G = L D L^T:
//   - right-looking LDL^T, one thread per upper-triangle entry; the thread
//     that finishes pivot j + 1 tests it (pivot <= ratio G_jj or not finite
//     is a breakdown, as in the Cholesky form) and forms 1/d_{j+1}, so each
//     column costs one barrier and no square root;
//   - M = L^{-1} by a column sweep (unit diagonal, no division);
//   - R = D^{1/2} L^T, so R^{-1} = M^T D^{-1/2}: (R^{-1})_kc = M_ck / sqrt(d_c).
// GB300 issues FP64 at a few instructions per SM and cycle with long
// latencies, and a Cholesky's chain of square roots and divisions made the
// t x t steps a visible part of an iteration; this form keeps three FP64
// FMAs per column on the chain.  sM: W x W scratch; sInv, sThr: W doubles.
// Needs kThreads threads, all of which must call it; returns false (the
// same on every thread) on breakdown.
template <int W>
__device__ bool cta_ldl_rinv(double* sA, double* sM, double* sInv, double* sThr, int* sflag, double ratio) {
  constexpr int E = W * (W + 1) / 2, EPT = (E + kThreads - 1) / kThreads;
  const int tid = threadIdx.x;
  int ei[EPT], ek[EPT];  // this thread's entries (i, k), i <= k
#pragma unroll
  for (int q = 0; q < EPT; q++) {
    const int e = tid + q * kThreads;
    if (e < E) upper_ab(e, W, ei[q], ek[q]);
    else ei[q] = ek[q] = -1;
  }
  for (int j = tid; j < W; j += kThreads) sThr[j] = ratio * sA[j * W + j];
  if (tid == 0) {
    *sflag = 0;
    const double d = sA[0];
    if (!pivot_ok(d, ratio * d)) *sflag = 1;
    else sInv[0] = recip_pos(d);
  }
  __syncthreads();
  if (*sflag) return false;
  for (int j = 0; j < W - 1; j++) {
    const double inv = sInv[j];
#pragma unroll
    for (int q = 0; q < EPT; q++) {
      const int i = ei[q], k = ek[q];
      if (i > j) {
        const double t = sA[j * W + i] * inv;
        const double v = fma(-t, sA[j * W + k], sA[i * W + k]);
        sA[i * W + k] = v;
        if (k == j + 1) {  // then i == j + 1: the next pivot
          if (!pivot_ok(v, sThr[j + 1])) *sflag = 1;
          else sInv[j + 1] = recip_pos(v);
        }
      }
    }
    __syncthreads();
  }
  if (*sflag) return false;  // a failed pivot only leaves later ones meaningless
  // L_ki = a_ik / d_i (i < k) into the upper part; M starts as -L
#pragma unroll
  for (int q = 0; q < EPT; q++) {
    const int i = ei[q], k = ek[q];
    if (i >= 0 && i < k) {
      const double l = sA[i * W + k] * sInv[i];
      sA[i * W + k] = l;
      sM[k * W + i] = -l;
    }
  }
  for (int j = tid; j < W; j += kThreads) sThr[j] = rsqrt_newton(sA[j * W + j]);
  __syncthreads();
  // M_ic -= L_ik M_kc for i > k > c: after step k, rows <= k + 1 are final
  for (int k = 1; k < W - 1; k++) {
#pragma unroll
    for (int q = 0; q < EPT; q++) {
      const int c = ei[q], i = ek[q];
      if (c >= 0 && i > k && k > c) sM[i * W + c] = fma(-sA[k * W + i], sM[k * W + c], sM[i * W + c]);
    }
    __syncthreads();
  }
  for (int e = tid; e < W * W; e += kThreads) {
    const int k = e / W, c = e % W;
    sA[e] = (k == c) ? sThr[c] : (k < c) ? sM[c * W + k] * sThr[c] : 0.0;
  }
  __syncthreads();
  return true;
}

// Euclidean step of Pre-CholQR: reduce X^T X, factor, store R_e^{-1}.
template <int W>
__global__ void __launch_bounds__(kThreads) k_small_e(KP P, int gw, int gx) {
  constexpr int E = W * (W + 1) / 2;
  DevState* st = P.st;
  if (skip(st, gw)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sG = (double*)smem_raw;
  double* sM = sG + W * W;
  double* sInv = sM + W * W;
  double* sThr = sInv + W;
  __shared__ int sflag;
  const double* red = P.small + kSmallG;  // X^T X reduced by k_reduce_partials
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    int a, b;
    upper_ab(e, W, a, b);
    const double s = red[e];
    sG[a * W + b] = s;
    sG[b * W + a] = s;
  }
  (void)gx;
  __syncthreads();
  if (!cta_ldl_rinv<W>(sG, sM, sInv, sThr, &sflag, st->breakdown_ratio)) {
    if (threadIdx.x == 0) {
      st->stop = 1;
      st->status = ST_EBREAKDOWN;
    }
    return;
  }
  for (int i = threadIdx.x; i < W * W; i += blockDim.x) P.small[kSmallRe + i] = sG[i];
}

// 4 x 4 blocks of the FP32 spmm_gram: the upper blocks (ab <= bb) of G and
// the column chunk C4 (r) for g.
template <int W>
struct GramBlocks {
  static constexpr int C4 = W / 4, EU = C4 * (C4 + 1) / 2, EB = EU + C4, RS = kThreads / EB;
};

// tri_row4 for two rows x and z against the same U (acc = x U, acz = z U):
// each 16-byte row of U is read once for both.
template <int W>
__device__ __forceinline__ void tri_row4_pair(const float* x, const float* z, const float* U, float4 (&acc)[W / 4],
                                              float4 (&acz)[W / 4]) {
  constexpr int C4 = W / 4;
#pragma unroll
  for (int c = 0; c < C4; c++) acc[c] = acz[c] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int m = 0; m < C4; m++) {
    const float4 xa = *reinterpret_cast<const float4*>(x + 4 * m);
    const float4 za = *reinterpret_cast<const float4*>(z + 4 * m);
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const float xl = f4c(xa, u), zl = f4c(za, u);
      const float4* Ul = reinterpret_cast<const float4*>(U + (4 * m + u) * W);
#pragma unroll
      for (int c = m; c < C4; c++) {
        const float4 uv = Ul[c];
        f4fma(acc[c], xl, uv);
        f4fma(acz[c], zl, uv);
      }
    }
  }
}

// Shared memory (bytes) of the FP32 spmm_gram: the X and Y tiles (padded
// rows), R_e^{-1}, and each thread's 16 FP64 running sums.
template <int W>
__host__ __device__ constexpr size_t smem_spmm_f32_tiles() {
  return sizeof(float) * (2 * kThreads * PadStride<W>::SP + W * W);
}
template <int W>
constexpr size_t smem_spmm_f32() {
  return smem_spmm_f32_tiles<W>() + sizeof(double) * 16 * kThreads;
}

// k_spmm_gram for FP32 and W in {4, 8, 16}.  Tiles of kThreads rows:
//  1. Y = A X four columns per item (float4 gathers of X), Y to global
//     memory and to shared memory with the tile's X rows and r;
//  2. PRE: q = X R_e^{-1}, v = Y R_e^{-1} in place, one thread per row;
//  3. each thread owns a 4 x 4 block of [q^T v | q^T r] (upper blocks of
//     G, and the r chunk) and a slice of the rows.  Per-tile sums are FP32,
//     added across tiles into FP64 running sums in shared memory ([16] x
//     [thread], so that a warp's accesses are consecutive).
// The row slices are summed at the end; the partials have
// the layout of the scalar form ([G upper | g] per CTA).  Returns false,
// before touching shared memory, when X or Y is not 16-byte aligned.
template <int W, bool PRE>
__device__ __forceinline__ bool spmm_gram_f32(const KP& P, const float* Xin, float* Yout) {
  constexpr int R = kThreads, C4 = W / 4, SP = PadStride<W>::SP;
  constexpr int EU = GramBlocks<W>::EU, EB = GramBlocks<W>::EB, RS = GramBlocks<W>::RS, E = W * (W + 1) / 2;
  constexpr int IT = R * C4 / kThreads;
  if ((((uintptr_t)Xin | (uintptr_t)Yout) & 15) != 0) return false;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sX = (float*)smem_raw;  // R x SP: X, then q
  float* sY = sX + R * SP;       // R x SP: [Y | r 0 0 0], then [v | r 0 0 0]
  float* sRe = sY + R * SP;      // W x W
  double* acc = (double*)(smem_raw + smem_spmm_f32_tiles<W>());  // 16 x kThreads
  const float* val = values<float>(P);
  const float* rvec = (const float*)P.r;
  const float4* X4 = reinterpret_cast<const float4*>(Xin);
  float4* Y4 = reinterpret_cast<float4*>(Yout);
  if (PRE)
    for (int i = threadIdx.x; i < W * W; i += blockDim.x) sRe[i] = (float)P.small[kSmallRe + i];
  const int eb = threadIdx.x % EB, rs = threadIdx.x / EB;
  const bool active = rs < RS;
  int ab, bb;
  if (eb < EU) {
    upper_ab(eb, C4, ab, bb);
  } else {
    ab = eb - EU;
    bb = C4;
  }
#pragma unroll
  for (int k = 0; k < 16; k++) acc[k * kThreads + threadIdx.x] = 0.0;
  int r0, r1;
  cta_rows(P.n, r0, r1);
  for (int row0 = r0; row0 < r1; row0 += R) {
    const int nr = min(R, r1 - row0);
    int pb[IT], pe[IT];
    float4 y[IT];
    int kmax = 0;
#pragma unroll
    for (int q = 0; q < IT; q++) {
      const int r = (threadIdx.x + q * kThreads) / C4;
      pb[q] = pe[q] = 0;
      if (r < nr) {
        pb[q] = P.rowptr[row0 + r];
        pe[q] = P.rowptr[row0 + r + 1];
      }
      kmax = max(kmax, pe[q] - pb[q]);
      y[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int k = 0; k < kmax; k++) {
#pragma unroll
      for (int q = 0; q < IT; q++) {
        const int p = pb[q] + k;
        if (p < pe[q]) {
          const int c = (threadIdx.x + q * kThreads) % C4;
          f4fma(y[q], val[p], X4[(long long)P.col[p] * C4 + c]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < IT; q++) {
      const int idx = threadIdx.x + q * kThreads, r = idx / C4, c = idx % C4;
      float4 xv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < nr) {
        const long long o = (long long)(row0 + r) * C4 + c;
        Y4[o] = y[q];
        xv = X4[o];
      }
      *reinterpret_cast<float4*>(sY + r * SP + 4 * c) = y[q];
      *reinterpret_cast<float4*>(sX + r * SP + 4 * c) = xv;
    }
    {
      const int r = threadIdx.x;
      *reinterpret_cast<float4*>(sY + r * SP + W) = make_float4((r < nr) ? rvec[row0 + r] : 0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    if (PRE) {
      const int r = threadIdx.x;
      if (r < nr) {
        float4 tq[C4], tv[C4];
        tri_row4_pair<W>(sX + r * SP, sY + r * SP, sRe, tq, tv);
#pragma unroll
        for (int c = 0; c < C4; c++) {
          *reinterpret_cast<float4*>(sX + r * SP + 4 * c) = tq[c];
          *reinterpret_cast<float4*>(sY + r * SP + 4 * c) = tv[c];
        }
      }
      __syncthreads();
    }
    if (active) {
      float sv[16];
#pragma unroll
      for (int k = 0; k < 16; k++) sv[k] = 0.f;
      for (int r = rs; r < nr; r += RS) {
        const float4 qa = *reinterpret_cast<const float4*>(sX + r * SP + 4 * ab);
        const float4 vb = *reinterpret_cast<const float4*>(sY + r * SP + 4 * bb);
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const float qu = f4c(qa, u);
          sv[u * 4 + 0] = fmaf(qu, vb.x, sv[u * 4 + 0]);
          sv[u * 4 + 1] = fmaf(qu, vb.y, sv[u * 4 + 1]);
          sv[u * 4 + 2] = fmaf(qu, vb.z, sv[u * 4 + 2]);
          sv[u * 4 + 3] = fmaf(qu, vb.w, sv[u * 4 + 3]);
        }
      }
#pragma unroll
      for (int k = 0; k < 16; k++) acc[k * kThreads + threadIdx.x] += (double)sv[k];
    }
    __syncthreads();
  }
  // sum the row slices: thread rs * EB + eb holds block eb of slice rs
  __syncthreads();
  double* out = P.part_buf + (long long)blockIdx.x * (E + W);
  for (int e = threadIdx.x; e < E + W; e += blockDim.x) {
    int ebe, k;
    if (e < E) {
      int a, b;
      upper_ab(e, W, a, b);
      const int ba = a / 4, bq = b / 4;
      ebe = ba * C4 - ba * (ba - 1) / 2 + (bq - ba);
      k = (a % 4) * 4 + (b % 4);
    } else {
      const int a = e - E;
      ebe = EU + a / 4;
      k = (a % 4) * 4;
    }
    double s = 0.0;
    for (int q = 0; q < RS; q++) s += acc[k * kThreads + q * EB + ebe];
    out[e] = s;
  }
  return true;
}

// Y = A X; with GRAM, per-CTA partials of G = q^T (A q) (upper) and
// g = q^T r, q = X R_e^{-1} when PRE (else q = X).  ROWS: the FP32
// register-blocked form (k_spmm_gram_rows), else the scalar one.
template <typename T, int W, bool GRAM, bool PRE, bool ROWS>
__device__ __forceinline__ void spmm_gram_body(const KP& P, int gw, const T* Xin, T* Yout) {
  constexpr int R = Tile<W>::R;
  constexpr int E = W * (W + 1) / 2;
  constexpr int EPT = (E + kThreads - 1) / kThreads;
  constexpr int EPT2 = (R * W + kThreads - 1) / kThreads;
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  if constexpr (ROWS) {
    if (spmm_gram_f32<W, PRE>(P, (const float*)Xin, (float*)Yout)) return;
  }
  const T* val = values<T>(P);
  const T* rvec = (const T*)P.r;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sX = (T*)smem_raw;           // R x W
  T* sY = sX + R * W;             // R x W
  T* sQ = sY + R * W;             // R x W (PRE)
  T* sV = sQ + R * W;             // R x W (PRE)
  T* sRe = sV + R * W;            // W x W (PRE)
  T* sr = sRe + W * W;            // R
  int ea[EPT], eb[EPT];
  RowAcc<T> acc[EPT];
  RowAcc<T> accg;
  if (GRAM) {
#pragma unroll
    for (int q = 0; q < EPT; q++) {
      int e = threadIdx.x + q * kThreads;
      if (e < E) upper_ab(e, W, ea[q], eb[q]);
      else ea[q] = eb[q] = 0;
    }
    if (PRE) {
      for (int i = threadIdx.x; i < W * W; i += blockDim.x) sRe[i] = (T)P.small[kSmallRe + i];
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
        T y = 0, xv = 0;
        if (r < nr) {
          const int i = row0 + r;
          const int pe = P.rowptr[i + 1];
          for (int p = P.rowptr[i]; p < pe; p++) y = fma(val[p], Xin[(long long)P.col[p] * W + bb], y);
          Yout[(long long)i * W + bb] = y;
          xv = Xin[(long long)i * W + bb];
        }
        sY[idx] = y;
        sX[idx] = xv;
      }
    }
    if (GRAM) {
      for (int r = threadIdx.x; r < R; r += blockDim.x) sr[r] = (r < nr) ? rvec[row0 + r] : T(0);
      __syncthreads();
      const T* q_ = sX;
      const T* v_ = sY;
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
            T q1, q2, v1, v2;
            tri_pair2<T, W>(sX + r * W, sY + r * W, sRe, bp, q1, q2, v1, v2);
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
          T s = acc[q].begin();
          for (int r = 0; r < nr; r++) s = fma(q_[r * W + ea[q]], v_[r * W + eb[q]], s);
          acc[q].end(s);
        }
      }
      if (threadIdx.x < W) {
        T s = accg.begin();
        for (int r = 0; r < nr; r++) s = fma(q_[r * W + threadIdx.x], sr[r], s);
        accg.end(s);
      }
      __syncthreads();
    }
  }
  if (GRAM) {
    double* out = P.part_buf + (long long)blockIdx.x * (E + W);
#pragma unroll
    for (int q = 0; q < EPT; q++) {
      int e = threadIdx.x + q * kThreads;
      if (e < E) out[e] = acc[q].value();
    }
    if (threadIdx.x < W) out[E + threadIdx.x] = accg.value();
  }
}

template <typename T, int W, bool GRAM, bool PRE>
__global__ void __launch_bounds__(kThreads) k_spmm_gram(KP P, int gw, const T* Xin, T* Yout) {
  spmm_gram_body<T, W, GRAM, PRE, false>(P, gw, Xin, Yout);
}

// The FP32 register-blocked form (W in {4, 8, 16}) at three CTAs per SM.
template <int W, bool PRE>
__global__ void __launch_bounds__(kThreads, 3) k_spmm_gram_rows(KP P, int gw, const float* Xin, float* Yout) {
  spmm_gram_body<float, W, true, PRE, true>(P, gw, Xin, Yout);
}

// A-CholQR step: reduce G and g, G = S^T S, R^{-1} = [R_e^{-1}] S^{-1},
// alpha = S^{-T} g (= W_k^T r_{k-1}).
template <int W, bool PRE>
__global__ void __launch_bounds__(kThreads) k_small_a(KP P, int gw, int gx) {
  constexpr int E = W * (W + 1) / 2;
  DevState* st = P.st;
  if (skip(st, gw)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sG = (double*)smem_raw;
  double* sM = sG + W * W;
  double* sInv = sM + W * W;
  double* sThr = sInv + W;
  double* sg = sThr + W;
  __shared__ int sflag;
  const double* red = P.small + kSmallG;  // [G upper | g] reduced by k_reduce_partials
  for (int e = threadIdx.x; e < E + W; e += blockDim.x) {
    const double s = red[e];
    if (e < E) {
      int a, b;
      upper_ab(e, W, a, b);
      sG[a * W + b] = s;
      sG[b * W + a] = s;
    } else {
      sg[e - E] = s;
    }
  }
  (void)gx;
  __syncthreads();
  if (!cta_ldl_rinv<W>(sG, sM, sInv, sThr, &sflag, st->breakdown_ratio)) {
    if (threadIdx.x == 0) {
      st->stop = 1;
      st->status = ST_EBREAKDOWN;
    }
    return;
  }
  // sG = S^{-1}; R^{-1} = R_e^{-1} S^{-1} (Pre-CholQR) or S^{-1}
  if (PRE) {
    for (int i = threadIdx.x; i < W * W; i += blockDim.x) sM[i] = P.small[kSmallRe + i];
    __syncthreads();
  }
  for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
    int a = e / W, b = e % W;
    double s = 0.0;
    if (a <= b) {
      if (PRE) {
        for (int l = a; l <= b; l++) s = fma(sM[a * W + l], sG[l * W + b], s);
      } else {
        s = sG[e];
      }
    }
    P.small[kSmallRi + e] = s;
  }
  if (threadIdx.x < W) {
    const int b = threadIdx.x;
    double s = 0.0;
    for (int a = 0; a <= b; a++) s = fma(sG[a * W + b], sg[a], s);
    P.small[kSmallAl + b] = s;
  }
}

// k_final for FP32 and W in {4, 8, 16}, one thread per row: the thread
// reads its rows of X and Y from the stage, forms W_k = X R^{-1} and
// V_k = Y R^{-1} in registers (R^{-1} read as broadcast 16-byte rows),
// stores both rows, and updates x and r with W_k alpha and V_k alpha.  For
// MSDO-CG, V_k replaces Y in the stage and the CTA sums V_k^T r_k over row
// slices.  Returns false, before touching shared memory, when the blocks do
// not suit the bulk copies; the caller then takes the scalar form.
template <int W>
__device__ __forceinline__ bool final_f32(const KP& P, const DevState* st, const float* Xin, const float* Yin,
                                          float* Wout, float* Vout, float* xio, float* rio) {
  constexpr int R = kThreads, C4 = W / 4, S = kFinStages, RSB = kThreads / W;
  if ((((uintptr_t)Xin | (uintptr_t)Yin | (uintptr_t)Wout | (uintptr_t)Vout) & 15) != 0) return false;
  __shared__ BulkStream sst[kMaxStreams];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sbuf = (double*)smem_raw;                        // kThreads
  uint64_t* sbar = (uint64_t*)(sbuf + kThreads);           // 64 bytes
  float* stg = (float*)((unsigned char*)sbar + 64);        // S stages of [R x W | R x W]
  float* sRi = stg + S * 2 * R * W;                        // W x W
  float* sal = sRi + W * W;                                // W
  float* srn = sal + W;                                    // R
  double* sbr = (double*)(srn + R);                        // RSB x W
  for (int i = threadIdx.x; i < W * W; i += blockDim.x) sRi[i] = (float)P.small[kSmallRi + i];
  for (int i = threadIdx.x; i < W; i += blockDim.x) sal[i] = P.block ? 0.f : (float)P.small[kSmallAl + i];
  BulkTiles<S> bt;
  bt.st = sst;
  bt.bar = sbar;
  bt.stage = (unsigned char*)stg;
  bt.R = R;
  bt.add(Xin, W * (int)sizeof(float));
  bt.add(Yin, W * (int)sizeof(float));
  cta_rows_aligned(P.n, R, bt.r0, bt.r1);
  bt.ntiles = (bt.r1 - bt.r0 + R - 1) / R;
  bt.start();  // its barrier also publishes sRi and sal
  double rho_acc = 0.0;
  RowAcc<float> beta_acc;
  const bool beta = P.want_beta != 0;
  const int bcol = threadIdx.x % W, bsl = threadIdx.x / W;
  for (int i = 0; i < bt.ntiles; i++) {
    if (!bt.ready(i, (DevState*)st)) return true;
    float* tX = (float*)bt.tile(i);
    float* tY = tX + R * W;
    const int nr = bt.rows(i), row0 = bt.r0 + i * R;
    const int r = threadIdx.x;
    float rn = 0.f;
    if (r < nr) {
      float4 w[C4], v[C4];
      tri_row4_pair<W>(tX + r * W, tY + r * W, sRi, w, v);
      const long long o = (long long)(row0 + r) * C4;
      float dx = 0.f, dr = 0.f;
#pragma unroll
      for (int c = 0; c < C4; c++) {
        reinterpret_cast<float4*>(Wout)[o + c] = w[c];
        reinterpret_cast<float4*>(Vout)[o + c] = v[c];
        const float4 al = *reinterpret_cast<const float4*>(sal + 4 * c);
        dx = fmaf(w[c].x, al.x, fmaf(w[c].y, al.y, fmaf(w[c].z, al.z, fmaf(w[c].w, al.w, dx))));
        dr = fmaf(v[c].x, al.x, fmaf(v[c].y, al.y, fmaf(v[c].z, al.z, fmaf(v[c].w, al.w, dr))));
      }
      const int gi = row0 + r;
      xio[gi] += dx;
      rn = rio[gi] - dr;
      rio[gi] = rn;
      rho_acc += (double)rn * (double)rn;
      if (beta) {
#pragma unroll
        for (int c = 0; c < C4; c++) *reinterpret_cast<float4*>(tY + r * W + 4 * c) = v[c];
      }
    }
    if (beta) {
      srn[r] = rn;
      fence_proxy_async();  // the stage is refilled by the async proxy next
      __syncthreads();
      float s = 0.f;
      for (int q = bsl; q < nr; q += RSB) s = fmaf(tY[q * W + bcol], srn[q], s);
      beta_acc.end(s);
    }
    bt.next(i);
  }
  const double tot = block_sum(rho_acc, sbuf);
  if (threadIdx.x == 0) P.rho_part[blockIdx.x] = tot;
  if (beta) {
    sbr[bsl * W + bcol] = beta_acc.value();
    __syncthreads();
    if (threadIdx.x < W) {
      double s = 0.0;
      for (int q = 0; q < RSB; q++) s += sbr[q * W + threadIdx.x];
      P.beta_part[(long long)blockIdx.x * 64 + threadIdx.x] = s;
    }
  }
  return true;
}

// W_k = X R^{-1}, V_k = Y R^{-1} (written to Wout / Vout), x += W_k alpha,
// r -= V_k alpha; per-CTA ||r_k||^2 and, for MSDO-CG, V_k^T r_k partials.
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) k_final(KP P, int gw, const T* Xin, const T* Yin, T* Wout, T* Vout,
                                                     T* xio, T* rio) {
  constexpr int R = Tile<W>::R;
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  if (Wout == nullptr) {  // the solver's window slot
    const long long s = st->next_slot;
    Wout = (T*)P.slotW + s * P.slot_stride;
    Vout = (T*)P.slotV + s * P.slot_stride;
  }
  if constexpr (F32Rows<T, W>::on) {
    if (final_f32<W>(P, st, (const float*)Xin, (const float*)Yin, (float*)Wout, (float*)Vout, (float*)xio,
                     (float*)rio))
      return;
  }
  constexpr int S = Stages<T>::S;
  __shared__ BulkStream sst[kMaxStreams];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sbuf = (double*)smem_raw;                       // kThreads
  uint64_t* sbar = (uint64_t*)(sbuf + kThreads);          // 64 bytes
  T* sX = (T*)((unsigned char*)sbar + 64);                // S stages of [R x W | R x W]
  T* sWa = sX + S * 2 * R * W;                            // R x W
  T* sVa = sWa + R * W;                                   // R x W
  T* sVk = sVa + R * W;                                   // R x W
  T* sRi = sVk + R * W;                                   // W x W
  T* sal = sRi + W * W;                                   // W
  T* srn = sal + W;                                       // R
  for (int i = threadIdx.x; i < W * W; i += blockDim.x) sRi[i] = (T)P.small[kSmallRi + i];
  // block-residual mode: x and r are updated by k_block_update instead
  for (int i = threadIdx.x; i < W; i += blockDim.x) sal[i] = P.block ? T(0) : (T)P.small[kSmallAl + i];
  double rho_acc = 0.0;
  RowAcc<T> beta_acc;
  BulkTiles<S> bt;
  bt.st = sst;
  bt.bar = sbar;
  bt.stage = (unsigned char*)sX;
  bt.R = R;
  const bool bulk = bt.add(Xin, W * (int)sizeof(T)) && bt.add(Yin, W * (int)sizeof(T));
  int r0, r1;
  if (bulk) {
    cta_rows_aligned(P.n, R, r0, r1);
    bt.r0 = r0;
    bt.r1 = r1;
    bt.ntiles = (r1 - r0 + R - 1) / R;
    bt.start();
  } else {
    cta_rows(P.n, r0, r1);
  }
  for (int i = 0, row0 = r0; row0 < r1; i++, row0 += R) {
    const int nr = min(R, r1 - row0);
    const T* tX = sX;
    const T* tY = sX + R * W;
    if (bulk) {
      if (!bt.ready(i, (DevState*)st)) return;
      tX = (const T*)bt.tile(i);
      tY = tX + R * W;
    } else {
      for (int idx = threadIdx.x; idx < R * W; idx += blockDim.x) {
        bool in = idx / W < nr;
        sX[idx] = in ? Xin[(long long)row0 * W + idx] : T(0);
        sX[R * W + idx] = in ? Yin[(long long)row0 * W + idx] : T(0);
      }
      __syncthreads();
    }
    if (W == 1) {
      for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const T wk = tX[r] * sRi[0], vk = tY[r] * sRi[0];
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
        T w1, w2, v1, v2;
        tri_pair2<T, W>(tX + r * W, tY + r * W, sRi, bp, w1, w2, v1, v2);
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
    if (bulk) bt.refill(i);  // tile i is no longer read
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      T rn = 0;
      if (r < nr) {
        T dx = 0, dr = 0;
        for (int bb = 0; bb < W; bb++) {
          dx += sWa[r * W + bb];
          dr += sVa[r * W + bb];
        }
        const int i = row0 + r;
        xio[i] += dx;
        rn = rio[i] - dr;
        rio[i] = rn;
        rho_acc += (double)rn * (double)rn;
      }
      srn[r] = rn;
    }
    __syncthreads();
    if (P.want_beta && threadIdx.x < W) {
      T s = beta_acc.begin();
      for (int r = 0; r < nr; r++) s = fma(sVk[r * W + threadIdx.x], srn[r], s);
      beta_acc.end(s);
    }
    __syncthreads();
  }
  double tot = block_sum(rho_acc, sbuf);
  if (threadIdx.x == 0) P.rho_part[blockIdx.x] = tot;
  if (P.want_beta && threadIdx.x < W) P.beta_part[(long long)blockIdx.x * 64 + threadIdx.x] = beta_acc.value();
}

// X <- X R_e^{-1} in place (R_e^{-1} upper, in P.small): the Euclidean half
// of Pre-CholQR made explicit, q = X R_e^{-1}, so that the SpMM that follows
// applies A to the orthonormalised block (Pre-CholQR's order: Q_e, then
// A Q_e) and the A-CholQR step needs no per-row transform.  One (row,
// column pair) per thread, W + 1 FMAs each; tiles of Tile<W>::R rows
// through the bulk-copy pipeline when X suits it.
template <typename T, int W>
__host__ __device__ constexpr size_t smem_tri_right() {
  return 64 + sizeof(T) * ((size_t)Stages<T>::S * Tile<W>::R * W + W * W);
}
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) k_tri_right(KP P, int gw, T* X) {
  constexpr int R = Tile<W>::R;
  constexpr int H = (W > 1) ? W / 2 : 1;
  constexpr int S = Stages<T>::S;
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  __shared__ BulkStream sst[kMaxStreams];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* sbar = (uint64_t*)smem_raw;  // 64 bytes
  T* sX = (T*)(smem_raw + 64);           // S stages of R x W (one tile on the register path)
  T* sU = sX + S * R * W;                // W x W
  for (int i = threadIdx.x; i < W * W; i += blockDim.x) sU[i] = (T)P.small[kSmallRe + i];
  BulkTiles<S> bt;
  bt.st = sst;
  bt.bar = sbar;
  bt.stage = (unsigned char*)sX;
  bt.R = R;
  const bool bulk = bt.add(X, W * (int)sizeof(T));
  int r0, r1;
  if (bulk) {
    cta_rows_aligned(P.n, R, r0, r1);
    bt.r0 = r0;
    bt.r1 = r1;
    bt.ntiles = (r1 - r0 + R - 1) / R;
    bt.start();  // its barrier also publishes sU
  } else {
    cta_rows(P.n, r0, r1);
  }
  for (int i = 0, row0 = r0; row0 < r1; i++, row0 += R) {
    const int nr = min(R, r1 - row0);
    const T* tX = sX;
    if (bulk) {
      if (!bt.ready(i, (DevState*)st)) return;
      tX = (const T*)bt.tile(i);
    } else {
      for (int idx = threadIdx.x; idx < R * W; idx += blockDim.x)
        sX[idx] = (idx / W < nr) ? X[(long long)row0 * W + idx] : T(0);
      __syncthreads();
    }
    for (int idx = threadIdx.x; idx < R * H; idx += blockDim.x) {
      const int r = idx / H, bp = idx - r * H;
      if (r < nr) {
        const long long o = (long long)(row0 + r) * W;
        if (W == 1) {
          X[o] = tX[r] * sU[0];
        } else {
          T y1, y2;
          tri_pair1<T, W>(tX + r * W, sU, bp, y1, y2);
          X[o + bp] = y1;
          X[o + W - 1 - bp] = y2;
        }
      }
    }
    __syncthreads();  // tile i is no longer read
    if (bulk) bt.refill(i);
  }
}

// ------------------------------------------------ block Jacobi preconditioner

// IC(0) of every diagonal block (one CTA per block, rows level by level, one
// thread per row):
//   l_ij = (a_ij - sum_{k < j} l_ik l_jk) / l_jj   over the pattern of A,
//   l_ii = sqrt(a_ii - sum_{k < i} l_ik^2).
// The rows a row references sit on earlier levels, finished by the barrier
// that closes each level.  *flag = 1 when a pivot is not positive.
__global__ void __launch_bounds__(kThreads) k_ic0_factor(PrecSweep F, const int* lp, const int* lc,
                                                         const int* rowptr, const int* col, const double* val,
                                                         double* lv, double* ld, int* flag) {
  const int b = blockIdx.x;
  for (int l = F.blk[b]; l < F.blk[b + 1]; l++) {
    for (int q = F.lev[l] + threadIdx.x; q < F.lev[l + 1]; q += blockDim.x) {
      const int i = F.rows[q];
      const int e0 = lp[i], e1 = lp[i + 1];
      for (int e = e0; e < e1; e++) {
        const int j = lc[e];
        double s = 0.0;
        for (int a = rowptr[i]; a < rowptr[i + 1]; a++)
          if (col[a] == j) s += val[a];
        int u = e0, v = lp[j];
        const int vend = lp[j + 1];
        while (u < e && v < vend) {
          const int cu = lc[u], cv = lc[v];
          if (cu == cv) {
            s -= lv[u] * lv[v];
            u++;
            v++;
          } else if (cu < cv) {
            u++;
          } else {
            v++;
          }
        }
        lv[e] = s / ld[j];
      }
      double d = 0.0;
      for (int a = rowptr[i]; a < rowptr[i + 1]; a++)
        if (col[a] == i) d += val[a];
      for (int e = e0; e < e1; e++) d -= lv[e] * lv[e];
      if (!(d > 0.0)) {
        *flag = 1;
        d = 1.0;
      }
      ld[i] = sqrt(d);
    }
    __syncthreads();
  }
}

// Level-ordered values of one sweep from the factor: val[e] = lv[map[e]],
// diag[q] = 1 / ld[rows[q]], in FP64 and (when vf != nullptr) FP32.
__global__ void k_prec_gather(int npos, int nent, const int* map, const int* rows, const double* lv,
                              const double* ld, double* v, double* d, float* vf, float* df) {
  const int stride = gridDim.x * blockDim.x;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nent; e += stride) {
    const double x = lv[map[e]];
    v[e] = x;
    if (vf) vf[e] = (float)x;
  }
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < npos; q += stride) {
    const double x = 1.0 / ld[rows[q]];
    d[q] = x;
    if (df) df[q] = (float)x;
  }
}

// One substitution sweep over the levels of block b for the columns
// [c0, c0 + nc) of an n x w block: out_i = (src_i - sum_k val_k out_{col_k}) * diag
// with src = in (forward) or out itself (backward, in place).  Rows of one
// level are independent: each thread computes kU of them (all loads first,
// then the stores), and a barrier closes the level.
template <typename T, int KM, bool FWD>
__device__ void prec_sweep(const PrecSweep& S, int b, const T* in, T* out, int w, int c0, int nc) {
  constexpr int kU = 2;
  const T* val = (const T*)S.val;
  const T* diag = (const T*)S.diag;
  const int K = S.K;
  for (int l = S.blk[b]; l < S.blk[b + 1]; l++) {
    const int q0 = S.lev[l];
    const int items = (S.lev[l + 1] - q0) * nc;
    for (int base = threadIdx.x; base < items; base += kU * blockDim.x) {
      T sv[kU];
      long long dst[kU];
#pragma unroll
      for (int u = 0; u < kU; u++) {
        const int it = base + u * blockDim.x;
        dst[u] = -1;
        if (it < items) {
          const int qi = it / nc;
          const int q = q0 + qi;
          const int c = c0 + (it - qi * nc);
          const int i = S.rows[q];
          const int cnt = S.cnt[q];
          T acc = FWD ? in[(long long)i * w + c] : out[(long long)i * w + c];
          if (KM > 0) {
#pragma unroll
            for (int k = 0; k < KM; k++)
              if (k < cnt) acc -= val[(long long)q * K + k] * out[(long long)S.col[(long long)q * K + k] * w + c];
          } else {
            for (int k = 0; k < cnt; k++)
              acc -= val[(long long)q * K + k] * out[(long long)S.col[(long long)q * K + k] * w + c];
          }
          sv[u] = acc * diag[q];
          dst[u] = (long long)i * w + c;
        }
      }
#pragma unroll
      for (int u = 0; u < kU; u++)
        if (dst[u] >= 0) out[dst[u]] = sv[u];
    }
    __syncthreads();
  }
}

// Columns of an n x w block one preconditioner CTA solves for.
constexpr int kPrecCols = 4;

// Level-local sweep: when every entry of a row references a row of the
// level just before (the lexicographic order of a 5- or 7-point stencil
// block does this), the previous level's results stay in shared memory, so
// the chain from one level to the next runs through shared memory and a
// barrier only.  Each thread prefetches the data of its (up to two) items
// of the next level (structure, right-hand side) before the barrier that
// ends the current one.
template <typename T, int KM>
struct PrecItem {
  int i, cnt;
  T rhs, diag;
  T v[KM];
  int d[KM];
};

template <typename T, int KM, bool FWD>
__device__ void prec_sweep_local(const PrecSweep& S, int b, const T* in, T* out, int w, int c0, int nc, T* sprev,
                                 T* scur) {
  constexpr int U = 2;
  const T* val = (const T*)S.val;
  const T* diag = (const T*)S.diag;
  const int K = S.K;
  const int l0 = S.blk[b], l1 = S.blk[b + 1];
  auto load = [&](int l, int u, PrecItem<T, KM>& it) -> bool {
    const int q0 = S.lev[l];
    const int idx = threadIdx.x + u * blockDim.x;
    if (idx >= (S.lev[l + 1] - q0) * nc) return false;
    const int qi = idx / nc, c = idx - qi * nc;
    const int q = q0 + qi;
    it.i = S.rows[q];
    it.cnt = S.cnt[q];
    it.rhs = FWD ? in[(long long)it.i * w + c0 + c] : out[(long long)it.i * w + c0 + c];
    it.diag = diag[q];
#pragma unroll
    for (int k = 0; k < KM; k++) {
      it.v[k] = (k < it.cnt) ? val[(long long)q * K + k] : T(0);
      it.d[k] = (k < it.cnt) ? S.dep[(long long)q * K + k] : 0;
    }
    return true;
  };
  PrecItem<T, KM> cur[U];
  bool have[U];
  if (l0 < l1)
#pragma unroll
    for (int u = 0; u < U; u++) have[u] = load(l0, u, cur[u]);
  for (int l = l0; l < l1; l++) {
    const int items = (S.lev[l + 1] - S.lev[l]) * nc;
    if (items <= U * (int)blockDim.x) {
#pragma unroll
      for (int u = 0; u < U; u++) {
        if (!have[u]) continue;
        const int idx = threadIdx.x + u * blockDim.x;
        const int qi = idx / nc, c = idx - qi * nc;
        T acc = cur[u].rhs;
#pragma unroll
        for (int k = 0; k < KM; k++)
          if (k < cur[u].cnt) acc -= cur[u].v[k] * sprev[cur[u].d[k] * nc + c];
        acc = acc * cur[u].diag;
        scur[qi * nc + c] = acc;
        out[(long long)cur[u].i * w + c0 + c] = acc;
      }
    } else {  // a level wider than the prefetch: plain loop
      for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
        const int qi = idx / nc, c = idx - qi * nc;
        const int q = S.lev[l] + qi;
        const int i = S.rows[q], cnt = S.cnt[q];
        T acc = FWD ? in[(long long)i * w + c0 + c] : out[(long long)i * w + c0 + c];
        for (int k = 0; k < cnt; k++) acc -= val[(long long)q * K + k] * sprev[S.dep[(long long)q * K + k] * nc + c];
        acc = acc * diag[q];
        scur[qi * nc + c] = acc;
        out[(long long)i * w + c0 + c] = acc;
      }
    }
    if (l + 1 < l1)
#pragma unroll
      for (int u = 0; u < U; u++) have[u] = load(l + 1, u, cur[u]);
    __syncthreads();
    T* t = sprev;
    sprev = scur;
    scur = t;
  }
}

// Chunked level-local sweep.  Per chunk of consecutive levels (at most qc
// positions), the CTA first copies the chunk's structure (level bounds,
// rows, counts, reciprocal pivots, values, dependencies) into shared
// memory, then gathers the right-hand sides of its rows; the levels of the
// chunk then run from shared memory with one barrier each.  A chunk costs
// two memory latencies; a level no global load.
constexpr int kChunkLevels = 256;

// Bytes of the chunk buffers for qc positions, K entries per row and T: one
// 16-byte-aligned region per array, each but the right-hand sides with 16
// bytes of slack, so that a chunk's copy of a contiguous range can start at
// the same address modulo 16 as its source (prec_sweep_chunks).
__host__ __device__ constexpr size_t pad16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ constexpr size_t prec_chunk_bytes(int qc, int K, int tsize) {
  return pad16((size_t)qc * tsize + 16) + pad16((size_t)qc * K * tsize + 16) +
         pad16((size_t)qc * kPrecCols * tsize) + 2 * pad16((size_t)qc * sizeof(int) + 16) +
         pad16((size_t)qc * K * sizeof(int) + 16) + pad16(sizeof(int) * (kChunkLevels + 1) + 16);
}

// Asynchronous 4- or 8-byte copies global -> shared (cp.async): a thread
// issues all of its copies before it waits, so a chunk's loads cost one
// memory latency rather than one per loop iteration.
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* sdst, const void* gsrc) {
  static_assert(BYTES == 4 || BYTES == 8, "4- or 8-byte elements");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(sdst)), "l"(gsrc), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}
// The n elements of E bytes at gsrc into sdst (the same address modulo 16),
// by the CTA: 16-byte copies for the aligned body, element copies for the
// ends.
template <int E>
__device__ __forceinline__ void cp_async_span(void* sdst, const void* gsrc, int n) {
  unsigned char* d = (unsigned char*)sdst;
  const unsigned char* g = (const unsigned char*)gsrc;
  const int bytes = n * E;
  const int head = min(bytes, (int)((16 - ((uintptr_t)g & 15)) & 15));
  const int body = (bytes - head) & ~15;
  for (int i = threadIdx.x; i < head / E; i += blockDim.x) cp_async_elem<E>(d + i * E, g + i * E);
  for (int i = threadIdx.x; i < body / 16; i += blockDim.x) cp_async_16(d + head + 16 * i, g + head + 16 * i);
  for (int i = threadIdx.x; i < (bytes - head - body) / E; i += blockDim.x)
    cp_async_elem<E>(d + head + body + i * E, g + head + body + i * E);
}
// The first address at or after p with the same remainder modulo 16 as g.
__device__ __forceinline__ unsigned char* align_like(unsigned char* p, const void* g) {
  const uintptr_t pp = (uintptr_t)p;
  return (unsigned char*)(pp + ((((uintptr_t)g & 15) - pp) & 15));
}

template <typename T, int KM, bool FWD>
__device__ void prec_sweep_chunks(const PrecSweep& S, int b, const T* in, T* out, int w, int c0, int nc, int qc,
                                  T* sprev, T* scur, unsigned char* cbuf) {
  const int K = S.K;
  // regions of the chunk buffer (prec_chunk_bytes); each chunk places its
  // arrays at the alignment of their sources, so that the contiguous ranges
  // move as 16-byte copies
  unsigned char* r_diag = cbuf;
  unsigned char* r_val = r_diag + pad16((size_t)qc * sizeof(T) + 16);
  T* s_rhs = (T*)(r_val + pad16((size_t)qc * K * sizeof(T) + 16));  // qc x kPrecCols
  unsigned char* r_rows = (unsigned char*)s_rhs + pad16((size_t)qc * kPrecCols * sizeof(T));
  unsigned char* r_cnt = r_rows + pad16((size_t)qc * sizeof(int) + 16);
  unsigned char* r_dep = r_cnt + pad16((size_t)qc * sizeof(int) + 16);
  unsigned char* r_lev = r_dep + pad16((size_t)qc * K * sizeof(int) + 16);
  const T* val = (const T*)S.val;
  const T* diag = (const T*)S.diag;
  const T* src = FWD ? in : out;  // backward: y = L^{-1} in, already in out
  // a position's kPrecCols right-hand sides are one or two 16-byte pieces
  constexpr int RB = kPrecCols * (int)sizeof(T);
  const bool rhs16 = (nc == kPrecCols) && (RB % 16 == 0) && ((w * (int)sizeof(T)) % 16 == 0) &&
                     ((c0 * (int)sizeof(T)) % 16 == 0) && (((uintptr_t)src & 15) == 0);
  for (int j = S.cblk[b]; j < S.cblk[b + 1]; j++) {
    const int la = S.cpos[j], lb = S.cpos[j + 1];
    const int qa = S.cq[j], nq = S.cq[j + 1] - qa, nl = lb - la;
    T* s_diag = (T*)align_like(r_diag, diag + qa);                      // nq
    T* s_val = (T*)align_like(r_val, val + (long long)qa * K);           // nq x K
    int* s_rows = (int*)align_like(r_rows, S.rows + qa);                 // nq
    int* s_cnt = (int*)align_like(r_cnt, S.cnt + qa);                    // nq
    int* s_dep = (int*)align_like(r_dep, S.dep + (long long)qa * K);     // nq x K
    int* s_lev = (int*)align_like(r_lev, S.lev + la);                    // nl + 1
    __syncthreads();  // the previous chunk's buffers are no longer read
    // level bounds stay global positions (the level loop subtracts qa)
    cp_async_span<4>(s_lev, S.lev + la, nl + 1);
    cp_async_span<4>(s_rows, S.rows + qa, nq);
    cp_async_span<4>(s_cnt, S.cnt + qa, nq);
    cp_async_span<sizeof(T)>(s_diag, diag + qa, nq);
    cp_async_span<sizeof(T)>(s_val, val + (long long)qa * K, nq * K);
    cp_async_span<4>(s_dep, S.dep + (long long)qa * K, nq * K);
    cp_async_wait_all();
    __syncthreads();
    if (rhs16) {
      constexpr int PC = RB / 16;  // 16-byte pieces per position
      for (int i = threadIdx.x; i < nq * PC; i += blockDim.x) {
        const int qi = i / PC, h = i - qi * PC;
        cp_async_16((unsigned char*)&s_rhs[qi * kPrecCols] + 16 * h,
                    (const unsigned char*)&src[(long long)s_rows[qi] * w + c0] + 16 * h);
      }
    } else {
      for (int i = threadIdx.x; i < nq * nc; i += blockDim.x) {
        const int qi = i / nc, c = i - qi * nc;
        cp_async_elem<sizeof(T)>(&s_rhs[qi * kPrecCols + c], &src[(long long)s_rows[qi] * w + c0 + c]);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    if (nc == kPrecCols && K == KM) {
      // kPrecCols columns and K entries known at compile time: each result
      // replaces its right-hand side in s_rhs, and the chunk's results go to
      // global memory after its last level
      for (int l = 0; l < nl; l++) {
        const int p0 = s_lev[l] - qa, items = (s_lev[l + 1] - s_lev[l]) * kPrecCols;
        for (int idx = threadIdx.x; idx < items; idx += kThreads) {
          const int qi = idx / kPrecCols, c = idx % kPrecCols, q = p0 + qi;
          T acc = s_rhs[q * kPrecCols + c];
          const int cn = s_cnt[q];
#pragma unroll
          for (int k = 0; k < KM; k++)
            if (k < cn) acc -= s_val[q * KM + k] * sprev[s_dep[q * KM + k] * kPrecCols + c];
          acc = acc * s_diag[q];
          scur[qi * kPrecCols + c] = acc;
          s_rhs[q * kPrecCols + c] = acc;
        }
        __syncthreads();
        T* t = sprev;
        sprev = scur;
        scur = t;
      }
      for (int i = threadIdx.x; i < nq * kPrecCols; i += kThreads)
        out[(long long)s_rows[i / kPrecCols] * w + c0 + i % kPrecCols] = s_rhs[i];
      continue;
    }
    for (int l = 0; l < nl; l++) {
      const int p0 = s_lev[l] - qa, items = (s_lev[l + 1] - qa - p0) * nc;
      for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
        const int qi = idx / nc;
        const int c = idx - qi * nc, q = p0 + qi;
        T acc = s_rhs[q * kPrecCols + c];
        const int cn = s_cnt[q];
#pragma unroll
        for (int k = 0; k < KM; k++)
          if (k < cn) acc -= s_val[q * K + k] * sprev[s_dep[q * K + k] * nc + c];
        acc = acc * s_diag[q];
        scur[qi * nc + c] = acc;
        out[(long long)s_rows[q] * w + c0 + c] = acc;
      }
      __syncthreads();
      T* t = sprev;
      sprev = scur;
      scur = t;
    }
  }
}

// out = M^{-1} in = L^{-T} (L^{-1} in) for columns [c0, c0 + nc) of an n x w
// block; out holds y = L^{-1} in after the first sweep.
template <typename T, int KM>
__device__ void prec_solve_block(const PrecP& Q, int b, const T* in, T* out, int w, int c0, int nc) {
  if (KM > 0 && Q.local && Q.qc > 0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s0 = (T*)smem_raw;           // Q.maxw x kPrecCols
    T* s1 = s0 + Q.maxw * kPrecCols;  // Q.maxw x kPrecCols
    unsigned char* cbuf = (unsigned char*)(s1 + Q.maxw * kPrecCols);
    prec_sweep_chunks<T, (KM > 0 ? KM : 1), true>(Q.f, b, in, out, w, c0, nc, Q.qc, s0, s1, cbuf);
    prec_sweep_chunks<T, (KM > 0 ? KM : 1), false>(Q.b, b, in, out, w, c0, nc, Q.qc, s0, s1, cbuf);
    return;
  }
  if (KM > 0 && Q.local) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s0 = (T*)smem_raw;           // Q.maxw x kPrecCols
    T* s1 = s0 + Q.maxw * kPrecCols;  // Q.maxw x kPrecCols
    prec_sweep_local<T, (KM > 0 ? KM : 1), true>(Q.f, b, in, out, w, c0, nc, s0, s1);
    prec_sweep_local<T, (KM > 0 ? KM : 1), false>(Q.b, b, in, out, w, c0, nc, s0, s1);
    return;
  }
  prec_sweep<T, KM, true>(Q.f, b, in, out, w, c0, nc);
  prec_sweep<T, KM, false>(Q.b, b, in, out, w, c0, nc);
}

// The preconditioned generators of Section 3 (eq. (zsre2), (zmsd2),
// Algorithm 5) with diagonal blocks inside the subdomains, where
// L^{-T}[T(L^{-1} r)] = [T(M^{-1} r)]:
//   GEN_SRE:   X = M^{-1} V_{k-1}  (= M^{-1} A W_{k-1}),
//   otherwise: z = M^{-1} r_{k-1}, split by k_generate; for GEN_MSDO also
//              the partial sums of beta_k = -V_{k-1}^T z of this block.
// With in != nullptr: out = M^{-1} in for an n x w block (step-level call).
// Grid: blockIdx.x = diagonal block, blockIdx.y = group of kPrecCols
// columns (the 1-column solves use blockIdx.y == 0 only).  KM bounds the
// entries per row of both sweeps (0: any).
template <typename T, int W, int KM>
__global__ void __launch_bounds__(kThreads) k_prec_solve(KP P, PrecP Q, int gw, const T* in, T* out, int w) {
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  const int b = blockIdx.x;
  const int c0 = blockIdx.y * kPrecCols;
  if (in != nullptr) {
    if (c0 < w) prec_solve_block<T, KM>(Q, b, in, out, w, c0, min(kPrecCols, w - c0));
    return;
  }
  const int gen = st->gen;
  const T* vprev = (st->nq > 0) ? (const T*)P.desc[st->nq - 1].V : nullptr;
  if (gen == GEN_SRE) {
    if (c0 < W) prec_solve_block<T, KM>(Q, b, vprev, (T*)P.X, W, c0, min(kPrecCols, W - c0));
    return;
  }
  if (blockIdx.y != 0) return;
  T* z = (T*)P.z;
  prec_solve_block<T, KM>(Q, b, (const T*)P.r, z, 1, 0, 1);
  if (gen != GEN_MSDO) return;
  // -V_{k-1}^T z over this block's rows: thread (g, c), c = column
  __shared__ double sred[kThreads];
  constexpr int G = kThreads / W;
  const int c = threadIdx.x % W, g = threadIdx.x / W;
  const int q0 = Q.f.lev[Q.f.blk[b]], q1 = Q.f.lev[Q.f.blk[b + 1]];
  double acc = 0.0;
  if (g < G)
    for (int q = q0 + g; q < q1; q += G) {
      const int i = Q.f.rows[q];
      acc += (double)vprev[(long long)i * W + c] * (double)z[i];
    }
  sred[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < W) {
    double s = 0.0;
    for (int gg = 0; gg < G; gg++) s += sred[gg * W + threadIdx.x];
    Q.part[(long long)b * W + threadIdx.x] = -s;
  }
}

// ------------------------------------------------ block-residual mode

// R_0 = [T^t(r_0)] (n x t).
__global__ void k_block_split(KP P, const double* r, double* Rb) {
  const long long total = (long long)P.n * P.t;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / P.t), j = (int)(e - (long long)i * P.t);
    Rb[e] = (j == P.part[i]) ? r[i] : 0.0;
  }
}

// Per-CTA partial sums of alpha_k = W_k^T R_{k-1} (W x W), W_k the block
// k_final just wrote into the window slot; one thread per entry.
template <int W>
__global__ void __launch_bounds__(kThreads) k_block_alpha(KP P, int gw) {
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  const double* Wk = (const double*)P.slotW + (long long)st->next_slot * P.slot_stride;
  int r0, r1;
  cta_rows(P.n, r0, r1);
  for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
    const int a = e / W, b = e - a * W;
    double s = 0.0;
    for (int i = r0; i < r1; i++) s = fma(Wk[(long long)i * W + a], P.Rb[(long long)i * W + b], s);
    P.part_buf[(long long)blockIdx.x * W * W + e] = s;
  }
}

// R_k = R_{k-1} - V_k alpha_k, x_k = x_{k-1} + W_k alpha_k 1, r_k = R_k 1,
// partial ||r_k||^2 (one thread per row).
template <int W>
__global__ void __launch_bounds__(kThreads) k_block_update(KP P, int gw) {
  __shared__ double sal[W * W];
  __shared__ double sbuf[kThreads];
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  const long long slot = st->next_slot;
  const double* Wk = (const double*)P.slotW + slot * P.slot_stride;
  const double* Vk = (const double*)P.slotV + slot * P.slot_stride;
  double* x = (double*)P.x;
  double* r = (double*)P.r;
  for (int e = threadIdx.x; e < W * W; e += blockDim.x) sal[e] = P.small[kSmallAb + e];
  __syncthreads();
  int r0, r1;
  cta_rows(P.n, r0, r1);
  double acc = 0.0;
  // columns of alpha in chunks of CU, each against the whole row of W_k and
  // V_k (re-read from L1), so that no row is held in registers
  constexpr int CU = W < 4 ? W : 4;
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const double* wi = Wk + (long long)i * W;
    const double* vi = Vk + (long long)i * W;
    double* Ri = P.Rb + (long long)i * W;
    double dx = 0.0, rs = 0.0;
    for (int c0 = 0; c0 < W; c0 += CU) {
      double sx[CU], sr[CU];
#pragma unroll
      for (int u = 0; u < CU; u++) sx[u] = sr[u] = 0.0;
#pragma unroll 4
      for (int a = 0; a < W; a++) {
        const double wa = wi[a], va = vi[a];
#pragma unroll
        for (int u = 0; u < CU; u++) {
          sx[u] = fma(wa, sal[a * W + c0 + u], sx[u]);
          sr[u] = fma(va, sal[a * W + c0 + u], sr[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < CU; u++) {
        const double rn = Ri[c0 + u] - sr[u];
        Ri[c0 + u] = rn;
        dx += sx[u];
        rs += rn;
      }
    }
    x[i] += dx;
    r[i] = rs;
    acc += rs * rs;
  }
  const double tot = block_sum(acc, sbuf);
  if (threadIdx.x == 0) P.rho_part[blockIdx.x] = tot;
}


// End of iteration k: rho_k, tol1, window push, stop and switch tests.
// elem_bytes is the size of the solve's scalar type (slot addresses).
__device__ void finish_state(const KP& P, DevState* st, int W, double s, int elem_bytes);

// The device state is copied into shared memory with coalesced loads, thread
// 0 updates the copy, and the CTA writes it back: the updates are a chain of
// dependent field reads and writes, each a round trip to L2 when done in
// global memory.
__global__ void k_finish(KP P, int gw, int gx, int elem_bytes) {
  __shared__ double sbuf[kThreads];
  __shared__ DevState sdev;
  static_assert(sizeof(DevState) % 4 == 0, "DevState is copied as 32-bit words");
  constexpr int NW = (int)(sizeof(DevState) / 4);
  DevState* gst = P.st;
  for (int i = threadIdx.x; i < NW; i += blockDim.x)
    reinterpret_cast<int*>(&sdev)[i] = reinterpret_cast<const int*>(gst)[i];
  __syncthreads();
  DevState* st = &sdev;
  if (skip(st, gw)) return;
  double s = 0.0;
  for (int c = threadIdx.x; c < gx; c += blockDim.x) s += P.rho_part[c];
  s = block_sum(s, sbuf);
  const int W = st->width;
  if (P.want_beta) {  // beta_{k+1} = -V_k^T r_k, one warp per column
    const int lane = threadIdx.x & 31;
    for (int col = threadIdx.x >> 5; col < W; col += blockDim.x >> 5) {
      const double bsum = warp_sum_partials(P.beta_part + col, 64, gx, lane);
      if (lane == 0) P.small[kSmallBe + col] = -bsum;
    }
  }
  if (threadIdx.x == 0) finish_state(P, st, W, s, elem_bytes);
  __syncthreads();
  for (int i = threadIdx.x; i < NW; i += blockDim.x)
    reinterpret_cast<int*>(gst)[i] = reinterpret_cast<const int*>(&sdev)[i];
}

// k_finish's serial part (one thread) on the state st: rho_k, the history,
// the window push, the stopping test, restarts and the flexible switch.
__device__ void finish_state(const KP& P, DevState* st, int W, double s, int elem_bytes) {
  const int k = st->k;
  const double rho = sqrt(s);
  st->rho = rho;
  P.history[st->hist_off + k] = rho;
  st->tol1 = fabs(rho - st->rho_prev) / st->rho0;
  st->rtol1 = fabs(rho - st->rho_prev) / st->rho_cycle;
  st->rho_prev = rho;
  st->iters = k;
  if (st->stag_iters > 0 && !(rho >= 0.99 * st->rho_best)) {
    st->rho_best = rho;
    st->best_k = k;
  }
  // memory count: the window used this iteration plus the new block
  long long stored = W;
  for (int j = 0; j < st->nq; j++) stored += P.desc[j].w;
  if (stored > st->mem) st->mem = stored;
  // push (W_k, V_k), dropping the oldest block beyond the capacity
  BlockDesc nb;
  nb.slot = st->next_slot;
  nb.W = (unsigned char*)P.slotW + (long long)nb.slot * P.slot_stride * elem_bytes;
  nb.V = (unsigned char*)P.slotV + (long long)nb.slot * P.slot_stride * elem_bytes;
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
  } else if (st->stag_iters > 0 && k - st->best_k >= st->stag_iters) {
    st->stop = 1;  // stagnated: the caller's refinement continues from x_k
    st->status = ST_ENOCONV;
  } else {
    const bool do_switch = st->switch_tol > 0.0 && st->counter == 0 && st->tol1 < st->switch_tol;
    // Section 3: fixed-cycle restarts (k mod j == 1), restarts on the
    // residual-change test relative to the cycle's initial residual, and the
    // restart at the switch (Tables 8, 9)
    const bool do_restart =
        (st->restart_every >= 2 && knext % st->restart_every == 1) ||
        (st->restart_tol > 0.0 && st->rtol1 < st->restart_tol &&
         (st->restart_max == 0 || st->restarts < st->restart_max)) ||
        (do_switch && st->restart_at_switch);
    if (do_restart) {  // discard the stored blocks; the next block is [T(r)]
      st->nq = 0;
      st->next_slot = 0;
      st->restarts++;
      st->rho_cycle = rho;  // the new cycle starts from r_k
    }
    if (do_switch) {
      st->gen = GEN_SPLIT;  // W_k = [T^{t/2}(r_{k-1})]
      st->width = W / 2;
      st->counter = 1;
      st->switch_it = k;
    } else if (do_restart) {
      st->gen = GEN_SPLIT;
    } else {
      st->gen = (st->variant == 0) ? GEN_SRE : (st->variant == 1 ? GEN_MSDO : GEN_SPLIT);
    }
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

// ------------------------------------------------ iterative refinement

// bf = (float)(r * scale): right-hand side of an FP32 inner solve.
__global__ void k_to_float_scaled(int n, const double* r, float* bf, double scale) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    bf[i] = (float)(r[i] * scale);
}

// x += scale * (double)df: FP64 update by the FP32 inner correction.
__global__ void k_axpy_from_float(int n, double* x, const float* df, double scale) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x[i] = fma(scale, (double)df[i], x[i]);
}

// Matrix values rounded to FP32.
// One damped Jacobi sweep on A x = b: xout = xin + omega D^{-1} (b - A xin)
// (FP64; xin and xout distinct).
__global__ void k_jacobi(KP P, const double* xin, const double* b, double omega, double* xout) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
    double ax = 0.0, d = 0.0;
    for (int p = P.rowptr[i]; p < P.rowptr[i + 1]; p++) {
      const int j = P.col[p];
      ax += P.val[p] * xin[j];
      if (j == i) d += P.val[p];
    }
    xout[i] = xin[i] + omega * (b[i] - ax) / d;
  }
}

__global__ void k_vals_to_float(long long nnz, const double* v, float* vf) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nnz;
       i += (long long)gridDim.x * blockDim.x)
    vf[i] = (float)v[i];
}

}  // namespace ecg
