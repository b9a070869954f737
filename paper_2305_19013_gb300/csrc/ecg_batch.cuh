// ecg_batch.cuh -- persistent sm_103a kernel that runs truncated SRE-CG2
// (S. Moufawad, "Flexibly Enlarged Conjugate Gradient methods", arXiv
// 2305.19013: Algorithm 1 with the truncated window of Section 3) on many
// independent systems of uneven size in one cooperative launch.
//
// Layout.  The systems' rows are concatenated (system s owns rows
// [off_s, off_s + n_s)); every n x W block (the raw block X, Y = A X and the
// m window pairs W_j, V_j) is one N x W row-major array over all systems.
// The matrix is stored in SELL-C-sigma form per system: slices of C slots,
// slot -> row through `srow` (rows sorted by length inside windows of sigma
// rows), entries of a slice stored column-major (entry k of slot l at
// sptr[slice] + k*C + l), so a warp reads consecutive values and columns.
//
// Work split.  Each system gets a group of CTAs in proportion to its rows;
// CTA q of a group owns a row range and a slot range.  The group runs the
// iteration on its own, phase by phase; a phase that needs sums over all of
// the system's rows (CGS coefficients, Grams, ||r||^2) ends with per-CTA
// partial sums and a group barrier, after which every CTA adds the group's
// partials in the same order and so takes the same decisions.  The t x t
// factorisations are recomputed by every CTA of the group.
//
// Per iteration k (one group):
//   P1  X = generator (V_{k-1}, or [T(r)] at k = 1); C1 = V_win^T X
//   P2  X -= Q_win C1; C2 = V_win^T X                        (CGS2, pass 2)
//   P3  X -= Q_win C2; G_e = X^T X                            (Pre-CholQR)
//   P4  R_e = chol(G_e); X = X R_e^{-1}
//   P5  Y = A X; G = X^T Y; g = X^T r
//   P6  S = chol(G); alpha = S^{-T} g; W_k = X S^{-1}, V_k = Y S^{-1} into
//       the window; x += W_k alpha; r -= V_k alpha; partial ||r||^2
//   P7  rho_k, stop test, window push
// With A-CholQR alone (ortho = 1) P3 computes no Gram and P4 is skipped.
//
// Barriers are counters in global memory; every wait is bounded by
// %globaltimer and a wait that runs out marks the system ECG_ETIMEOUT and
// returns.  The cooperative launch guarantees that all CTAs are resident.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ecgb {

constexpr int kBThreads = 256;
constexpr int kBMaxW = 8;
constexpr int kBMaxM = 4;
constexpr int kBPartStride = kBMaxM * kBMaxW * kBMaxW + kBMaxW;  // doubles per CTA partial

enum BStatus { B_RUN = 0, B_OK = 1, B_NOCONV = 2, B_BREAKDOWN = 3, B_TIMEOUT = 4 };

// Per-system state of the inner solve.
struct SysState {
  int k;         // iteration about to run (1-based)
  int status;    // BStatus
  int iters;     // iterations done
  int nq;        // blocks in the window
  int head;      // ring position of the oldest window block
  int kmax;      // the solve stops at k = kmax
  int hist_off;  // history offset of this inner solve
  int pad;
  double rho0;     // ||r_0|| of this inner solve
  double rho;      // ||r_k||
  double eps;      // stop when rho <= eps * rho0
  double scale;    // mixed: ||r|| of the outer residual the inner solve started from
};

// Per-CTA placement.
struct CtaInfo {
  int sys;    // system
  int q;      // index inside the group
  int first;  // global index of the group's CTA 0
  int gsize;  // CTAs in the group
  int r0, r1; // rows (global)
  int s0, s1; // SELL slots (global slot index)
};

struct BatchP {
  int nsys;
  int m;       // window blocks
  int pre;     // 1: Pre-CholQR, 0: A-CholQR
  int C;       // SELL slice height
  const CtaInfo* cta;
  const int* part;     // N: subdomain of each row
  const int* srow;     // slots: row of each slot (-1: padding)
  const int* sptr;     // slices + 1 (per system, global numbering)
  const int* slen;     // slices: entries per slot
  const int* scol;     // entries: column (global row)
  const void* sval;    // entries (T)
  void* X;             // N x W
  void* Y;             // N x W
  void* QW;            // m slots of N x W
  void* QV;            // m slots of N x W
  long long slot_stride;  // elements between window slots (N * W)
  void* x;             // N
  void* r;             // N
  double* part_buf;    // CTAs x kBPartStride
  SysState* st;        // nsys
  unsigned* bar;       // nsys barrier counters (zero at launch)
  double* hist;        // nsys x hist_cap
  int hist_cap;
  unsigned long long wait_ns;
  int bar_extra;       // test hook: every barrier waits for this many extra arrivals
};

__device__ __forceinline__ unsigned long long b_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned b_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier of one group: arrival count reaches epoch * gsize (+ bar_extra).
// Returns false (uniformly over the CTA) when the wait ran out.
__device__ bool b_group_barrier(const BatchP& B, const CtaInfo& ci, unsigned& epoch, int* sflag) {
  // this thread's generic-proxy writes become visible to later bulk copies
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  epoch++;  // every thread keeps the count (it selects the partial buffers)
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&B.bar[ci.sys], 1u);
    const unsigned target = epoch * (unsigned)ci.gsize + (unsigned)B.bar_extra;
    int ok = 1;
    if (b_ld_acquire(&B.bar[ci.sys]) < target) {
      const unsigned long long t0 = b_globaltimer();
      ok = 0;
      for (long long it = 0; it < (1LL << 40); it++) {
        if (b_ld_acquire(&B.bar[ci.sys]) >= target) {
          ok = 1;
          break;
        }
        if ((it & 63) == 63 && b_globaltimer() - t0 > B.wait_ns) break;
        __nanosleep(64);
      }
    }
    __threadfence();
    *sflag = ok;
  }
  __syncthreads();
  return *sflag != 0;
}

// Sum of values held by the lanes of a warp that share `sub` (lanes
// sub, sub + SPL, ...); the result is valid in lanes 0 .. SPL-1.
template <typename T, int SPL>
__device__ __forceinline__ T b_warp_sum_sub(T v) {
#pragma unroll
  for (int o = SPL; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CTA reduction of per-thread accumulators acc[NA] (entry e of column
// group sub maps to out index idx(sub, e)) into part[0 .. E): warps first,
// then a fixed-order sum over warps.  sred holds kBThreads/32 x SPL x NA.
template <typename T, int SPL, int NA, typename IDX>
__device__ void b_cta_reduce(const T (&acc)[NA], double* sred, double* part, IDX idx) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = kBThreads / 32;
#pragma unroll
  for (int e = 0; e < NA; e++) {
    const T v = b_warp_sum_sub<T, SPL>(acc[e]);
    if (lane < SPL) sred[(warp * SPL + lane) * NA + e] = (double)v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < SPL * NA; t += blockDim.x) {
    const int sub = t / NA, e = t - sub * NA;
    double s = 0.0;
    for (int w = 0; w < NW; w++) s += sred[(w * SPL + sub) * NA + e];
    part[idx(sub, e)] = s;
  }
  __syncthreads();
}

// Partial sums are double-buffered by barrier parity: a CTA writes its
// partials for the next barrier into buffer (epoch & 1), where epoch counts
// the group barriers it has passed, and reads the group's partials of the
// barrier just passed from buffer ((epoch - 1) & 1).  A CTA can be one phase
// ahead of another but not two, so no write meets a read of the same buffer.
__device__ __forceinline__ double* b_part_w(const BatchP& B, unsigned epoch) {
  return B.part_buf + ((long long)(epoch & 1u) * gridDim.x + blockIdx.x) * kBPartStride;
}
__device__ __forceinline__ const double* b_part_r(const BatchP& B, unsigned epoch, int cta) {
  return B.part_buf + ((long long)((epoch - 1u) & 1u) * gridDim.x + cta) * kBPartStride;
}

// Sum of the group's partials of the barrier just passed, entries [0, E),
// in CTA order, into dst.
template <typename T>
__device__ void b_group_sum(const BatchP& B, const CtaInfo& ci, unsigned epoch, int E, T* dst) {
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < ci.gsize; q++) s += b_part_r(B, epoch, ci.first + q)[e];
    dst[e] = (T)s;
  }
  __syncthreads();
}

// Upper Cholesky G = R^T R (W x W, full symmetric input in sG) and the
// inverse of R, by thread 0; false on a pivot <= 1e-14 (FP64) or 1e-8
// (FP32) of its starting value.
template <typename T, int W>
__device__ bool b_chol_inv(const T* sG, T* sRinv, int* sflag) {
  if (threadIdx.x == 0) {
    double R[W][W], Ri[W][W];
    const double ratio = sizeof(T) == 8 ? 1e-14 : 1e-8;
    int ok = 1;
    for (int i = 0; i < W; i++)
      for (int j = 0; j < W; j++) R[i][j] = 0.0;
    for (int j = 0; j < W && ok; j++) {
      double d = (double)sG[j * W + j];
      for (int k = 0; k < j; k++) d -= R[k][j] * R[k][j];
      if (!(d > ratio * (double)sG[j * W + j]) || !isfinite(d)) {
        ok = 0;
        break;
      }
      R[j][j] = sqrt(d);
      for (int i = j + 1; i < W; i++) {
        double s = (double)sG[j * W + i];
        for (int k = 0; k < j; k++) s -= R[k][j] * R[k][i];
        R[j][i] = s / R[j][j];
      }
    }
    if (ok) {
      for (int i = 0; i < W; i++)
        for (int j = 0; j < W; j++) Ri[i][j] = 0.0;
      for (int j = W - 1; j >= 0; j--) {  // column j of R^{-1} (upper)
        Ri[j][j] = 1.0 / R[j][j];
        for (int i = j - 1; i >= 0; i--) {
          double s = 0.0;
          for (int k = i + 1; k <= j; k++) s += R[i][k] * Ri[k][j];
          Ri[i][j] = -s / R[i][i];
        }
      }
      for (int i = 0; i < W; i++)
        for (int j = 0; j < W; j++) sRinv[i * W + j] = (T)Ri[i][j];
    }
    *sflag = ok;
  }
  __syncthreads();
  return *sflag != 0;
}

// One row of an n x W block (rows are 16-byte aligned when W * sizeof(T) is
// a multiple of 16, which the vector loads rely on).
template <typename T, int W>
__device__ __forceinline__ void b_load_row(const T* base, long long i, T (&v)[W]) {
  if constexpr (sizeof(T) == 4 && W % 4 == 0) {
    const float4* p = reinterpret_cast<const float4*>(base + i * W);
#pragma unroll
    for (int a = 0; a < W / 4; a++) {
      const float4 f = p[a];
      v[4 * a] = f.x;
      v[4 * a + 1] = f.y;
      v[4 * a + 2] = f.z;
      v[4 * a + 3] = f.w;
    }
  } else if constexpr (sizeof(T) == 8 && W % 2 == 0) {
    const double2* p = reinterpret_cast<const double2*>(base + i * W);
#pragma unroll
    for (int a = 0; a < W / 2; a++) {
      const double2 f = p[a];
      v[2 * a] = f.x;
      v[2 * a + 1] = f.y;
    }
  } else {
#pragma unroll
    for (int a = 0; a < W; a++) v[a] = base[i * W + a];
  }
}

// ------------------------------------------------------ bulk-copy row tiles
//
// The phases that stream whole n x W blocks over a CTA's own rows (P1-P4,
// P6) receive them as row tiles through cp.async.bulk (the TMA engine) into
// a shared-memory ring with one mbarrier per stage counting
// the bytes.  The mbarriers are initialised once per launch; tiles are numbered by
// a counter that runs across phases, so stage g % S completes its phase
// with parity (g / S) & 1.  Every wait is bounded by
// %globaltimer.  Generic-proxy writes of a block (X, Y, the window) are
// made visible to later bulk copies by fence.proxy.async at every group
// barrier.

__device__ __forceinline__ uint32_t b_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void b_mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b_smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void b_mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b_smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool b_mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(b_smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void b_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   b_smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(b_smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool b_mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  if (b_mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = b_globaltimer();
  for (long long p = 0; p < (1LL << 30); p++) {
    if (b_mbar_try_wait(bar, parity)) return true;
    if ((p & 63) == 63 && b_globaltimer() - t0 > limit_ns) return false;
  }
  return false;
}

// Rows of a tile (one per row group) and the shared memory of the kernel.
template <typename T, int W, int MM>
struct BGeom {
  // columns per thread: the CGS coefficients a thread accumulates
  // (MM x W x CPT) stay within 64 registers' worth
  static constexpr int CPT = (MM * W * W <= 64) ? W : ((MM * W * (W / 2) <= 64) ? W / 2 : (W >= 4 ? W / 4 : 1));
  static constexpr int SPL = W / CPT;          // threads per row
  static constexpr int RG = kBThreads / SPL;   // rows per pass of the CTA = rows per tile
  static constexpr int ROWB = W * (int)sizeof(T);
  static constexpr int MAXS = 1 + 2 * MM;      // streams of the busiest phase (P2)
  static constexpr int STAGE = MAXS * RG * ROWB;
  // two stages: deeper rings took L1 capacity from the SpMM's gathers and
  // ran slower on the 64-system workload
  static constexpr int S = 2;
  static constexpr int SMEM = 64 + S * STAGE;
};

// The persistent inner solve: SRE-CG2 truncated to M window blocks (M = B.m
// at most MM), block width W, scalar T, for every system of the batch.
template <typename T, int W, int MM>
__global__ void __launch_bounds__(kBThreads, sizeof(T) == 4 ? 2 : 1) k_batch_sre(BatchP B) {
  using G_ = BGeom<T, W, MM>;
  constexpr int CPT = G_::CPT, SPL = G_::SPL, RG = G_::RG, ROWB = G_::ROWB, kS = G_::S;
  constexpr int NA1 = MM * W * CPT;    // CGS accumulators per thread
  constexpr int NAG = W * CPT + CPT;   // Gram (+ rhs) accumulators per thread
  __shared__ double sred[(kBThreads / 32) * SPL * (NA1 > NAG ? NA1 : NAG)];
  __shared__ T sC[MM * W * W];
  __shared__ T sG[W * W + W];
  __shared__ T sRe[W * W];
  __shared__ T sS[W * W];
  __shared__ T salpha[W];
  __shared__ int sflag;
  __shared__ double srho;
  extern __shared__ __align__(16) unsigned char bsm[];
  uint64_t* pbar = (uint64_t*)bsm;
  unsigned char* pstage = bsm + 64;
  const CtaInfo ci = B.cta[blockIdx.x];
  SysState* st = B.st + ci.sys;
  if (st->status != B_RUN) return;
  const int m = B.m;
  const int sub = threadIdx.x % SPL, rg = threadIdx.x / SPL;
  const int c0 = sub * CPT;
  const int lane = threadIdx.x & 31;
  const unsigned gmask = ((SPL == 32) ? 0xffffffffu : ((1u << SPL) - 1u)) << (lane & ~(SPL - 1));
  T* X = (T*)B.X;
  T* Y = (T*)B.Y;
  T* x = (T*)B.x;
  T* r = (T*)B.r;
  unsigned epoch = 0;
  auto fail = [&](int code) {
    if (threadIdx.x == 0) atomicCAS(&st->status, B_RUN, code);
  };
  if (threadIdx.x == 0) {
    for (int s = 0; s < kS; s++) b_mbar_init(&pbar[s]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  unsigned gt = 0;  // tiles issued in earlier phases (same in every thread)

  // Stream nstr blocks (bases[j], n x W) over the CTA's rows in tiles of RG
  // rows and call body(i, tile) for row i of every tile, tile(j) being row
  // i of stream j in shared memory.  False after a wait ran out (the copies
  // still in flight are waited for, boundedly).
  auto stream_rows = [&](int nstr, const T* const* bases, auto&& body) -> bool {
    const int ntiles = (ci.r1 - ci.r0 + RG - 1) / RG;
    auto issue = [&](int t) {
      const unsigned g = gt + (unsigned)t;
      const int s = (int)(g % kS);
      const int row0 = ci.r0 + t * RG;
      const int nr = min(RG, ci.r1 - row0);
      b_mbar_expect_tx(&pbar[s], (uint32_t)(nstr * nr * ROWB));
      unsigned char* dst = pstage + (long long)s * G_::STAGE;
      for (int j = 0; j < nstr; j++)
        b_bulk_g2s(dst + (long long)j * RG * ROWB, (const unsigned char*)bases[j] + (long long)row0 * ROWB,
                   (uint32_t)(nr * ROWB), &pbar[s]);
    };
    if (threadIdx.x == 0)
      for (int t = 0; t < min(kS, ntiles); t++) issue(t);
    bool ok = true;
    for (int t = 0; t < ntiles; t++) {
      const unsigned g = gt + (unsigned)t;
      const bool w = b_mbar_wait(&pbar[g % kS], (g / kS) & 1u, B.wait_ns);
      if (!__syncthreads_and(w)) {
        if (threadIdx.x == 0)
          for (int u = t; u < min(t + kS, ntiles); u++)
            b_mbar_wait(&pbar[(gt + u) % kS], ((gt + u) / kS) & 1u, B.wait_ns);
        __syncthreads();
        ok = false;
        break;
      }
      const int row0 = ci.r0 + t * RG;
      const int nr = min(RG, ci.r1 - row0);
      const T* stg = (const T*)(pstage + (long long)(g % kS) * G_::STAGE);
      if (rg < nr) body(row0 + rg, [&](int j) { return stg + ((long long)j * RG + rg) * W; });
      __syncthreads();
      if (threadIdx.x == 0 && t + kS < ntiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(t + kS);
      }
    }
    gt += (unsigned)ntiles;
    return ok;
  };

  // local copies of the group's state, identical in every CTA
  int k = st->k, nq = st->nq, head = st->head;
  const int kmax = st->kmax;
  const double eps = st->eps;
  double rho0;
  auto wslot = [&](int j) { return (head + j) % m; };
  auto QWb = [&](int slot) { return (T*)B.QW + (long long)slot * B.slot_stride; };
  auto QVb = [&](int slot) { return (T*)B.QV + (long long)slot * B.slot_stride; };

  // ---- P0: rho_0 = ||r||
  {
    double acc = 0.0;
    for (int i = ci.r0 + threadIdx.x; i < ci.r1; i += blockDim.x) acc += (double)r[i] * (double)r[i];
    double accs[1] = {acc};
    b_cta_reduce<double, 1, 1>(accs, sred, b_part_w(B, epoch), [](int, int) { return 0; });
    if (!b_group_barrier(B, ci, epoch, &sflag)) return fail(B_TIMEOUT);
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int q = 0; q < ci.gsize; q++) s += b_part_r(B, epoch, ci.first + q)[0];
      srho = sqrt(s);
    }
    __syncthreads();
    rho0 = srho;
    if (ci.q == 0 && threadIdx.x == 0) {
      st->rho0 = rho0;
      st->rho = rho0;
      if (st->hist_off < B.hist_cap) B.hist[(long long)ci.sys * B.hist_cap + st->hist_off] = rho0 * st->scale;
    }
    if (!(rho0 > 0.0) || !(rho0 > eps * rho0) || k >= kmax) {
      if (ci.q == 0 && threadIdx.x == 0) st->status = (rho0 > eps * rho0) ? B_NOCONV : B_OK;
      return;
    }
  }

  for (;;) {
    const int nwin = nq;  // window blocks used by CGS; k >= 2 <=> nwin >= 1
    const T* vprev = (nq > 0) ? QVb(wslot(nq - 1)) : nullptr;
    // ---- P1, P2: CGS2 against the window (X = V_{k-1} for k >= 2)
    if (nwin > 0) {
      for (int pass = 0; pass < 2; pass++) {
        T acc[NA1];
#pragma unroll
        for (int e = 0; e < NA1; e++) acc[e] = T(0);
        if (pass == 1) b_group_sum<T>(B, ci, epoch, nwin * W * W, sC);
        // streams: vprev, [Q_0 .. Q_{nwin-1}] (pass 1), V_0 .. V_{nwin-1}
        const T* bases[G_::MAXS];
        int ns = 0;
        bases[ns++] = vprev;
        if (pass == 1)
          for (int j = 0; j < nwin; j++) bases[ns++] = QWb(wslot(j));
        const int vbase = ns;
        for (int j = 0; j < nwin; j++) bases[ns++] = QVb(wslot(j));
        const bool ok = stream_rows(ns, bases, [&](int i, auto&& row) {
          T xc[CPT];
          const T* g0 = row(0);
#pragma unroll
          for (int c = 0; c < CPT; c++) xc[c] = g0[c0 + c];
          if (pass == 1) {  // X - Q C1, regenerated from V_{k-1}
            for (int j = 0; j < nwin; j++) {
              const T* qr = row(1 + j);
#pragma unroll
              for (int a = 0; a < W; a++)
#pragma unroll
                for (int c = 0; c < CPT; c++) xc[c] -= qr[a] * sC[(j * W + a) * W + c0 + c];
            }
#pragma unroll
            for (int c = 0; c < CPT; c++) X[(long long)i * W + c0 + c] = xc[c];
          }
#pragma unroll
          for (int j = 0; j < MM; j++) {
            if (j < nwin) {
              const T* vr = row(vbase + j);
#pragma unroll
              for (int a = 0; a < W; a++)
#pragma unroll
                for (int c = 0; c < CPT; c++) acc[(j * W + a) * CPT + c] += vr[a] * xc[c];
            }
          }
        });
        if (!ok) return fail(B_TIMEOUT);
        b_cta_reduce<T, SPL, NA1>(acc, sred, b_part_w(B, epoch),
                                  [](int s, int e) { return (e / CPT) * W + s * CPT + (e % CPT); });
        if (!b_group_barrier(B, ci, epoch, &sflag)) return fail(B_TIMEOUT);
      }
    }
    // ---- P3: X -= Q C2 (or X = [T(r)] at k = 1); G_e = X^T X
    {
      if (nwin > 0) b_group_sum<T>(B, ci, epoch, nwin * W * W, sC);
      T acc[NAG];
#pragma unroll
      for (int e = 0; e < NAG; e++) acc[e] = T(0);
      auto finish_row = [&](int i, T (&xc)[CPT]) {
#pragma unroll
        for (int c = 0; c < CPT; c++) X[(long long)i * W + c0 + c] = xc[c];
        if (B.pre) {
          T xr[W];  // the full row from the row group's lanes
#pragma unroll
          for (int s2 = 0; s2 < SPL; s2++)
#pragma unroll
            for (int c = 0; c < CPT; c++)
              xr[s2 * CPT + c] = __shfl_sync(gmask, xc[c], (lane & ~(SPL - 1)) + s2);
#pragma unroll
          for (int a = 0; a < W; a++)
#pragma unroll
            for (int c = 0; c < CPT; c++) acc[a * CPT + c] += xr[a] * xc[c];
        }
      };
      if (nwin > 0) {
        const T* bases[G_::MAXS];
        int ns = 0;
        bases[ns++] = X;
        for (int j = 0; j < nwin; j++) bases[ns++] = QWb(wslot(j));
        const bool ok = stream_rows(ns, bases, [&](int i, auto&& row) {
          T xc[CPT];
          const T* xr0 = row(0);
#pragma unroll
          for (int c = 0; c < CPT; c++) xc[c] = xr0[c0 + c];
          for (int j = 0; j < nwin; j++) {
            const T* qr = row(1 + j);
#pragma unroll
            for (int a = 0; a < W; a++)
#pragma unroll
              for (int c = 0; c < CPT; c++) xc[c] -= qr[a] * sC[(j * W + a) * W + c0 + c];
          }
          finish_row(i, xc);
        });
        if (!ok) return fail(B_TIMEOUT);
      } else {  // k = 1: [T^t(r_0)]
        for (int i = ci.r0 + rg; i < ci.r1; i += RG) {
          T xc[CPT];
          const int pj = B.part[i];
          const T ri = r[i];
#pragma unroll
          for (int c = 0; c < CPT; c++) xc[c] = (c0 + c == pj) ? ri : T(0);
          finish_row(i, xc);
        }
      }
      if (B.pre) {
        b_cta_reduce<T, SPL, NAG>(acc, sred, b_part_w(B, epoch), [](int s, int e) {
          return e < W * CPT ? (e / CPT) * W + s * CPT + (e % CPT) : W * W + s * CPT + (e - W * CPT);
        });
      }
      if (!b_group_barrier(B, ci, epoch, &sflag)) return fail(B_TIMEOUT);
    }
    // ---- P4: R_e = chol(X^T X); X = X R_e^{-1}   (Pre-CholQR)
    if (B.pre) {
      b_group_sum<T>(B, ci, epoch, W * W, sG);
      if (!b_chol_inv<T, W>(sG, sRe, &sflag)) {
        if (ci.q == 0 && threadIdx.x == 0) atomicCAS(&st->status, B_RUN, B_BREAKDOWN);
        return;
      }
      const T* bases[1] = {X};
      const bool ok = stream_rows(1, bases, [&](int i, auto&& row) {
        const T* xr = row(0);
#pragma unroll
        for (int c = 0; c < CPT; c++) {
          T s = T(0);
#pragma unroll
          for (int a = 0; a < W; a++) s += xr[a] * sRe[a * W + c0 + c];
          X[(long long)i * W + c0 + c] = s;
        }
      });
      if (!ok) return fail(B_TIMEOUT);
      if (!b_group_barrier(B, ci, epoch, &sflag)) return fail(B_TIMEOUT);
    }
    // ---- P5: Y = A X over my slots; G = X^T Y, g = X^T r
    {
      const T* sval = (const T*)B.sval;
      T acc[NAG];
#pragma unroll
      for (int e = 0; e < NAG; e++) acc[e] = T(0);
      for (int s = ci.s0 + rg; s < ci.s1; s += RG) {
        const int i = B.srow[s];
        if (i < 0) continue;  // padding slot (uniform over the row group)
        const int slice = s / B.C, l = s - slice * B.C;
        const int base = B.sptr[slice] + l, len = B.slen[slice];
        T y[CPT];
#pragma unroll
        for (int c = 0; c < CPT; c++) y[c] = T(0);
        for (int kk = 0; kk < len; kk++) {
          const T a = sval[base + kk * B.C];
          const long long j = B.scol[base + kk * B.C];
#pragma unroll
          for (int c = 0; c < CPT; c++) y[c] += a * X[j * W + c0 + c];
        }
#pragma unroll
        for (int c = 0; c < CPT; c++) Y[(long long)i * W + c0 + c] = y[c];
        T xr[W];
        b_load_row<T, W>(X, i, xr);
        const T ri = r[i];
#pragma unroll
        for (int a = 0; a < W; a++)
#pragma unroll
          for (int c = 0; c < CPT; c++) acc[a * CPT + c] += xr[a] * y[c];
#pragma unroll
        for (int c = 0; c < CPT; c++) acc[W * CPT + c] += xr[c0 + c] * ri;
      }
      b_cta_reduce<T, SPL, NAG>(acc, sred, b_part_w(B, epoch), [](int s, int e) {
        return e < W * CPT ? (e / CPT) * W + s * CPT + (e % CPT) : W * W + s * CPT + (e - W * CPT);
      });
      if (!b_group_barrier(B, ci, epoch, &sflag)) return fail(B_TIMEOUT);
    }
    // ---- P6: S = chol(G), alpha = S^{-T} g, W_k, V_k, x, r, ||r||^2
    const int newslot = (nq < m) ? (head + nq) % m : head;
    {
      b_group_sum<T>(B, ci, epoch, W * W + W, sG);
      if (!b_chol_inv<T, W>(sG, sS, &sflag)) {
        if (ci.q == 0 && threadIdx.x == 0) atomicCAS(&st->status, B_RUN, B_BREAKDOWN);
        return;
      }
      if (threadIdx.x < W) {  // alpha = S^{-T} g = (S^{-1})^T g
        T s = T(0);
        for (int a = 0; a <= (int)threadIdx.x; a++) s += sS[a * W + threadIdx.x] * sG[W * W + a];
        salpha[threadIdx.x] = s;
      }
      __syncthreads();
      T* Wn = QWb(newslot);
      T* Vn = QVb(newslot);
      double racc = 0.0;
      const T* bases[2] = {X, Y};
      const bool ok = stream_rows(2, bases, [&](int i, auto&& row) {
        const T* xr = row(0);
        const T* yr = row(1);
        T dx = T(0), dr = T(0);
#pragma unroll
        for (int c = 0; c < CPT; c++) {
          T w = T(0), v = T(0);
#pragma unroll
          for (int a = 0; a < W; a++) {
            w += xr[a] * sS[a * W + c0 + c];
            v += yr[a] * sS[a * W + c0 + c];
          }
          Wn[(long long)i * W + c0 + c] = w;
          Vn[(long long)i * W + c0 + c] = v;
          dx += w * salpha[c0 + c];
          dr += v * salpha[c0 + c];
        }
#pragma unroll
        for (int o = 1; o < SPL; o <<= 1) {
          dx += __shfl_xor_sync(gmask, dx, o);
          dr += __shfl_xor_sync(gmask, dr, o);
        }
        if (sub == 0) {
          x[i] += dx;
          const T rn = r[i] - dr;
          r[i] = rn;
          racc += (double)rn * (double)rn;
        }
      });
      if (!ok) return fail(B_TIMEOUT);
      double accs[1] = {racc};
      b_cta_reduce<double, 1, 1>(accs, sred, b_part_w(B, epoch), [](int, int) { return 0; });
      if (!b_group_barrier(B, ci, epoch, &sflag)) return fail(B_TIMEOUT);
    }
    // ---- P7: rho_k, stop test, window push (same decisions in every CTA)
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int q = 0; q < ci.gsize; q++) s += b_part_r(B, epoch, ci.first + q)[0];
      srho = sqrt(s);
    }
    __syncthreads();
    const double rho = srho;
    if (nq < m) nq++;
    else head = (head + 1) % m;
    const int knext = k + 1;
    int status = B_RUN;
    if (!(rho > eps * rho0)) status = B_OK;
    else if (knext >= kmax) status = B_NOCONV;
    if (ci.q == 0 && threadIdx.x == 0) {
      st->rho = rho;
      st->iters = k;
      st->k = knext;
      st->nq = nq;
      st->head = head;
      if (st->hist_off + k < B.hist_cap) B.hist[(long long)ci.sys * B.hist_cap + st->hist_off + k] = rho * st->scale;
      if (status != B_RUN) atomicCAS(&st->status, B_RUN, status);
    }
    k = knext;
    if (status != B_RUN) return;
  }
}

// ------------------------------------------------------------ outer loop

// Outer (refinement) state of one system.
struct Outer {
  double rho0;      // ||b - A x_0||
  double rho_last;  // residual norm at the previous round
  double scale;     // ||r|| the current inner solve started from
  int iters;        // inner iterations of all rounds
  int done;         // 1: finished
  int status;       // ECG status code once done
  int ran;          // the inner solve ran in the current round
  int rounds;       // rounds started
  int pad;
};

__device__ __forceinline__ int b_ecg_status(int bs) {
  // ECG_OK 0, ECG_ENOCONV 1, ECG_EBREAKDOWN -4, ECG_ETIMEOUT -6
  return bs == B_OK ? 0 : (bs == B_NOCONV ? 1 : (bs == B_BREAKDOWN ? -4 : (bs == B_TIMEOUT ? -6 : 1)));
}

// r = b - A x (FP64) over the CTA's slots, with per-CTA partial sums of
// ||r||^2 and ||b||^2 in part2[2 * cta + {0, 1}].
__global__ void __launch_bounds__(kBThreads) k_batch_residual(BatchP B, const double* sval64, const double* xx,
                                                              const double* bb, double* rr, double* part2) {
  __shared__ double sred[2 * (kBThreads / 32)];
  const CtaInfo ci = B.cta[blockIdx.x];
  double a_rr = 0.0, a_bb = 0.0;
  for (int s = ci.s0 + threadIdx.x; s < ci.s1; s += blockDim.x) {
    const int i = B.srow[s];
    if (i < 0) continue;
    const int slice = s / B.C, l = s - slice * B.C;
    const int base = B.sptr[slice] + l, len = B.slen[slice];
    double y = 0.0;
    for (int k = 0; k < len; k++) y += sval64[base + k * B.C] * xx[B.scol[base + k * B.C]];
    const double ri = bb[i] - y;
    rr[i] = ri;
    a_rr += ri * ri;
    a_bb += bb[i] * bb[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a_rr += __shfl_xor_sync(0xffffffffu, a_rr, o);
    a_bb += __shfl_xor_sync(0xffffffffu, a_bb, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sred[2 * warp] = a_rr;
    sred[2 * warp + 1] = a_bb;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s2 += sred[2 * w + threadIdx.x];
    part2[2 * blockIdx.x + threadIdx.x] = s2;
  }
}

// Per-system sums of the residual partials, CTA order.
__global__ void k_batch_norms(int nsys, const int* first, const int* gsize, const double* part2, double* rr,
                              double* bb) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  double a = 0.0, b = 0.0;
  for (int q = 0; q < gsize[s]; q++) {
    a += part2[2 * (first[s] + q)];
    b += part2[2 * (first[s] + q) + 1];
  }
  rr[s] = a;
  bb[s] = b;
}

// Start of a round: account for the previous inner solve, decide whether
// the system is done, and set up the next inner solve.  Mixed precision
// (refine = 1): the inner FP32 solve starts from r / ||r|| and needs to
// reach only what is left of the tolerance; the outer test is the FP64
// ||b - A x|| <= tol ||b - A x_0||, with a stop when a round makes no
// progress.  FP64 (refine = 0): one inner solve with the paper's test
// rho_k <= tol rho_0, whose status is the result.
__global__ void k_batch_round_begin(int nsys, SysState* st, Outer* o, const double* rr, double tol, double inner_tol,
                                    int kmax, int refine, int max_rounds, int* active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  Outer& O = o[s];
  SysState& S = st[s];
  if (O.ran) {
    O.ran = 0;
    O.iters += S.iters;
    if (!refine) {
      O.done = 1;
      O.status = b_ecg_status(S.status);
    } else if (S.status == B_TIMEOUT) {
      O.done = 1;
      O.status = -6;
    } else if (S.status == B_BREAKDOWN && S.iters == 0) {
      O.done = 1;
      O.status = -4;
    }
  }
  const double rho = sqrt(rr[s]);
  if (O.rounds == 0 && !O.done) O.rho0 = rho;
  if (!O.done) {
    if (!(rho > tol * O.rho0)) {
      O.done = 1;
      O.status = 0;
    } else if (O.rounds > 0 && !(rho < O.rho_last)) {
      O.done = 1;
      O.status = 1;
    } else if (O.iters >= kmax - 1 || O.rounds >= max_rounds) {
      O.done = 1;
      O.status = 1;
    }
  }
  O.rho_last = rho;
  if (O.done) {
    if (S.status == B_RUN) S.status = B_OK;
    return;
  }
  O.rounds++;
  O.ran = 1;
  O.scale = refine ? rho : 1.0;
  S.k = 1;
  S.status = B_RUN;
  S.iters = 0;
  S.nq = 0;
  S.head = 0;
  S.kmax = kmax - O.iters;
  S.hist_off = O.iters;
  S.rho0 = 0.0;
  S.rho = 0.0;
  S.eps = refine ? fmin(0.5, fmax(inner_tol, 0.1 * tol * O.rho0 / rho)) : tol;
  S.scale = O.scale;
  atomicAdd(active, 1);
}

// Mixed precision, per CTA rows: rf = r / scale and xf = 0 for the systems
// whose inner solve runs in this refinement step.
__global__ void k_batch_scale(BatchP B, const Outer* o, const double* rr, float* rf, float* xf) {
  const CtaInfo ci = B.cta[blockIdx.x];
  if (!o[ci.sys].ran) return;
  const double inv = 1.0 / o[ci.sys].scale;
  for (int i = ci.r0 + threadIdx.x; i < ci.r1; i += blockDim.x) {
    rf[i] = (float)(rr[i] * inv);
    xf[i] = 0.0f;
  }
}

// Mixed precision, per CTA rows: x += scale * xf after the inner solve.
__global__ void k_batch_round_end(BatchP B, const Outer* o, double* xx, const float* xf) {
  const CtaInfo ci = B.cta[blockIdx.x];
  if (!o[ci.sys].ran) return;
  const double sc = o[ci.sys].scale;
  for (int i = ci.r0 + threadIdx.x; i < ci.r1; i += blockDim.x) xx[i] += sc * (double)xf[i];
}

// Y = A X over all slots (SELL-C-sigma), the product the autotuner times.
template <typename T, int W>
__global__ void __launch_bounds__(kBThreads) k_batch_spmm(BatchP B, int nslots) {
  const T* sval = (const T*)B.sval;
  const T* X = (const T*)B.X;
  T* Y = (T*)B.Y;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslots; s += gridDim.x * blockDim.x) {
    const int i = B.srow[s];
    if (i < 0) continue;
    const int slice = s / B.C, l = s - slice * B.C;
    const int base = B.sptr[slice] + l, len = B.slen[slice];
    T y[W];
#pragma unroll
    for (int c = 0; c < W; c++) y[c] = T(0);
    for (int k = 0; k < len; k++) {
      const T a = sval[base + k * B.C];
      T xr[W];
      b_load_row<T, W>(X, B.scol[base + k * B.C], xr);
#pragma unroll
      for (int c = 0; c < W; c++) y[c] += a * xr[c];
    }
#pragma unroll
    for (int c = 0; c < W; c++) Y[(long long)i * W + c] = y[c];
  }
}

}  // namespace ecgb
