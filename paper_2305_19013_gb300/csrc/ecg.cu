// ecg.cu -- host side of libecg: the C ABI of include/ecg.h, device memory,
// and the iteration driver of the enlarged CG methods (S. Moufawad,
// "Flexibly Enlarged Conjugate Gradient methods", arXiv 2305.19013,
// Algorithms 1-4).
//
// The driver never waits on the device inside the iteration loop: it issues
// `check_every` iterations of the kernel chain of ecg_kernels.cuh, queues an
// asynchronous copy of the device state into pinned host memory, issues the
// next group, and only then reads the state of the previous group.  The
// device decides when to stop (rho_k <= eps rho_0 or k = k_max, breakdown)
// and when to switch to t/2 vectors; kernels issued after either event
// return at once.  With a truncated window the group of iterations is
// captured once as a CUDA graph and replayed.
//
// Mixed precision (ECG_MIXED): an FP64 iterative-refinement loop around FP32
// inner solves.  Each outer step computes the true residual r = b - A x in
// FP64, runs the same enlarged CG iteration in FP32 on A d = r / ||r|| (the
// t x t factorisations, alpha and beta stay FP64), and updates
// x += ||r|| d in FP64.  It stops on the FP64 true residual.  (Keeping the
// window and only replacing the FP32 residual by the FP64 one was tried and
// converges far worse: SRE-CG builds new directions from A W, so error
// components of the replaced residual along directions that left the window
// are never revisited; a restart rebuilds directions from T^t(r).)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ecg.h"
#include "ecg_kernels.cuh"
#include "ecg_tc.cuh"

using namespace ecg;

namespace {

constexpr int kWidths[] = {1, 2, 4, 8, 16, 32, 64};
constexpr double kBreakdownFP64 = 1e-14;  // Cholesky pivot test, FP64 data
constexpr double kBreakdownFP32 = 1e-8;   // FP32 blocks: Grams carry ~1e-7 rounding
// FP32 rounds of mixed precision end after this many iterations without a 1%
// smaller residual (see run_solve)
constexpr int kStagIters = 400;
constexpr int kMaxOuter = 64;             // refinement steps of the mixed method

int width_index(int w) {
  for (int i = 0; i < 7; i++)
    if (kWidths[i] == w) return i;
  return -1;
}

struct Prof {
  // per kernel class: total device ms and launches, accumulated while
  // profiling is on
  double ms[16];
  long long launches[16];
};

const char* kProfNames[] = {"generate", "cgs_tdot", "cgs_update", "gram_e", "small_e", "spmm_gram",
                            "small_a",  "final",    "finish",     "setup",  "precond"};
constexpr int kProfClasses = 11;

}  // namespace

struct ecg_ctx {
  int n = 0;
  int64_t nnz = 0;
  int t = 0;
  ecg_opts opts;
  int dev = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int* d_rowptr = nullptr;
  int* d_col = nullptr;
  double* d_val = nullptr;
  float* d_valf = nullptr;  // mixed precision only
  int* d_pmap = nullptr;    // subdomain of each row
  double *d_X = nullptr, *d_Y = nullptr;  // work blocks, n x t doubles (also hold FP32 blocks)
  double *d_x = nullptr, *d_r = nullptr, *d_b = nullptr;
  float *d_xf = nullptr, *d_rf = nullptr, *d_bf = nullptr;  // FP32 inner solve vectors
  double *d_sx = nullptr, *d_sr = nullptr;  // scratch x, r for step-level calls
  DevState* d_st = nullptr;
  DevState* d_opst = nullptr;
  BlockDesc* d_desc = nullptr;
  int desc_cap = 0;
  BlockDesc* d_opdesc = nullptr;
  int opdesc_cap = 0;
  void *d_slotW = nullptr, *d_slotV = nullptr;  // window storage
  int slot_cap = 0;
  double* d_C = nullptr;
  size_t C_cap = 0;
  double* d_partial = nullptr;  // per-CTA partial sums
  size_t part_cap = 0;
  double* d_small = nullptr;
  double* d_hist = nullptr;
  int hist_cap = 0;
  double *d_rho_part = nullptr, *d_beta_part = nullptr, *d_bb_part = nullptr;
  int gx = 1;
  // FP32 spmm_gram / final grids by block width index (log2 W): one wave at
  // the kernels' occupancy, at most gx
  int gx_spmm32[7] = {}, gx_fin32[7] = {}, gx_gram32[7] = {};
  int gx_spmm64[7] = {};  // FP64 A-CholQR SpMM + Gram: one wave at its occupancy (not capped at gx)
  // occupancy-sized grids of the CGS kernels by (kernel, shared memory)
  struct OccEntry {
    const void* kernel;
    size_t smem;
    int grid;
  };
  std::vector<OccEntry> occ;
  std::vector<double> h_hist;
  DevState* h_flags = nullptr;  // pinned, 2 entries
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaGraphExec_t gexec[14] = {};  // [FP32 ? 7 : 0] + width index
  int graph_iters[14] = {};
  // block Jacobi preconditioner (prec_nb == 0: none)
  struct Sweep {  // one substitution in level order (see PrecSweep)
    int *blk = nullptr, *lev = nullptr, *rows = nullptr, *cnt = nullptr, *col = nullptr, *map = nullptr;
    int* dep = nullptr;  // level-local mode: index of each entry's row in the previous level
    int *cpos = nullptr, *cq = nullptr, *cblk = nullptr;  // chunks of levels (see PrecSweep)
    double *val = nullptr, *diag = nullptr;
    float *valf = nullptr, *diagf = nullptr;
    int K = 1;
  };
  int prec_nb = 0;
  int prec_local = 0, prec_maxw = 0;           // level-local mode (see PrecP)
  int prec_qc = 0;                             // chunked level-local mode (see PrecP)
  Sweep pf, pb;                                // forward and backward sweeps
  int *d_lp = nullptr, *d_lc = nullptr;        // L by rows (factorisation)
  double *d_lv = nullptr, *d_ld = nullptr;
  double* d_z = nullptr;
  float* d_zf = nullptr;
  double* d_ppart = nullptr;  // nb x 64
  double* d_Rb = nullptr;     // block residual (n x t), block-residual mode
  int* d_pflag = nullptr;
  bool profiling = false;
  std::vector<cudaEvent_t> pev;  // profiling event pool
  size_t pev_used = 0;
  std::vector<int> pev_class;
  Prof prof;
};

namespace {

#define CK(call)                     \
  do {                               \
    cudaError_t e_ = (call);         \
    if (e_ != cudaSuccess) {         \
      last_cuda_error() = e_;        \
      return ECG_ECUDA;              \
    }                                \
  } while (0)

cudaError_t& last_cuda_error() {
  static thread_local cudaError_t e = cudaSuccess;
  return e;
}

template <typename T>
int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return (e == cudaErrorMemoryAllocation) ? ECG_ENOMEM : ECG_ECUDA;
  }
  return ECG_OK;
}

int dalloc_bytes(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 1;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return (e == cudaErrorMemoryAllocation) ? ECG_ENOMEM : ECG_ECUDA;
  }
  return ECG_OK;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T, int W>
constexpr size_t smem_spmm() {
  return sizeof(T) * (4 * Tile<W>::R * W + W * W + Tile<W>::R);
}
// k_spmm_gram_rows: its own layout, or the scalar one when it falls back
template <int W>
constexpr size_t smem_spmm_rows() {
  return smem_spmm_f32<W>() > smem_spmm<float, W>() ? smem_spmm_f32<W>() : smem_spmm<float, W>();
}
template <int W>
constexpr size_t smem_small() {
  return sizeof(double) * (3 * W * W + 2 * W);
}

template <typename T, int W>
int set_smem_attrs_t() {
  CK(cudaFuncSetAttribute(k_tdot_window<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)smem_tdot<T, W>()));
  CK(cudaFuncSetAttribute(k_update<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_update<T, W>()));
  CK(cudaFuncSetAttribute(k_spmm_gram<T, W, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)smem_spmm<T, W>()));
  CK(cudaFuncSetAttribute(k_spmm_gram<T, W, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)smem_spmm<T, W>()));
  CK(cudaFuncSetAttribute(k_spmm_gram<T, W, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)smem_spmm<T, W>()));
  CK(cudaFuncSetAttribute(k_final<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_final<T, W>()));
  CK(cudaFuncSetAttribute(k_gram_self<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)smem_gram_self<T, W>()));
  CK(cudaFuncSetAttribute(k_tri_right<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)smem_tri_right<T, W>()));
  if constexpr (F32Rows<T, W>::on) {
    CK(cudaFuncSetAttribute(k_spmm_gram_rows<W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)smem_spmm_rows<W>()));
    CK(cudaFuncSetAttribute(k_spmm_gram_rows<W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)smem_spmm_rows<W>()));
  }
  return ECG_OK;
}

// The chunked preconditioner sweeps use up to about 104 KB of dynamic
// shared memory; allow that for every instantiation.
template <typename T, int W>
int set_prec_smem_attrs() {
  constexpr int kBytes = 160 * 1024;
  CK(cudaFuncSetAttribute(k_prec_solve<T, W, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBytes));
  CK(cudaFuncSetAttribute(k_prec_solve<T, W, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBytes));
  CK(cudaFuncSetAttribute(k_prec_solve<T, W, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBytes));
  return ECG_OK;
}

template <int W>
int set_smem_attrs() {
  int rc;
  if ((rc = set_smem_attrs_t<double, W>())) return rc;
  if ((rc = set_smem_attrs_t<float, W>())) return rc;
  if ((rc = set_prec_smem_attrs<double, W>())) return rc;
  if ((rc = set_prec_smem_attrs<float, W>())) return rc;
  CK(cudaFuncSetAttribute(k_small_e<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_small<W>()));
  CK(cudaFuncSetAttribute(k_small_a<W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)smem_small<W>()));
  CK(cudaFuncSetAttribute(k_small_a<W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)smem_small<W>()));
  return ECG_OK;
}

int set_all_smem_attrs() {
  int rc = ECG_OK;
  CK(cudaFuncSetAttribute(tc::k_update_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)tc::smem_update_tc<16>()));
  CK(cudaFuncSetAttribute(tc::k_final_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)tc::smem_final_tc<16>()));
  CK(cudaFuncSetAttribute(tc::k_tdot_tc<double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)tc::smem_tdot_tc<double, 16>()));
  CK(cudaFuncSetAttribute(tc::k_tdot_tc<float, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)tc::smem_tdot_tc<float, 16>()));
  if ((rc = set_smem_attrs<1>())) return rc;
  if ((rc = set_smem_attrs<2>())) return rc;
  if ((rc = set_smem_attrs<4>())) return rc;
  if ((rc = set_smem_attrs<8>())) return rc;
  if ((rc = set_smem_attrs<16>())) return rc;
  if ((rc = set_smem_attrs<32>())) return rc;
  return set_smem_attrs<64>();
}

KP make_kp(ecg_ctx* c, DevState* st, BlockDesc* desc, bool fp32) {
  KP P;
  P.n = c->n;
  P.t = c->t;
  P.rowptr = c->d_rowptr;
  P.col = c->d_col;
  P.val = c->d_val;
  P.valf = c->d_valf;
  P.part = c->d_pmap;
  P.X = c->d_X;
  P.Y = c->d_Y;
  P.x = fp32 ? (void*)c->d_xf : (void*)c->d_x;
  P.r = fp32 ? (void*)c->d_rf : (void*)c->d_r;
  P.b = fp32 ? (const void*)c->d_bf : (const void*)c->d_b;
  P.st = st;
  P.desc = desc;
  P.slotW = c->d_slotW;
  P.slotV = c->d_slotV;
  P.slot_stride = (long long)c->n * c->t;
  P.C = c->d_C;
  P.part_buf = c->d_partial;
  P.small = c->d_small;
  P.history = c->d_hist;
  P.rho_part = c->d_rho_part;
  P.beta_part = c->d_beta_part;
  // the step-level entry points (own state) never precondition
  P.prec = (c->prec_nb > 0 && st == c->d_st) ? 1 : 0;
  P.want_beta = (c->opts.variant == ECG_MSDO && !P.prec) ? 1 : 0;
  P.z = fp32 ? (void*)c->d_zf : (void*)c->d_z;
  P.block = (c->opts.block_residual && st == c->d_st) ? 1 : 0;
  P.Rb = c->d_Rb;
  P.wcap = kChunk;
  P.sre_src = 0;
  return P;
}

PrecSweep make_sweep(const ecg_ctx::Sweep& w, bool fp32) {
  PrecSweep S;
  S.blk = w.blk;
  S.lev = w.lev;
  S.rows = w.rows;
  S.cnt = w.cnt;
  S.col = w.col;
  S.val = fp32 ? (const void*)w.valf : (const void*)w.val;
  S.diag = fp32 ? (const void*)w.diagf : (const void*)w.diag;
  S.dep = w.dep;
  S.K = w.K;
  S.cpos = w.cpos;
  S.cq = w.cq;
  S.cblk = w.cblk;
  return S;
}

PrecP make_precp(const ecg_ctx* c, bool fp32) {
  PrecP Q;
  Q.nb = c->prec_nb;
  Q.local = c->prec_local;
  Q.maxw = c->prec_maxw;
  Q.qc = c->prec_qc;
  Q.f = make_sweep(c->pf, fp32);
  Q.b = make_sweep(c->pb, fp32);
  Q.part = c->d_ppart;
  return Q;
}

// Entries per row bound of the substitution kernels (0: any).
int prec_km(const ecg_ctx* c) {
  const int K = std::max(c->pf.K, c->pb.K);
  return K <= 2 ? 2 : (K <= 4 ? 4 : (K <= 8 ? 8 : 0));
}

template <typename T, int W>
void launch_prec(ecg_ctx* c, const KP& P, const PrecP& Q, int gw, const T* in, T* out, int w) {
  const dim3 grid(c->prec_nb, (std::max(W, w) + kPrecCols - 1) / kPrecCols);
  // level-local mode: two levels of kPrecCols columns in shared memory,
  // and in chunked mode the chunk buffers
  const size_t smem = Q.local ? 2 * (size_t)Q.maxw * kPrecCols * sizeof(T) +
                                    (Q.qc > 0 ? prec_chunk_bytes(Q.qc, std::max(Q.f.K, Q.b.K), (int)sizeof(T)) : 0)
                              : 0;
  switch (prec_km(c)) {
    case 2: k_prec_solve<T, W, 2><<<grid, kThreads, smem, c->stream>>>(P, Q, gw, in, out, w); break;
    case 4: k_prec_solve<T, W, 4><<<grid, kThreads, smem, c->stream>>>(P, Q, gw, in, out, w); break;
    case 8: k_prec_solve<T, W, 8><<<grid, kThreads, smem, c->stream>>>(P, Q, gw, in, out, w); break;
    default: k_prec_solve<T, W, 0><<<grid, kThreads, 0, c->stream>>>(P, Q, gw, in, out, w); break;
  }
}

// Row-CTAs for a window product with gy column chunks.
int window_gx(const ecg_ctx* c, int gy) {
  int target = 4 * c->num_sms;
  int g = (target + gy - 1) / gy;
  return std::max(1, std::min(c->gx, g));
}

void invalidate_graphs(ecg_ctx* c) {
  for (auto& g : c->gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

int ensure_part(ecg_ctx* c, size_t doubles) {
  if (doubles <= c->part_cap) return ECG_OK;
  invalidate_graphs(c);
  dfree(c->d_partial);
  c->part_cap = 0;
  int rc = dalloc(&c->d_partial, doubles);
  if (rc) return rc;
  c->part_cap = doubles;
  return ECG_OK;
}

int ensure_C(ecg_ctx* c, size_t doubles) {
  if (doubles <= c->C_cap) return ECG_OK;
  invalidate_graphs(c);
  dfree(c->d_C);
  c->C_cap = 0;
  int rc = dalloc(&c->d_C, doubles);
  if (rc) return rc;
  c->C_cap = doubles;
  return ECG_OK;
}

void prof_mark(ecg_ctx* c, int cls) {
  if (!c->profiling) return;
  if (c->pev_used >= c->pev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    c->pev.push_back(e);
    c->pev_class.push_back(-1);
  }
  cudaEventRecord(c->pev[c->pev_used], c->stream);
  c->pev_class[c->pev_used] = cls;
  c->pev_used++;
}

void prof_collect(ecg_ctx* c) {
  if (!c->profiling || c->pev_used < 2) {
    c->pev_used = 0;
    return;
  }
  cudaEventSynchronize(c->pev[c->pev_used - 1]);
  for (size_t i = 1; i < c->pev_used; i++) {
    int cls = c->pev_class[i];
    if (cls < 0) continue;  // -1 marks a start point
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->pev[i - 1], c->pev[i]) == cudaSuccess) {
      c->prof.ms[cls] += ms;
      c->prof.launches[cls] += 1;
    }
  }
  c->pev_used = 0;
}

// Reduce the gx per-CTA partials of nent small-matrix entries into
// P.small[kSmallG ..] (one warp per entry).
void reduce_small(ecg_ctx* c, const KP& P, int gw, int nent, int count = 0) {
  const int blocks = (nent * 32 + kThreads - 1) / kThreads;
  k_reduce_partials<<<blocks, kThreads, 0, c->stream>>>(P.st, gw, P.part_buf, count > 0 ? count : c->gx, nent,
                                                        P.small + kSmallG);
}

// Blocks per SM of a kernel at kThreads threads and smem bytes, times the
// SM count, at most gx (gx when the query fails).
int occupancy_grid(const ecg_ctx* c, const void* kernel, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return c->gx;
  }
  return std::max(1, std::min(c->gx, per_sm * c->num_sms));
}

// occupancy_grid through the context's cache: the CGS kernels' shared
// memory depends on the window size, so their grids are looked up per
// launch; enqueue_group fills the cache before it captures a graph.
int occ_grid_cached(ecg_ctx* c, const void* kernel, size_t smem) {
  for (const auto& e : c->occ)
    if (e.kernel == kernel && e.smem == smem) return e.grid;
  const int g = occupancy_grid(c, kernel, smem);
  c->occ.push_back({kernel, smem, g});
  return g;
}

// Grids of k_tdot_window and k_update: one wave at their occupancy.
template <typename T, int W>
void cgs_grids(ecg_ctx* c, int wcap, int& gt, int& gu) {
  gt = occ_grid_cached(c, (const void*)k_tdot_window<T, W>, smem_tdot<T, W>(wcap));
  gu = occ_grid_cached(c, (const void*)k_update<T, W>, smem_update<T, W>(wcap));
}

template <typename T>
void warm_cgs_grids(ecg_ctx* c, int W, int wcap) {
  int gt, gu;
  switch (W) {
    case 1: cgs_grids<T, 1>(c, wcap, gt, gu); break;
    case 2: cgs_grids<T, 2>(c, wcap, gt, gu); break;
    case 4: cgs_grids<T, 4>(c, wcap, gt, gu); break;
    case 8: cgs_grids<T, 8>(c, wcap, gt, gu); break;
    case 16: cgs_grids<T, 16>(c, wcap, gt, gu); break;
    case 32: cgs_grids<T, 32>(c, wcap, gt, gu); break;
    case 64: cgs_grids<T, 64>(c, wcap, gt, gu); break;
  }
}

template <int W>
void set_f32_grid(ecg_ctx* c, int wi) {
  const int a = occupancy_grid(c, (const void*)k_spmm_gram_rows<W, true>, smem_spmm_rows<W>());
  const int b = occupancy_grid(c, (const void*)k_spmm_gram_rows<W, false>, smem_spmm_rows<W>());
  c->gx_spmm32[wi] = std::min(a, b);
  c->gx_fin32[wi] = occupancy_grid(c, (const void*)k_final<float, W>, smem_final<float, W>());
  c->gx_gram32[wi] = occupancy_grid(c, (const void*)k_gram_self<float, W>, smem_gram_self<float, W>());
}

// The FP64 SpMM + Gram on q waits on its gathers between FMA phases; it
// runs at its full occupancy (8 CTAs per SM at t = 16), beyond gx, and at most
// one CTA per 32 rows.
template <int W>
void set_f64_spmm_grid(ecg_ctx* c) {
  int per_sm = 0;
  int g = c->gx;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_spmm_gram<double, W, true, false>, kThreads,
                                                    smem_spmm<double, W>()) == cudaSuccess &&
      per_sm > 0)
    g = std::max(1, std::min(per_sm * c->num_sms, (c->n + 31) / 32));
  else
    cudaGetLastError();
  c->gx_spmm64[width_index(W)] = std::max(g, 1);
}

void set_f32_grids(ecg_ctx* c) {
  for (int i = 0; i < 7; i++) c->gx_spmm32[i] = c->gx_fin32[i] = c->gx_gram32[i] = c->gx;
  set_f32_grid<4>(c, width_index(4));
  set_f32_grid<8>(c, width_index(8));
  set_f32_grid<16>(c, width_index(16));
  set_f64_spmm_grid<1>(c);
  set_f64_spmm_grid<2>(c);
  set_f64_spmm_grid<4>(c);
  set_f64_spmm_grid<8>(c);
  set_f64_spmm_grid<16>(c);
  set_f64_spmm_grid<32>(c);
  set_f64_spmm_grid<64>(c);
}

// Grid of the tensor-core kernels: two CTAs per SM, at most one per
// 128-row tile.
int tc_grid(const ecg_ctx* c) {
  return (int)std::max<long long>(1, std::min<long long>(2LL * c->num_sms, ((long long)c->n + 127) / 128));
}

// The CGS update X -= Q C (C in d_C or Cin): the tensor-core form where it
// applies (FP64, W = 16, at most 32 window columns, tensor_cores on), else
// the CUDA-core kernel.  The tensor-core form runs two CTAs per SM (each
// holds 256 of the SM's 512 TMEM columns).
// wmax is the most window columns the launch can see; the CUDA-core
// kernel's shared memory follows P.wcap, the size that kernel assumes.
template <typename T, int W>
void launch_update(ecg_ctx* c, const KP& P, T* X, const double* Cin, int wmax, int gup) {
  if constexpr (tc::update_tc_ok<T, W>(32)) {
    if (c->opts.tensor_cores && tc::update_tc_ok<T, W>(wmax)) {
      tc::k_update_tc<W><<<tc_grid(c), 256, tc::smem_update_tc<W>(), c->stream>>>(P, W, (double*)X, Cin);
      return;
    }
  }
  k_update<T, W><<<gup, kThreads, smem_update<T, W>(P.wcap), c->stream>>>(P, W, X, Cin);
}

// C = V^T B over the window (CGS coefficients) into Cout: the tensor-core
// form where it applies (FP64, W = 16, at most 32 window columns,
// tensor_cores on), else the CUDA-core kernel; then the fixed-order
// reduction of the per-CTA partials.
template <typename T, int W>
void launch_tdot(ecg_ctx* c, const KP& P, const T* B, double* Cout, int wmax, int gy, int gxw) {
  if constexpr (tc::tdot_tc_ok<T, W>(32)) {
    // FP64 with tensor_cores >= 1; the FP32 Grams of the mixed method only
    // with tensor_cores == 2 (slower than the CUDA-core FP32 kernel here)
    const bool want = sizeof(T) == 8 ? c->opts.tensor_cores >= 1 : c->opts.tensor_cores == 2;
    if (want && tc::tdot_tc_ok<T, W>(wmax) && gy == 1) {
      const int g = tc_grid(c);
      tc::k_tdot_tc<T, W><<<g, 256, tc::smem_tdot_tc<T, W>(), c->stream>>>(P, W, B);
      k_reduce_C<W><<<dim3((kChunk * W * 32 + kThreads - 1) / kThreads, 1), kThreads, 0, c->stream>>>(P, W, g, Cout);
      return;
    }
  }
  k_tdot_window<T, W><<<dim3(gxw, gy), kThreads, smem_tdot<T, W>(P.wcap), c->stream>>>(P, W, B);
  k_reduce_C<W><<<dim3((kChunk * W * 32 + kThreads - 1) / kThreads, gy), kThreads, 0, c->stream>>>(P, W, gxw, Cout);
}

// One iteration of the kernel chain for scalar type T and block width W.
template <typename T, int W>
int enqueue_iteration(ecg_ctx* c, int gy, int wcap) {
  cudaStream_t s = c->stream;
  const bool fp32 = sizeof(T) == 4;
  KP P = make_kp(c, c->d_st, c->d_desc, fp32);
  P.wcap = wcap;
  T* X = (T*)c->d_X;
  T* Y = (T*)c->d_Y;
  T* x = (T*)P.x;
  T* r = (T*)P.r;
  const bool pre = (c->opts.ortho == ECG_PRE_CHOLQR);
  int gtd, gup;
  cgs_grids<T, W>(c, wcap, gtd, gup);
  const int gxw = std::min(window_gx(c, gy), gtd);
  // the FP32 row-blocked kernels run one wave at their own occupancy
  const int gsp = F32Rows<T, W>::on ? c->gx_spmm32[width_index(W)] : c->gx;
  const int gfin = F32Rows<T, W>::on ? c->gx_fin32[width_index(W)] : c->gx;
  const int ggs = F32Rows<T, W>::on ? c->gx_gram32[width_index(W)] : c->gx;
  const long long tot = (long long)c->n * W;
  // the generator is a no-op on the SRE iterations of the FP32 and
  // preconditioned solves, where the cost of a launch is its CTAs: two per SM,
  // grid-stride otherwise
  const int ggen = (int)std::max<long long>(1, std::min<long long>((tot + kThreads - 1) / kThreads, 2LL * c->num_sms));
  prof_mark(c, -1);
  if (c->prec_nb > 0) {  // preconditioned generators (Section 3, Algorithm 5)
    const PrecP Q = make_precp(c, fp32);
    launch_prec<T, W>(c, P, Q, W, nullptr, nullptr, 0);
    if (c->opts.variant == ECG_MSDO)
      k_reduce_partials<<<(W * 32 + kThreads - 1) / kThreads, kThreads, 0, s>>>(P.st, W, Q.part, c->prec_nb, W,
                                                                               P.small + kSmallBe);
    prof_mark(c, 10);
  }
  P.sre_src = 1;  // an SRE block goes from V_{k-1} straight into the first CGS pass
  k_generate<T, W><<<ggen, kThreads, 0, s>>>(P, W);
  prof_mark(c, 0);
  for (int pass = 0; pass < 2; pass++) {
    P.sre_src = (pass == 0) ? 1 : 0;
    launch_tdot<T, W>(c, P, X, c->d_C, wcap, gy, gxw);
    prof_mark(c, 1);
    launch_update<T, W>(c, P, X, c->d_C, wcap, gup);
    prof_mark(c, 2);
  }
  if (pre && !fp32) {
    // FP64: q = X R_e^{-1} explicitly, then the A-CholQR step on q (the
    // SpMM's FP64 FMAs are its bound, and a per-row transform would double them)
    k_gram_self<T, W><<<ggs, kThreads, smem_gram_self<T, W>(), s>>>(P, W, X);
    prof_mark(c, 3);
    reduce_small(c, P, W, W * (W + 1) / 2, ggs);
    k_small_e<W><<<1, kThreads, smem_small<W>(), s>>>(P, W, c->gx);
    prof_mark(c, 4);
    k_tri_right<T, W><<<c->gx, kThreads, smem_tri_right<T, W>(), s>>>(P, W, X);
    prof_mark(c, 3);
    const int gsp64 = c->gx_spmm64[width_index(W)];
    k_spmm_gram<T, W, true, false><<<gsp64, kThreads, smem_spmm<T, W>(), s>>>(P, W, X, Y);
    prof_mark(c, 5);
    reduce_small(c, P, W, W * (W + 1) / 2 + W, gsp64);
    k_small_a<W, false><<<1, kThreads, smem_small<W>(), s>>>(P, W, gsp64);
  } else if (pre) {
    k_gram_self<T, W><<<ggs, kThreads, smem_gram_self<T, W>(), s>>>(P, W, X);
    prof_mark(c, 3);
    reduce_small(c, P, W, W * (W + 1) / 2, ggs);
    k_small_e<W><<<1, kThreads, smem_small<W>(), s>>>(P, W, c->gx);
    prof_mark(c, 4);
    if constexpr (F32Rows<T, W>::on)
      k_spmm_gram_rows<W, true><<<gsp, kThreads, smem_spmm_rows<W>(), s>>>(P, W, X, Y);
    else
      k_spmm_gram<T, W, true, true><<<gsp, kThreads, smem_spmm<T, W>(), s>>>(P, W, X, Y);
    prof_mark(c, 5);
    reduce_small(c, P, W, W * (W + 1) / 2 + W, gsp);
    k_small_a<W, true><<<1, kThreads, smem_small<W>(), s>>>(P, W, gsp);
  } else {
    if constexpr (F32Rows<T, W>::on)
      k_spmm_gram_rows<W, false><<<gsp, kThreads, smem_spmm_rows<W>(), s>>>(P, W, X, Y);
    else
      k_spmm_gram<T, W, true, false><<<gsp, kThreads, smem_spmm<T, W>(), s>>>(P, W, X, Y);
    prof_mark(c, 5);
    reduce_small(c, P, W, W * (W + 1) / 2 + W, gsp);
    k_small_a<W, false><<<1, kThreads, smem_small<W>(), s>>>(P, W, gsp);
  }
  prof_mark(c, 6);
  int gf = gfin;  // CTAs that write rho / beta partials
  bool fin_tc = false;
  if constexpr (tc::final_tc_ok<T, W>()) {
    // the block-residual mode takes rho from k_block_update's c->gx partials
    if (c->opts.tensor_cores && !P.block) {
      fin_tc = true;
      gf = tc_grid(c);
      tc::k_final_tc<W><<<gf, 256, tc::smem_final_tc<W>(), s>>>(P, W, (const double*)X, (const double*)Y, nullptr,
                                                              nullptr, (double*)x, (double*)r);
    }
  }
  if (!fin_tc) k_final<T, W><<<gfin, kThreads, smem_final<T, W>(), s>>>(P, W, X, Y, nullptr, nullptr, x, r);
  if constexpr (sizeof(T) == 8) {
    if (P.block) {  // block-residual mode: alpha = W_k^T R, R -= V_k alpha, x, r = R 1
      k_block_alpha<W><<<c->gx, kThreads, 0, s>>>(P, W);
      k_reduce_partials<<<(W * W * 32 + kThreads - 1) / kThreads, kThreads, 0, s>>>(P.st, W, P.part_buf, c->gx,
                                                                                   W * W, P.small + kSmallAb);
      k_block_update<W><<<c->gx, kThreads, 0, s>>>(P, W);
    }
  }
  prof_mark(c, 7);
  k_finish<<<1, kThreads, 0, s>>>(P, W, gf, (int)sizeof(T));
  prof_mark(c, 8);
  CK(cudaGetLastError());
  return ECG_OK;
}

template <typename T>
int enqueue_iteration_w(ecg_ctx* c, int W, int gy, int wcap) {
  switch (W) {
    case 1: return enqueue_iteration<T, 1>(c, gy, wcap);
    case 2: return enqueue_iteration<T, 2>(c, gy, wcap);
    case 4: return enqueue_iteration<T, 4>(c, gy, wcap);
    case 8: return enqueue_iteration<T, 8>(c, gy, wcap);
    case 16: return enqueue_iteration<T, 16>(c, gy, wcap);
    case 32: return enqueue_iteration<T, 32>(c, gy, wcap);
    case 64: return enqueue_iteration<T, 64>(c, gy, wcap);
  }
  return ECG_EINVAL;
}

// Most window columns for an iteration index bounded by khost (every
// stored block is at most t wide).
long long window_cols(const ecg_ctx* c, int cap, int khost) {
  long long blocks = std::min<long long>(cap, std::max(0, khost - 1));
  return blocks * c->t;
}
// Column chunks of that window.
int window_chunks(const ecg_ctx* c, int cap, int khost) {
  return (int)std::max<long long>(1, (window_cols(c, cap, khost) + kChunk - 1) / kChunk);
}

// Issue `iters` iterations of width W, through a captured graph when the
// window size is fixed and the group is a full one.
int enqueue_group(ecg_ctx* c, bool fp32, int W, int iters, int cap, int khost) {
  const bool fixed = (c->opts.trunc > 0);
  const int kb = fixed ? cap + 1 : khost + iters;
  const int gy = window_chunks(c, cap, kb);
  const int wcap = (int)std::min<long long>(kChunk, std::max<long long>(1, window_cols(c, cap, kb)));
  auto one = [&]() {
    return fp32 ? enqueue_iteration_w<float>(c, W, gy, wcap) : enqueue_iteration_w<double>(c, W, gy, wcap);
  };
  if (fp32) warm_cgs_grids<float>(c, W, wcap);  // no occupancy queries inside a capture
  else warm_cgs_grids<double>(c, W, wcap);
  if (c->opts.use_graph && fixed && !c->profiling && iters == c->opts.check_every) {
    const int wi = width_index(W) + (fp32 ? 7 : 0);
    if (!c->gexec[wi] || c->graph_iters[wi] != iters) {
      if (c->gexec[wi]) cudaGraphExecDestroy(c->gexec[wi]);
      c->gexec[wi] = nullptr;
      cudaGraph_t g;
      CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      int rc = ECG_OK;
      for (int i = 0; i < iters && rc == ECG_OK; i++) rc = one();
      cudaError_t e = cudaStreamEndCapture(c->stream, &g);
      if (rc) return rc;
      CK(e);
      e = cudaGraphInstantiate(&c->gexec[wi], g, 0);
      cudaGraphDestroy(g);
      CK(e);
      c->graph_iters[wi] = iters;
    }
    CK(cudaGraphLaunch(c->gexec[wi], c->stream));
    return ECG_OK;
  }
  for (int i = 0; i < iters; i++) {
    int rc = one();
    if (rc) return rc;
  }
  return ECG_OK;
}

// One enlarged CG solve on the device (Algorithms 1-4): the right-hand side
// is in b (FP64 d_b or FP32 d_bf) and the initial iterate in x; have_x0 =
// false means x = 0 (already cleared).  Writes rho_k to history[hist_off+k]
// and the final state to *fin.
int run_solve(ecg_ctx* c, bool fp32, int kmax, int cap, double eps, int hist_off, bool have_x0, DevState* fin) {
  cudaStream_t s = c->stream;
  const int t = c->t;
  DevState init;
  std::memset(&init, 0, sizeof(init));
  init.kmax = kmax;
  init.variant = c->opts.variant;
  init.cap = cap;
  init.t = t;
  init.eps = eps;
  init.switch_tol = c->opts.switch_tol;
  init.breakdown_ratio = fp32 ? kBreakdownFP32 : kBreakdownFP64;
  init.hist_off = hist_off;
  init.restart_every = c->opts.restart_every;
  init.restart_tol = c->opts.restart_tol;
  init.restart_max = c->opts.restart_max;
  init.restart_at_switch = c->opts.restart_at_switch;
  // an FP32 round that stalls above its target (its floor lies near FP32
  // rounding times the conditioning) ends after kStagIters iterations without
  // a 1% smaller residual, instead of running to k_max
  init.stag_iters = fp32 ? kStagIters : 0;
  init.rho_best = HUGE_VAL;
  CK(cudaMemcpyAsync(c->d_st, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  KP P = make_kp(c, c->d_st, c->d_desc, fp32);
  prof_mark(c, -1);
  if (fp32) {
    k_residual<float><<<c->gx, kThreads, 0, s>>>(P, have_x0 ? c->d_xf : nullptr, c->d_rf, c->d_bf, c->d_rho_part,
                                                 nullptr);
  } else {
    k_residual<double><<<c->gx, kThreads, 0, s>>>(P, have_x0 ? c->d_x : nullptr, c->d_r, c->d_b, c->d_rho_part,
                                                  c->d_bb_part);
  }
  // ECG_STOP_B on the FP64 solve; the FP32 inner solves of mixed precision
  // get their tolerance from the outer loop
  k_start<<<1, kThreads, 0, s>>>(P, c->gx, (!fp32 && c->opts.stop_rule == ECG_STOP_B) ? c->d_bb_part : nullptr);
  if (P.block) {  // R_0 = [T^t(r_0)]
    const long long tot = (long long)c->n * c->t;
    const int g = (int)std::max<long long>(1, std::min<long long>((tot + 255) / 256, 8LL * c->num_sms));
    k_block_split<<<g, 256, 0, s>>>(P, c->d_r, c->d_Rb);
  }
  prof_mark(c, 9);
  CK(cudaGetLastError());
  // Groups of check_every iterations, polled one group behind.  The host
  // never issues iteration k_max or later; after the flexible switch it
  // rewinds its count to the device's k (the group in flight, issued for
  // the old width, does nothing).
  const int chunk = c->opts.check_every;
  int W = t;
  int khost = 1;  // next iteration the host issues
  int rc;
  auto issue = [&](int slot) -> int {
    const int nit = std::min(chunk, kmax - khost);
    if (nit > 0) {
      int r2 = enqueue_group(c, fp32, W, nit, cap, khost);
      if (r2) return r2;
      khost += nit;
    }
    CK(cudaMemcpyAsync(&c->h_flags[slot], c->d_st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(c->ev[slot], s));
    return ECG_OK;
  };
  if ((rc = issue(0))) return rc;
  int cur = 0;
  long long polls = 0;
  const long long max_polls = 4LL * ((long long)kmax / chunk + 4);
  while (true) {
    if ((rc = issue(1 - cur))) return rc;
    CK(cudaEventSynchronize(c->ev[cur]));
    const DevState f = c->h_flags[cur];
    if (f.stop) break;
    if (f.width != W) {
      if (width_index(f.width) < 0) return ECG_ECUDA;
      W = f.width;
      khost = f.k;
    }
    cur = 1 - cur;
    if (++polls > max_polls) {  // the device never stopped: not expected
      cudaStreamSynchronize(s);
      return ECG_ECUDA;
    }
  }
  CK(cudaMemcpyAsync(fin, c->d_st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return ECG_OK;
}

// ||b - A x||^2 and ||b||^2 in FP64 (r = b - A x kept in d_r).
int true_residual(ecg_ctx* c, bool keep_r, double* rr, double* bb) {
  cudaStream_t s = c->stream;
  KP P = make_kp(c, c->d_st, c->d_desc, false);
  k_residual<double><<<c->gx, kThreads, 0, s>>>(P, c->d_x, keep_r ? c->d_r : nullptr, c->d_b, c->d_rho_part,
                                                c->d_bb_part);
  CK(cudaGetLastError());
  std::vector<double> prr(c->gx), pbb(c->gx);
  CK(cudaMemcpyAsync(prr.data(), c->d_rho_part, sizeof(double) * c->gx, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(pbb.data(), c->d_bb_part, sizeof(double) * c->gx, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double a = 0.0, bsum = 0.0;
  for (int i = 0; i < c->gx; i++) {
    a += prr[i];
    bsum += pbb[i];
  }
  *rr = a;
  *bb = bsum;
  return ECG_OK;
}

int validate_opts(const ecg_opts* o, int t) {
  if (o->variant < 0 || o->variant > 2) return ECG_EINVAL;
  if (o->trunc < 0) return ECG_EINVAL;
  if (o->ortho < 0 || o->ortho > 1) return ECG_EINVAL;
  if (!(o->switch_tol >= 0.0)) return ECG_EINVAL;
  if (o->switch_tol > 0.0 && (t % 2 != 0)) return ECG_EINVAL;
  if (o->check_every < 1) return ECG_EINVAL;
  if (o->precision < 0 || o->precision > 1) return ECG_EINVAL;
  if (!(o->inner_tol >= 0.0 && o->inner_tol < 1.0)) return ECG_EINVAL;
  if (o->restart_every == 1 || o->restart_every < 0) return ECG_EINVAL;
  if (!(o->restart_tol >= 0.0) || o->restart_max < 0) return ECG_EINVAL;
  if (o->restart_at_switch && !(o->switch_tol > 0.0)) return ECG_EINVAL;
  if (o->block_residual != 0 && o->block_residual != 1) return ECG_EINVAL;
  if (o->stop_rule != ECG_STOP_R0 && o->stop_rule != ECG_STOP_B) return ECG_EINVAL;
  if (o->tensor_cores < 0 || o->tensor_cores > 2) return ECG_EINVAL;
  if (o->block_residual && (o->variant != ECG_SRE || o->switch_tol > 0.0 || o->precision != ECG_FP64 ||
                            o->restart_every || o->restart_tol > 0.0))
    return ECG_EINVAL;
  return ECG_OK;
}

// Launch helpers for the step-level entry points (FP64, width dispatch).
template <int W>
struct Ops {
  static void generate(ecg_ctx* c, KP P) {
    long long tot = (long long)c->n * W;
    int g = (int)std::max<long long>(1, std::min<long long>((tot + kThreads - 1) / kThreads, 8LL * c->num_sms));
    k_generate<double, W><<<g, kThreads, 0, c->stream>>>(P, W);
  }
  static void spmm(ecg_ctx* c, KP P, const double* X, double* Y) {
    k_spmm_gram<double, W, false, false><<<c->gx, kThreads, smem_spmm<double, W>(), c->stream>>>(P, W, X, Y);
  }
  static void tdot(ecg_ctx* c, KP P, int gw, const double* B, int gy, double* Cout, int wtot) {
    int gxw = window_gx(c, gy);
    launch_tdot<double, W>(c, P, B, Cout, wtot <= 32 ? wtot : kChunk, gy, gxw);
  }
  static void update(ecg_ctx* c, KP P, double* X, const double* Cin, int wtot) {
    launch_update<double, W>(c, P, X, Cin, wtot <= 32 ? wtot : kChunk, c->gx);
  }
  static void orth(ecg_ctx* c, KP P, double* Wio, double* V, double* x, double* r) {
    const bool pre = (c->opts.ortho == ECG_PRE_CHOLQR);
    double* Y = c->d_Y;
    if (pre) {
      k_gram_self<double, W><<<c->gx, kThreads, smem_gram_self<double, W>(), c->stream>>>(P, W, Wio);
      reduce_small(c, P, W, W * (W + 1) / 2);
      k_small_e<W><<<1, kThreads, smem_small<W>(), c->stream>>>(P, W, c->gx);
      k_tri_right<double, W><<<c->gx, kThreads, smem_tri_right<double, W>(), c->stream>>>(P, W, Wio);
      k_spmm_gram<double, W, true, false><<<c->gx, kThreads, smem_spmm<double, W>(), c->stream>>>(P, W, Wio, Y);
      reduce_small(c, P, W, W * (W + 1) / 2 + W);
      k_small_a<W, false><<<1, kThreads, smem_small<W>(), c->stream>>>(P, W, c->gx);
    } else {
      k_spmm_gram<double, W, true, false><<<c->gx, kThreads, smem_spmm<double, W>(), c->stream>>>(P, W, Wio, Y);
      reduce_small(c, P, W, W * (W + 1) / 2 + W);
      k_small_a<W, false><<<1, kThreads, smem_small<W>(), c->stream>>>(P, W, c->gx);
    }
    k_final<double, W><<<c->gx, kThreads, smem_final<double, W>(), c->stream>>>(P, W, Wio, Y, Wio, V, x, r);
  }
};

template <template <int> class F, typename... Args>
int dispatch_w(int w, Args... args) {
  switch (w) {
    case 1: F<1>::run(args...); return ECG_OK;
    case 2: F<2>::run(args...); return ECG_OK;
    case 4: F<4>::run(args...); return ECG_OK;
    case 8: F<8>::run(args...); return ECG_OK;
    case 16: F<16>::run(args...); return ECG_OK;
    case 32: F<32>::run(args...); return ECG_OK;
    case 64: F<64>::run(args...); return ECG_OK;
  }
  return ECG_EINVAL;
}

template <int W> struct RunGenerate { static void run(ecg_ctx* c, KP P) { Ops<W>::generate(c, P); } };
template <int W> struct RunSpmm { static void run(ecg_ctx* c, KP P, const double* X, double* Y) { Ops<W>::spmm(c, P, X, Y); } };
template <int W> struct RunTdot {
  static void run(ecg_ctx* c, KP P, int gw, const double* B, int gy, double* Cout, int wtot) {
    Ops<W>::tdot(c, P, gw, B, gy, Cout, wtot);
  }
};
template <int W> struct RunUpdate {
  static void run(ecg_ctx* c, KP P, double* X, const double* Cin, int wtot) { Ops<W>::update(c, P, X, Cin, wtot); }
};
template <int W> struct RunOrth {
  static void run(ecg_ctx* c, KP P, double* Wio, double* V, double* x, double* r) { Ops<W>::orth(c, P, Wio, V, x, r); }
};

// ------------------------------------------------ block Jacobi preconditioner

void free_sweep(ecg_ctx::Sweep& w) {
  dfree(w.blk);
  dfree(w.lev);
  dfree(w.rows);
  dfree(w.cnt);
  dfree(w.col);
  dfree(w.map);
  dfree(w.val);
  dfree(w.diag);
  dfree(w.valf);
  dfree(w.diagf);
  dfree(w.dep);
  dfree(w.cpos);
  dfree(w.cq);
  dfree(w.cblk);
  w.K = 1;
}

void prec_free(ecg_ctx* c) {
  invalidate_graphs(c);
  c->prec_nb = 0;
  c->prec_local = 0;
  c->prec_maxw = 0;
  c->prec_qc = 0;
  free_sweep(c->pf);
  free_sweep(c->pb);
  dfree(c->d_lp);
  dfree(c->d_lc);
  dfree(c->d_lv);
  dfree(c->d_ld);
  dfree(c->d_z);
  dfree(c->d_zf);
  dfree(c->d_ppart);
  dfree(c->d_pflag);
}

// Level lists of one substitution: rows grouped by block, then by level,
// increasing row order inside a level.  blk[b] .. blk[b+1] index lev, and
// lev[l] .. lev[l+1] index rows.
void level_lists(int n, int nb, const std::vector<int>& pb, const std::vector<int>& level, std::vector<int>& blk,
                 std::vector<int>& lev, std::vector<int>& rows) {
  std::vector<int> nlev(nb, 0);
  for (int i = 0; i < n; i++) nlev[pb[i]] = std::max(nlev[pb[i]], level[i] + 1);
  blk.assign(nb + 1, 0);
  for (int b = 0; b < nb; b++) blk[b + 1] = blk[b] + nlev[b];
  lev.assign(blk[nb] + 1, 0);
  for (int i = 0; i < n; i++) lev[blk[pb[i]] + level[i] + 1]++;
  for (int l = 0; l < blk[nb]; l++) lev[l + 1] += lev[l];
  std::vector<int> fill(lev.begin(), lev.end() - 1);
  rows.assign(n, 0);
  for (int i = 0; i < n; i++) rows[fill[blk[pb[i]] + level[i]]++] = i;
}

template <typename T>
int upload(T** d, const std::vector<T>& h) {
  int rc = dalloc(d, h.size());
  if (rc) return rc;
  if (!h.empty()) CK(cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return ECG_OK;
}

// Symbolic analysis on the host (pattern, transpose, level lists), then the
// IC(0) factorisation on the device.
int prec_build(ecg_ctx* c, const std::vector<int>& pb, int nb) {
  const int n = c->n;
  std::vector<int> rp(n + 1), ci(c->nnz), pt(n);
  CK(cudaMemcpy(rp.data(), c->d_rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(ci.data(), c->d_col, sizeof(int) * c->nnz, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(pt.data(), c->d_pmap, sizeof(int) * n, cudaMemcpyDeviceToHost));
  // every block non-empty and inside one subdomain, so that
  // L^{-T}[T(L^{-1} r)] = [T(M^{-1} r)] (and likewise for T^{t/2})
  std::vector<int> owner(nb, -1);
  for (int i = 0; i < n; i++) {
    if (pb[i] < 0 || pb[i] >= nb) return ECG_EINVAL;
    if (owner[pb[i]] < 0) owner[pb[i]] = pt[i];
    else if (owner[pb[i]] != pt[i]) return ECG_EINVAL;
  }
  for (int b = 0; b < nb; b++)
    if (owner[b] < 0) return ECG_EINVAL;
  // pattern of L: columns j < i of row i in the same block
  std::vector<int> lp(n + 1, 0), lc;
  lc.reserve((size_t)c->nnz / 2 + 1);
  std::vector<int> row;
  for (int i = 0; i < n; i++) {
    row.clear();
    for (int a = rp[i]; a < rp[i + 1]; a++) {
      const int j = ci[a];
      if (j < i && pb[j] == pb[i]) row.push_back(j);
    }
    std::sort(row.begin(), row.end());
    row.erase(std::unique(row.begin(), row.end()), row.end());
    lc.insert(lc.end(), row.begin(), row.end());
    lp[i + 1] = (int)lc.size();
  }
  const int nnzl = lp[n];
  // L^T rows (entries of column i of L), with the map to L's entries
  std::vector<int> up(n + 1, 0), uc(nnzl), umap(nnzl);
  for (int e = 0; e < nnzl; e++) up[lc[e] + 1]++;
  for (int i = 0; i < n; i++) up[i + 1] += up[i];
  {
    std::vector<int> fill(up.begin(), up.end() - 1);
    for (int i = 0; i < n; i++)
      for (int e = lp[i]; e < lp[i + 1]; e++) {
        const int q = fill[lc[e]]++;
        uc[q] = i;
        umap[q] = e;
      }
  }
  std::vector<int> levf(n, 0), levb(n, 0);
  for (int i = 0; i < n; i++) {
    int l = 0;
    for (int e = lp[i]; e < lp[i + 1]; e++) l = std::max(l, levf[lc[e]] + 1);
    levf[i] = l;
  }
  for (int i = n - 1; i >= 0; i--) {
    int l = 0;
    for (int e = up[i]; e < up[i + 1]; e++) l = std::max(l, levb[uc[e]] + 1);
    levb[i] = l;
  }
  std::vector<int> fblk, flev, frows, bblk, blev, brows;
  level_lists(n, nb, pb, levf, fblk, flev, frows);
  level_lists(n, nb, pb, levb, bblk, blev, brows);
  // level-ordered ELL of both sweeps; map = index of the entry in L's rows
  auto ell = [&](const std::vector<int>& rows, const std::vector<int>& ptr, const std::vector<int>& cols,
                 const std::vector<int>* emap, int& K, std::vector<int>& cnt, std::vector<int>& col,
                 std::vector<int>& map) {
    K = 1;
    for (int i = 0; i < n; i++) K = std::max(K, ptr[i + 1] - ptr[i]);
    cnt.assign(n, 0);
    col.assign((size_t)n * K, 0);
    map.assign((size_t)n * K, 0);
    for (int q = 0; q < n; q++) {
      const int i = rows[q];
      cnt[q] = ptr[i + 1] - ptr[i];
      for (int k = 0; k < cnt[q]; k++) {
        const int e = ptr[i] + k;
        col[(size_t)q * K + k] = cols[e];
        map[(size_t)q * K + k] = emap ? (*emap)[e] : e;
      }
    }
  };
  std::vector<int> fcnt, fcol, fmap, bcnt, bcol, bmap;
  int Kf = 1, Kb = 1;
  ell(frows, lp, lc, nullptr, Kf, fcnt, fcol, fmap);
  ell(brows, up, uc, &umap, Kb, bcnt, bcol, bmap);
  // Level-local mode: every entry references a row exactly one level
  // before (true for the lexicographic order of 5- and 7-point blocks);
  // dep holds that row's index inside its level.
  auto local_deps = [&](const std::vector<int>& level, const std::vector<int>& blk, const std::vector<int>& lev,
                        const std::vector<int>& rows, const std::vector<int>& cnt, const std::vector<int>& col, int K,
                        std::vector<int>& dep, int& maxw) {
    std::vector<int> loc(n);
    maxw = 0;
    for (int b = 0; b < nb; b++)
      for (int l = blk[b]; l < blk[b + 1]; l++) {
        maxw = std::max(maxw, lev[l + 1] - lev[l]);
        for (int q = lev[l]; q < lev[l + 1]; q++) loc[rows[q]] = q - lev[l];
      }
    dep.assign((size_t)n * K, 0);
    bool ok = true;
    for (int q = 0; q < n && ok; q++) {
      const int i = rows[q];
      for (int k = 0; k < cnt[q]; k++) {
        const int j = col[(size_t)q * K + k];
        if (level[j] != level[i] - 1) {
          ok = false;
          break;
        }
        dep[(size_t)q * K + k] = loc[j];
      }
    }
    return ok;
  };
  std::vector<int> fdep, bdep;
  int mwf = 0, mwb = 0;
  const bool lf = local_deps(levf, fblk, flev, frows, fcnt, fcol, Kf, fdep, mwf);
  const bool lb = local_deps(levb, bblk, blev, brows, bcnt, bcol, Kb, bdep, mwb);
  const int maxw = std::max(mwf, mwb);
  // two levels of kPrecCols FP64 columns within the default 48 KB
  const bool local = lf && lb && Kf <= 8 && Kb <= 8 && 2 * (size_t)maxw * kPrecCols * sizeof(double) <= 48 * 1024;
  const bool mixed = (c->opts.precision == ECG_MIXED);
  auto put_sweep = [&](ecg_ctx::Sweep& w, const std::vector<int>& blk, const std::vector<int>& lev,
                       const std::vector<int>& rows, const std::vector<int>& cnt, const std::vector<int>& col,
                       const std::vector<int>& map, int K) {
    int rc;
    w.K = K;
    if ((rc = upload(&w.blk, blk)) || (rc = upload(&w.lev, lev)) || (rc = upload(&w.rows, rows)) ||
        (rc = upload(&w.cnt, cnt)) || (rc = upload(&w.col, col)) || (rc = upload(&w.map, map)) ||
        (rc = dalloc(&w.val, col.size())) || (rc = dalloc(&w.diag, (size_t)n)))
      return rc;
    if (mixed && ((rc = dalloc(&w.valf, col.size())) || (rc = dalloc(&w.diagf, (size_t)n)))) return rc;
    return ECG_OK;
  };
  int rc;
  if ((rc = put_sweep(c->pf, fblk, flev, frows, fcnt, fcol, fmap, Kf)) ||
      (rc = put_sweep(c->pb, bblk, blev, brows, bcnt, bcol, bmap, Kb)) || (rc = upload(&c->d_lp, lp)) ||
      (rc = upload(&c->d_lc, lc)) || (rc = dalloc(&c->d_lv, (size_t)nnzl)) || (rc = dalloc(&c->d_ld, (size_t)n)) ||
      (rc = dalloc(&c->d_z, (size_t)n)) || (rc = dalloc(&c->d_ppart, (size_t)nb * 64)) ||
      (rc = dalloc(&c->d_pflag, (size_t)1)))
    return rc;
  if (mixed && (rc = dalloc(&c->d_zf, (size_t)n))) return rc;
  if (local && ((rc = upload(&c->pf.dep, fdep)) || (rc = upload(&c->pb.dep, bdep)))) return rc;
  // Chunked level-local mode: chunks of consecutive levels of at most qc
  // positions, qc chosen so that the FP64 chunk buffers and the two level
  // buffers stay near 104 KB (two CTAs per SM with the static buffers).
  int qc = 0;
  if (local) {
    const int K = std::max(Kf, Kb);
    const size_t fixed = 2 * (size_t)maxw * kPrecCols * sizeof(double);
    const size_t budget = 104 * 1024;
    const size_t per = sizeof(double) * (1 + K + kPrecCols) + sizeof(int) * (2 + K);
    const size_t extra = prec_chunk_bytes(0, K, (int)sizeof(double)) + 112;  // level bounds, slack, rounding
    if (budget > fixed + extra) qc = (int)std::min<size_t>(4096, (budget - fixed - extra) / per);
    if (qc < maxw) qc = 0;
  }
  auto chunks = [&](const std::vector<int>& blk, const std::vector<int>& lev, ecg_ctx::Sweep& w) {
    std::vector<int> cpos, cq, cblk(nb + 1, 0);
    for (int b = 0; b < nb; b++) {
      cblk[b] = (int)cpos.size();
      int l = blk[b];
      while (l < blk[b + 1]) {
        const int start = l;
        int rows = 0;
        while (l < blk[b + 1] && l - start < kChunkLevels && rows + (lev[l + 1] - lev[l]) <= qc) {
          rows += lev[l + 1] - lev[l];
          l++;
        }
        cpos.push_back(start);
        cq.push_back(lev[start]);
      }
    }
    cblk[nb] = (int)cpos.size();
    cpos.push_back(blk[nb]);
    cq.push_back(lev[blk[nb]]);
    int r;
    if ((r = upload(&w.cpos, cpos)) || (r = upload(&w.cq, cq)) || (r = upload(&w.cblk, cblk))) return r;
    return (int)ECG_OK;
  };
  if (qc > 0 && ((rc = chunks(fblk, flev, c->pf)) || (rc = chunks(bblk, blev, c->pb)))) return rc;
  c->prec_qc = qc;
  c->prec_local = local ? 1 : 0;
  c->prec_maxw = local ? maxw : 0;
  c->prec_nb = nb;
  const PrecP Q = make_precp(c, false);
  CK(cudaMemsetAsync(c->d_pflag, 0, sizeof(int), c->stream));
  k_ic0_factor<<<nb, kThreads, 0, c->stream>>>(Q.f, c->d_lp, c->d_lc, c->d_rowptr, c->d_col, c->d_val, c->d_lv,
                                               c->d_ld, c->d_pflag);
  for (ecg_ctx::Sweep* w : {&c->pf, &c->pb}) {
    const int nent = n * w->K;
    const int g = std::max(1, std::min(8 * c->num_sms, (nent + 255) / 256));
    k_prec_gather<<<g, 256, 0, c->stream>>>(n, nent, w->map, w->rows, c->d_lv, c->d_ld, w->val, w->diag, w->valf,
                                            w->diagf);
  }
  CK(cudaGetLastError());
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, c->d_pflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (flag) return ECG_ENOTSPD;
  return ECG_OK;
}

template <int W> struct RunPrec {
  static void run(ecg_ctx* c, KP P, const double* in, double* out, int w) {
    launch_prec<double, W>(c, P, make_precp(c, false), W, in, out, w);
  }
};

DevState op_state(const ecg_ctx* c, int width, int nq, int gen) {
  DevState s;
  std::memset(&s, 0, sizeof(s));
  s.k = 1;
  s.width = width;
  s.gen = gen;
  s.nq = nq;
  s.cap = nq;
  s.t = c->t;
  s.kmax = 2;
  s.variant = c->opts.variant;
  s.eps = 0.0;
  s.breakdown_ratio = kBreakdownFP64;
  return s;
}

int put_op_state(ecg_ctx* c, const DevState& s) {
  CK(cudaMemcpyAsync(c->d_opst, &s, sizeof(s), cudaMemcpyHostToDevice, c->stream));
  // the host copy is a stack temporary: finish the copy before returning
  CK(cudaStreamSynchronize(c->stream));
  return ECG_OK;
}

int ensure_opdesc(ecg_ctx* c, int m) {
  if (m <= c->opdesc_cap) return ECG_OK;
  dfree(c->d_opdesc);
  c->opdesc_cap = 0;
  int rc = dalloc(&c->d_opdesc, (size_t)m);
  if (rc) return rc;
  c->opdesc_cap = m;
  return ECG_OK;
}

int put_op_desc(ecg_ctx* c, const std::vector<BlockDesc>& d) {
  int rc = ensure_opdesc(c, (int)d.size());
  if (rc) return rc;
  CK(cudaMemcpyAsync(c->d_opdesc, d.data(), d.size() * sizeof(BlockDesc), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ECG_OK;
}

int finish_op(ecg_ctx* c, int* status) {
  CK(cudaGetLastError());
  DevState s;
  CK(cudaMemcpyAsync(&s, c->d_opst, sizeof(s), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (status) *status = s.stop ? s.status : ECG_OK;
  return ECG_OK;
}

}  // namespace

// ============================================================== C ABI

extern "C" {

void ecg_default_opts(ecg_opts* o) {
  if (!o) return;
  o->variant = ECG_SRE;
  o->trunc = 0;
  o->switch_tol = 0.0;
  o->ortho = ECG_PRE_CHOLQR;
  o->check_every = 16;
  o->use_graph = 1;
  o->precision = ECG_FP64;
  o->inner_tol = 1e-5;
  o->restart_every = 0;
  o->restart_tol = 0.0;
  o->restart_max = 0;
  o->restart_at_switch = 0;
  o->block_residual = 0;
  o->stop_rule = ECG_STOP_R0;
  o->tensor_cores = 1;
  o->stream = nullptr;
}

const char* ecg_strerror(int code) {
  switch (code) {
    case ECG_OK: return "converged";
    case ECG_ENOCONV: return "iteration limit reached before the tolerance";
    case ECG_EINVAL: return "invalid argument";
    case ECG_ENOMEM: return "out of memory";
    case ECG_ECUDA: return "CUDA error";
    case ECG_EBREAKDOWN: return "block became numerically rank deficient (breakdown)";
    case ECG_ENOTSPD: return "matrix has a non-positive diagonal entry";
    case ECG_ETIMEOUT: return "a bounded device-side wait ran out";
  }
  return "unknown status";
}

void ecg_destroy(ecg_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->dev);
  if (c->stream) cudaStreamSynchronize(c->stream);
  invalidate_graphs(c);
  for (auto e : c->pev) cudaEventDestroy(e);
  for (auto e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->e0) cudaEventDestroy(c->e0);
  if (c->e1) cudaEventDestroy(c->e1);
  dfree(c->d_rowptr);
  dfree(c->d_col);
  dfree(c->d_val);
  dfree(c->d_valf);
  dfree(c->d_pmap);
  dfree(c->d_partial);
  dfree(c->d_X);
  dfree(c->d_Y);
  dfree(c->d_x);
  dfree(c->d_r);
  dfree(c->d_b);
  dfree(c->d_xf);
  dfree(c->d_rf);
  dfree(c->d_bf);
  dfree(c->d_sx);
  dfree(c->d_sr);
  dfree(c->d_st);
  dfree(c->d_opst);
  dfree(c->d_desc);
  dfree(c->d_opdesc);
  dfree(c->d_slotW);
  dfree(c->d_slotV);
  dfree(c->d_C);
  dfree(c->d_small);
  dfree(c->d_hist);
  dfree(c->d_rho_part);
  dfree(c->d_beta_part);
  dfree(c->d_bb_part);
  dfree(c->d_Rb);
  prec_free(c);
  if (c->h_flags) cudaFreeHost(c->h_flags);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

int ecg_create(const ecg_csr* A, const int32_t* partition, int t, const ecg_opts* opts, ecg_ctx** out) {
  if (!out) return ECG_EINVAL;
  *out = nullptr;
  if (!A || !partition || !A->rowptr || !A->col || !A->val) return ECG_EINVAL;
  if (A->n <= 0 || A->n > 0x7fffffff || A->nnz < 0 || A->nnz > 0x7fffffff) return ECG_EINVAL;
  if (width_index(t) < 0) return ECG_EINVAL;
  ecg_opts o;
  ecg_default_opts(&o);
  if (opts) o = *opts;
  if (o.inner_tol == 0.0) o.inner_tol = 1e-5;
  int rc = validate_opts(&o, t);
  if (rc) return rc;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return ECG_ECUDA;
  }
  const int n = (int)A->n;
  const int64_t nnz = A->nnz;
  // Host copies for validation (and upload).
  std::vector<int64_t> rp(n + 1);
  std::vector<int32_t> ci(nnz);
  std::vector<double> va(nnz);
  std::vector<int32_t> pt(n);
  if (A->on_device) {
    if (cudaMemcpy(rp.data(), A->rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(ci.data(), A->col, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(va.data(), A->val, sizeof(double) * nnz, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(pt.data(), partition, sizeof(int32_t) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return ECG_ECUDA;
    }
  } else {
    std::memcpy(rp.data(), A->rowptr, sizeof(int64_t) * (n + 1));
    std::memcpy(ci.data(), A->col, sizeof(int32_t) * nnz);
    std::memcpy(va.data(), A->val, sizeof(double) * nnz);
    std::memcpy(pt.data(), partition, sizeof(int32_t) * n);
  }
  if (rp[0] != 0 || rp[n] != nnz) return ECG_EINVAL;
  std::vector<int> cnt(t, 0);
  for (int i = 0; i < n; i++) {
    if (rp[i + 1] < rp[i]) return ECG_EINVAL;
    if (pt[i] < 0 || pt[i] >= t) return ECG_EINVAL;
    cnt[pt[i]]++;
  }
  for (int j = 0; j < t; j++)
    if (cnt[j] == 0) return ECG_EINVAL;
  for (int i = 0; i < n; i++) {
    double d = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
      if (ci[p] < 0 || ci[p] >= n) return ECG_EINVAL;
      if (ci[p] == i) d += va[p];
    }
    if (!(d > 0.0)) return ECG_ENOTSPD;
  }
  std::vector<int> rp32(n + 1);
  for (int i = 0; i <= n; i++) rp32[i] = (int)rp[i];

  ecg_ctx* c = new (std::nothrow) ecg_ctx();
  if (!c) return ECG_ENOMEM;
  c->n = n;
  c->nnz = nnz;
  c->t = t;
  c->opts = o;
  std::memset(&c->prof, 0, sizeof(c->prof));
  auto fail = [&](int code) {
    ecg_destroy(c);
    return code;
  };
  if (cudaGetDevice(&c->dev) != cudaSuccess) return fail(ECG_ECUDA);
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess)
    return fail(ECG_ECUDA);
  if (o.stream) {
    c->stream = (cudaStream_t)o.stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(ECG_ECUDA);
    c->own_stream = true;
  }
  if ((rc = set_all_smem_attrs())) return fail(rc);
  c->gx = std::max(1, std::min(4 * c->num_sms, (n + 31) / 32));
  set_f32_grids(c);
  const size_t nt = (size_t)n * t;
  const bool mixed = (o.precision == ECG_MIXED);
  if ((rc = dalloc(&c->d_rowptr, (size_t)n + 1)) || (rc = dalloc(&c->d_col, (size_t)nnz)) ||
      (rc = dalloc(&c->d_val, (size_t)nnz)) || (rc = dalloc(&c->d_pmap, (size_t)n)) ||
      (rc = dalloc(&c->d_X, nt)) || (rc = dalloc(&c->d_Y, nt)) || (rc = dalloc(&c->d_x, (size_t)n)) ||
      (rc = dalloc(&c->d_r, (size_t)n)) || (rc = dalloc(&c->d_b, (size_t)n)) ||
      (rc = dalloc(&c->d_sx, (size_t)n)) || (rc = dalloc(&c->d_sr, (size_t)n)) ||
      (rc = dalloc(&c->d_st, (size_t)1)) || (rc = dalloc(&c->d_opst, (size_t)1)) ||
      (rc = dalloc(&c->d_small, (size_t)kSmallSize)) || (rc = dalloc(&c->d_rho_part, (size_t)c->gx)) ||
      (rc = dalloc(&c->d_bb_part, (size_t)c->gx)) || (rc = dalloc(&c->d_beta_part, (size_t)c->gx * 64)))
    return fail(rc);
  if (mixed && ((rc = dalloc(&c->d_valf, (size_t)nnz)) || (rc = dalloc(&c->d_xf, (size_t)n)) ||
                (rc = dalloc(&c->d_rf, (size_t)n)) || (rc = dalloc(&c->d_bf, (size_t)n))))
    return fail(rc);
  if (cudaMemcpy(c->d_rowptr, rp32.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_col, ci.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_val, va.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_pmap, pt.data(), sizeof(int) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(ECG_ECUDA);
  if (mixed) {
    k_vals_to_float<<<std::max(1, std::min(8 * c->num_sms, (int)((nnz + 255) / 256))), 256, 0, c->stream>>>(
        nnz, c->d_val, c->d_valf);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(ECG_ECUDA);
  }
  if (cudaMemset(c->d_sx, 0, sizeof(double) * n) != cudaSuccess ||
      cudaMemset(c->d_sr, 0, sizeof(double) * n) != cudaSuccess)
    return fail(ECG_ECUDA);
  if (cudaHostAlloc((void**)&c->h_flags, 2 * sizeof(DevState), cudaHostAllocDefault) != cudaSuccess)
    return fail(ECG_ENOMEM);
  for (auto& e : c->ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(ECG_ECUDA);
  if (cudaEventCreate(&c->e0) != cudaSuccess || cudaEventCreate(&c->e1) != cudaSuccess) return fail(ECG_ECUDA);
  *out = c;
  return ECG_OK;
}

int ecg_solve(ecg_ctx* c, const double* b, const double* x0, double* x_out, double tol, int maxit,
              ecg_result* res) {
  if (res) std::memset(res, 0, sizeof(*res));
  if (!c || !b || !x_out) return ECG_EINVAL;
  if (!(tol >= 0.0) || maxit < 0) return ECG_EINVAL;
  const int n = c->n, t = c->t;
  const bool mixed = (c->opts.precision == ECG_MIXED);
  const size_t elem = mixed ? sizeof(float) : sizeof(double);
  const int kmax = std::max(maxit, 1);
  const int cap = c->opts.trunc > 0 ? c->opts.trunc : std::max(kmax - 1, 1);
  cudaStream_t s = c->stream;
  int rc;
  CK(cudaStreamSynchronize(s));
  // ---- storage for the stored blocks, history, coefficients, partials
  if (cap > c->slot_cap) {
    invalidate_graphs(c);
    dfree(c->d_slotW);
    dfree(c->d_slotV);
    dfree(c->d_desc);
    c->slot_cap = 0;
    size_t freeb = 0, totb = 0;
    CK(cudaMemGetInfo(&freeb, &totb));
    double need = 2.0 * (double)cap * (double)n * (double)t * (double)elem;
    if (need > 0.92 * (double)freeb) return ECG_ENOMEM;
    if ((rc = dalloc_bytes(&c->d_slotW, (size_t)cap * n * t * elem)) ||
        (rc = dalloc_bytes(&c->d_slotV, (size_t)cap * n * t * elem)) || (rc = dalloc(&c->d_desc, (size_t)cap))) {
      dfree(c->d_slotW);
      dfree(c->d_slotV);
      dfree(c->d_desc);
      return rc;
    }
    c->slot_cap = cap;
    c->desc_cap = cap;
  }
  if (kmax + 1 > c->hist_cap) {
    invalidate_graphs(c);
    dfree(c->d_hist);
    c->hist_cap = 0;
    if ((rc = dalloc(&c->d_hist, (size_t)kmax + 1))) return rc;
    c->hist_cap = kmax + 1;
  }
  if ((rc = ensure_C(c, (size_t)cap * t * t))) return rc;
  {
    const size_t gymax = ((size_t)cap * t + kChunk - 1) / kChunk;
    size_t need = (4 * (size_t)c->num_sms + gymax) * kChunk * t;
    for (int i = 0; i < 7 && kWidths[i] <= t; i++) {  // every width a solve can use (t, t/2 after the switch)
      const size_t w = (size_t)kWidths[i];
      need = std::max(need, (size_t)std::max(c->gx, c->gx_spmm64[i]) * (w * (w + 1) / 2 + w));
    }
    if (c->opts.block_residual) need = std::max(need, (size_t)c->gx * t * t);
    if ((rc = ensure_part(c, need))) return rc;
  }
  if (c->opts.block_residual) {
    if (c->prec_nb > 0) return ECG_EINVAL;  // no preconditioned block-residual form
    if (!c->d_Rb && (rc = dalloc(&c->d_Rb, (size_t)n * t))) return rc;
  }
  // ---- inputs
  const bool dev_in = is_device_ptr(b);
  const bool dev_out = is_device_ptr(x_out);
  CK(cudaMemcpyAsync(c->d_b, b, sizeof(double) * n, dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  if (x0) {
    CK(cudaMemcpyAsync(c->d_x, x0, sizeof(double) * n,
                       is_device_ptr(x0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  } else {
    CK(cudaMemsetAsync(c->d_x, 0, sizeof(double) * n, s));
  }
  CK(cudaEventRecord(c->e0, s));
  int iters = 0, status = ECG_ENOCONV, switch_it = 0, restarts = 0;
  long long mem = 0;
  double relres = 0.0;
  if (!mixed) {
    DevState fin;
    if ((rc = run_solve(c, false, kmax, cap, tol, 0, x0 != nullptr, &fin))) return rc;
    iters = fin.iters;
    status = fin.status;
    switch_it = fin.switch_it;
    restarts = fin.restarts;
    mem = fin.mem;
    relres = fin.rho0 > 0.0 ? fin.rho_prev / fin.rho0 : fin.rho_prev;
    c->h_hist.assign((size_t)iters + 1, 0.0);
    CK(cudaMemcpy(c->h_hist.data(), c->d_hist, sizeof(double) * (iters + 1), cudaMemcpyDeviceToHost));
  } else {
    // FP64 iterative refinement around FP32 inner solves.
    double rr = 0.0, bb = 0.0;
    if ((rc = true_residual(c, true, &rr, &bb))) return rc;
    const double rho0 = std::sqrt(rr);
    // the outer test: ||b - A x|| <= tol * ref, ref = rho_0 or ||b||
    const double ref = (c->opts.stop_rule == ECG_STOP_B) ? std::sqrt(bb) : rho0;
    double rho = rho0;
    c->h_hist.assign(1, rho0);
    const int gcv = std::max(1, std::min(8 * c->num_sms, (n + 255) / 256));
    for (int outer = 0;; outer++) {
      if (!(rho > tol * ref)) {
        status = ECG_OK;
        break;
      }
      if (iters >= kmax - 1 || outer >= kMaxOuter) {
        status = ECG_ENOCONV;
        break;
      }
      // the inner solve needs to reach only what is left of the tolerance
      const double need = 0.1 * tol * ref / rho;
      const double eps_in = std::min(0.5, std::max(c->opts.inner_tol, need));
      k_to_float_scaled<<<gcv, 256, 0, s>>>(n, c->d_r, c->d_bf, 1.0 / rho);
      CK(cudaMemsetAsync(c->d_xf, 0, sizeof(float) * n, s));
      DevState fin;
      if ((rc = run_solve(c, true, kmax - iters, cap, eps_in, iters, false, &fin))) return rc;
      if (fin.status == ECG_ECUDA) {
        status = ECG_ECUDA;
        break;
      }
      const int it = fin.iters;
      if (fin.mem > mem) mem = fin.mem;
      if (fin.switch_it > 0 && switch_it == 0) switch_it = iters + fin.switch_it;
      restarts += fin.restarts;
      std::vector<double> seg((size_t)it + 1);
      CK(cudaMemcpy(seg.data(), c->d_hist + iters, sizeof(double) * (it + 1), cudaMemcpyDeviceToHost));
      if (it == 0) {
        status = (fin.status == ECG_EBREAKDOWN) ? ECG_EBREAKDOWN : ECG_ENOCONV;
        break;
      }
      k_axpy_from_float<<<gcv, 256, 0, s>>>(n, c->d_x, c->d_xf, rho);
      CK(cudaGetLastError());
      if ((rc = true_residual(c, true, &rr, &bb))) return rc;
      const double rho_new = std::sqrt(rr);
      for (int k = 1; k <= it; k++) c->h_hist.push_back(rho * seg[k]);
      c->h_hist.back() = rho_new;  // the true FP64 residual at the refinement point
      iters += it;
      if (!(rho_new < rho)) {  // no progress: stagnation of the inner solves
        rho = rho_new;
        status = (rho_new > tol * ref) ? ECG_ENOCONV : ECG_OK;
        break;
      }
      rho = rho_new;
    }
    relres = rho0 > 0.0 ? rho / rho0 : rho;
  }
  CK(cudaEventRecord(c->e1, s));
  CK(cudaStreamSynchronize(s));
  prof_collect(c);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->e0, c->e1);
  // true residual ||b - A x|| / ||b||
  double srr = 0.0, sbb = 0.0;
  if ((rc = true_residual(c, false, &srr, &sbb))) return rc;
  CK(cudaMemcpyAsync(x_out, c->d_x, sizeof(double) * n, dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     s));
  CK(cudaStreamSynchronize(s));
  if (res) {
    res->iters = iters;
    res->switch_it = switch_it;
    res->restarts = restarts;
    res->status = status;
    res->mem_vectors = mem;
    res->relres = relres;
    res->relres_true = sbb > 0.0 ? std::sqrt(srr / sbb) : std::sqrt(srr);
    res->device_ms = ms;
    res->history = c->h_hist.data();
  }
  return status;
}

int ecg_profile_enable(ecg_ctx* c, int on) {
  if (!c) return ECG_EINVAL;
  c->profiling = (on != 0);
  std::memset(&c->prof, 0, sizeof(c->prof));
  c->pev_used = 0;
  return ECG_OK;
}

int ecg_profile_read(ecg_ctx* c, int cls, const char** name, double* ms, long long* launches) {
  if (!c) return ECG_EINVAL;
  if (cls < 0 || cls >= kProfClasses) return kProfClasses;
  if (name) *name = kProfNames[cls];
  if (ms) *ms = c->prof.ms[cls];
  if (launches) *launches = c->prof.launches[cls];
  return kProfClasses;
}

// ------------------------------------------------------ FP64 rate probe

namespace {
// Each thread runs kProbeChains independent FP64 FMA chains; the result is
// written out so that no chain can be removed.
constexpr int kProbeChains = 8;
__global__ void __launch_bounds__(256) k_probe_dfma(int iters, double a, double b, double* sink) {
  double v[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; c++) v[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) v[c] = fma(v[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kProbeChains; c++) s += v[c];
  if (s == 1234.5678) sink[blockIdx.x] = s;  // practically never taken
}
}  // namespace

int ecg_probe_fp64(int iters, double* tflops) {
  if (iters < 1 || !tflops) return ECG_EINVAL;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  double* sink = nullptr;
  CK(cudaMalloc(&sink, sizeof(double) * 8 * sms));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = ECG_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = ECG_ECUDA;
  const int blocks = 8 * sms;
  float ms = 0.f;
  if (rc == ECG_OK) {
    k_probe_dfma<<<blocks, 256>>>(iters / 8 + 1, 0.999999, 1e-7, sink);  // warm-up
    cudaEventRecord(e0);
    k_probe_dfma<<<blocks, 256>>>(iters, 0.999999, 1e-7, sink);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
      rc = ECG_ECUDA;
  }
  if (rc == ECG_OK) *tflops = 2.0 * kProbeChains * (double)iters * blocks * 256 / (ms * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return rc;
}

// ------------------------------------------------------ step-level calls

int ecg_op_split(ecg_ctx* c, const double* r, double* W, int half) {
  if (!c || !r || !W) return ECG_EINVAL;
  if (half && (c->t % 2)) return ECG_EINVAL;
  const int w = half ? c->t / 2 : c->t;
  int rc;
  if ((rc = put_op_state(c, op_state(c, w, 0, GEN_SPLIT)))) return rc;
  KP P = make_kp(c, c->d_opst, c->d_opdesc, false);
  P.X = W;
  P.r = const_cast<double*>(r);
  if ((rc = dispatch_w<RunGenerate>(w, c, P))) return rc;
  return finish_op(c, nullptr);
}

int ecg_set_preconditioner(ecg_ctx* c, const int32_t* pblock, int nblocks, int kind) {
  if (!c) return ECG_EINVAL;
  if (kind == ECG_PREC_NONE) {
    prec_free(c);
    return ECG_OK;
  }
  if (kind != ECG_PREC_IC0 || !pblock || nblocks < 1 || nblocks > c->n) return ECG_EINVAL;
  CK(cudaSetDevice(c->dev));
  CK(cudaStreamSynchronize(c->stream));
  std::vector<int> pb(c->n);
  if (is_device_ptr(pblock)) {
    CK(cudaMemcpy(pb.data(), pblock, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(pb.data(), pblock, sizeof(int32_t) * c->n);
  }
  prec_free(c);
  const int rc = prec_build(c, pb, nblocks);
  if (rc) prec_free(c);
  return rc;
}

int ecg_smooth(ecg_ctx* c, const double* b, double* x, int sweeps, double omega) {
  if (!c || !b || !x || sweeps < 0 || !(omega > 0.0 && omega < 2.0)) return ECG_EINVAL;
  if (sweeps == 0) return ECG_OK;
  int rc;
  if ((rc = put_op_state(c, op_state(c, 1, 0, GEN_SPLIT)))) return rc;
  KP P = make_kp(c, c->d_opst, c->d_opdesc, false);
  const int g = std::max(1, std::min(8 * c->num_sms, (c->n + 255) / 256));
  double* tmp = c->d_sx;  // scratch vector of the step-level calls
  for (int k = 0; k < sweeps; k++) {
    k_jacobi<<<g, 256, 0, c->stream>>>(P, x, b, omega, tmp);
    CK(cudaMemcpyAsync(x, tmp, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->stream));
  }
  return finish_op(c, nullptr);
}

int ecg_op_prec_apply(ecg_ctx* c, const double* in, double* out, int w) {
  if (!c || !in || !out || w < 1 || w > 64 || c->prec_nb == 0) return ECG_EINVAL;
  int rc;
  if ((rc = put_op_state(c, op_state(c, 1, 0, GEN_SPLIT)))) return rc;
  KP P = make_kp(c, c->d_opst, c->d_opdesc, false);
  RunPrec<1>::run(c, P, in, out, w);
  return finish_op(c, nullptr);
}

int ecg_op_spmm(ecg_ctx* c, const double* X, double* Y, int w) {
  if (!c || !X || !Y || width_index(w) < 0) return ECG_EINVAL;
  int rc;
  if ((rc = put_op_state(c, op_state(c, w, 0, GEN_SPLIT)))) return rc;
  KP P = make_kp(c, c->d_opst, c->d_opdesc, false);
  if ((rc = dispatch_w<RunSpmm>(w, c, P, X, Y))) return rc;
  return finish_op(c, nullptr);
}

int ecg_op_tdot(ecg_ctx* c, int m, const double* const* X, const int* wx, const double* Y, int wy, double* C) {
  if (!c || m < 1 || m > 1024 || !X || !wx || !Y || !C || width_index(wy) < 0) return ECG_EINVAL;
  std::vector<BlockDesc> d(m);
  int off = 0;
  for (int j = 0; j < m; j++) {
    if (!X[j] || wx[j] < 1 || wx[j] > 128) return ECG_EINVAL;
    d[j].W = const_cast<double*>(X[j]);
    d[j].V = const_cast<double*>(X[j]);
    d[j].w = wx[j];
    d[j].off = off;
    d[j].slot = 0;
    d[j].pad = 0;
    off += wx[j];
  }
  const int gy = (off + kChunk - 1) / kChunk;
  int rc;
  if ((rc = ensure_part(c, (size_t)std::max(gy * window_gx(c, gy), tc_grid(c)) * kChunk * wy))) return rc;
  if ((rc = put_op_desc(c, d))) return rc;
  if ((rc = put_op_state(c, op_state(c, wy, m, GEN_SPLIT)))) return rc;
  KP P = make_kp(c, c->d_opst, c->d_opdesc, false);
  if ((rc = dispatch_w<RunTdot>(wy, c, P, wy, Y, gy, C, off))) return rc;
  return finish_op(c, nullptr);
}

int ecg_op_cgs2(ecg_ctx* c, int m, const double* const* Q, const double* const* V, const int* wq, double* W,
                int w) {
  if (!c || m < 1 || m > 1024 || !Q || !V || !wq || !W || width_index(w) < 0) return ECG_EINVAL;
  std::vector<BlockDesc> d(m);
  int off = 0;
  for (int j = 0; j < m; j++) {
    if (!Q[j] || !V[j] || wq[j] < 1 || wq[j] > 128) return ECG_EINVAL;
    d[j].W = const_cast<double*>(Q[j]);
    d[j].V = const_cast<double*>(V[j]);
    d[j].w = wq[j];
    d[j].off = off;
    d[j].slot = 0;
    d[j].pad = 0;
    off += wq[j];
  }
  const int gy = (off + kChunk - 1) / kChunk;
  int rc;
  if ((rc = ensure_part(c, (size_t)std::max(gy * window_gx(c, gy), tc_grid(c)) * kChunk * w))) return rc;
  if ((rc = ensure_C(c, (size_t)gy * kChunk * w))) return rc;
  if ((rc = put_op_desc(c, d))) return rc;
  if ((rc = put_op_state(c, op_state(c, w, m, GEN_SPLIT)))) return rc;
  KP P = make_kp(c, c->d_opst, c->d_opdesc, false);
  for (int pass = 0; pass < 2; pass++) {
    if ((rc = dispatch_w<RunTdot>(w, c, P, w, (const double*)W, gy, c->d_C, off))) return rc;
    if ((rc = dispatch_w<RunUpdate>(w, c, P, W, (const double*)c->d_C, off))) return rc;
  }
  return finish_op(c, nullptr);
}

int ecg_op_block_sub(ecg_ctx* c, int m, const double* const* Q, const int* wq, const double* Cm, double* W, int w) {
  if (!c || m < 1 || m > 1024 || !Q || !wq || !Cm || !W || width_index(w) < 0) return ECG_EINVAL;
  std::vector<BlockDesc> d(m);
  int off = 0;
  for (int j = 0; j < m; j++) {
    if (!Q[j] || wq[j] < 1 || wq[j] > 128) return ECG_EINVAL;
    d[j].W = const_cast<double*>(Q[j]);
    d[j].V = const_cast<double*>(Q[j]);
    d[j].w = wq[j];
    d[j].off = off;
    d[j].slot = 0;
    d[j].pad = 0;
    off += wq[j];
  }
  int rc;
  if ((rc = put_op_desc(c, d))) return rc;
  if ((rc = put_op_state(c, op_state(c, w, m, GEN_SPLIT)))) return rc;
  KP P = make_kp(c, c->d_opst, c->d_opdesc, false);
  if ((rc = dispatch_w<RunUpdate>(w, c, P, W, Cm, off))) return rc;
  return finish_op(c, nullptr);
}

static int op_orth(ecg_ctx* c, double* W, double* V, int w, double* x, double* r, double* rho) {
  if (!c || !W || !V || width_index(w) < 0) return ECG_EINVAL;
  int rc;
  if ((rc = ensure_part(c, (size_t)c->gx * (w * (w + 1) / 2 + w)))) return rc;
  if ((rc = put_op_state(c, op_state(c, w, 0, GEN_SPLIT)))) return rc;
  KP P = make_kp(c, c->d_opst, c->d_opdesc, false);
  P.r = r;
  P.want_beta = 0;
  if ((rc = dispatch_w<RunOrth>(w, c, P, W, V, x, r))) return rc;
  k_rho_only<<<1, kThreads, 0, c->stream>>>(P, c->gx);
  int status = ECG_OK;
  if ((rc = finish_op(c, &status))) return rc;
  if (rho) {
    DevState s;
    CK(cudaMemcpy(&s, c->d_opst, sizeof(s), cudaMemcpyDeviceToHost));
    *rho = s.rho;
  }
  return status;
}

int ecg_op_a_orthonormalize(ecg_ctx* c, double* W, double* V, int w) {
  if (!c) return ECG_EINVAL;
  return op_orth(c, W, V, w, c->d_sx, c->d_sr, nullptr);
}

int ecg_op_block_update(ecg_ctx* c, double* W, double* V, int w, double* x, double* r, double* rho) {
  if (!c || !x || !r) return ECG_EINVAL;
  return op_orth(c, W, V, w, x, r, rho);
}

int ecg_op_msdo_generate(ecg_ctx* c, const double* r, const double* P_prev, const double* V_prev, int w,
                         double* Pout) {
  if (!c || !r || !P_prev || !V_prev || !Pout) return ECG_EINVAL;
  if (!(w == c->t || (c->t % 2 == 0 && w == c->t / 2))) return ECG_EINVAL;
  std::vector<BlockDesc> d(1);
  d[0].W = const_cast<double*>(P_prev);
  d[0].V = const_cast<double*>(V_prev);
  d[0].w = w;
  d[0].off = 0;
  d[0].slot = 0;
  d[0].pad = 0;
  int rc;
  if ((rc = ensure_part(c, (size_t)window_gx(c, 1) * kChunk))) return rc;
  if ((rc = put_op_desc(c, d))) return rc;
  if ((rc = put_op_state(c, op_state(c, 1, 1, GEN_SPLIT)))) return rc;
  KP P = make_kp(c, c->d_opst, c->d_opdesc, false);
  if ((rc = dispatch_w<RunTdot>(1, c, P, 1, r, 1, c->d_small + kSmallG, w))) return rc;
  k_neg_copy<<<1, 64, 0, c->stream>>>(c->d_small + kSmallG, c->d_small + kSmallBe, w);
  if ((rc = put_op_state(c, op_state(c, w, 1, GEN_MSDO)))) return rc;
  P.X = Pout;
  P.r = const_cast<double*>(r);
  if ((rc = dispatch_w<RunGenerate>(w, c, P))) return rc;
  return finish_op(c, nullptr);
}

}  // extern "C"

// ===================================================== allocation-free call
//
// ecg_tdot_noalloc runs the same two kernels as ecg_op_tdot, but its
// partial sums, launch state and block descriptors live in the file-scope
// device arrays below instead of memory a context allocates.  Every GPU that
// loads this library holds these arrays (about 4.2 MB) until the process
// exits.  Host code must not pass the array names to a kernel: on the host
// they are stand-ins, not device addresses.  The device addresses come from
// cudaGetSymbolAddress, once per device, in noalloc_setup().

namespace {
constexpr int kNoAllocMaxBlocks = 64;         // blocks X_j per call
constexpr int kNoAllocMaxCols = 256;          // sum of their widths
constexpr size_t kNoAllocScratch = 1u << 19;  // doubles of partial sums (4 MiB)
}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];
static __device__ __align__(256) DevState g_noalloc_state;
static __device__ __align__(256) BlockDesc g_noalloc_desc[kNoAllocMaxBlocks];

namespace {

struct NoAllocDevice {
  double* scratch = nullptr;
  DevState* st = nullptr;
  BlockDesc* desc = nullptr;
  int sms = 0;
  bool ready = false;
};

constexpr int kNoAllocMaxDevices = 64;
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
std::mutex g_noalloc_mutex;

template <int WB>
cudaError_t noalloc_smem_attr() {
  return cudaFuncSetAttribute((const void*)k_tdot_window<double, WB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_tdot<double, WB>());
}

// Device addresses of the arrays above for the current device, looked up on
// the first call made on that device, which also raises the dynamic shared
// memory limit of the kernels it launches (some need more than the 48 KiB
// default; a context does the same in ecg_create, but this call needs none).
int noalloc_setup(NoAllocDevice** out) {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return ECG_EINVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoAllocDevice& d = g_noalloc_dev[dev];
  if (!d.ready) {
    CK(cudaGetSymbolAddress((void**)&d.scratch, g_noalloc_scratch));
    CK(cudaGetSymbolAddress((void**)&d.st, g_noalloc_state));
    CK(cudaGetSymbolAddress((void**)&d.desc, g_noalloc_desc));
    CK(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
    CK(noalloc_smem_attr<1>());
    CK(noalloc_smem_attr<2>());
    CK(noalloc_smem_attr<4>());
    CK(noalloc_smem_attr<8>());
    CK(noalloc_smem_attr<16>());
    CK(noalloc_smem_attr<32>());
    CK(noalloc_smem_attr<64>());
    d.ready = true;
  }
  *out = &d;
  return ECG_OK;
}

template <int WB>
void noalloc_launch(KP P, const double* Y, int gxw, int gy, double* C, cudaStream_t s) {
  k_tdot_window<double, WB><<<dim3(gxw, gy), kThreads, smem_tdot<double, WB>(), s>>>(P, WB, Y);
  k_reduce_C<WB><<<dim3((kChunk * WB * 32 + kThreads - 1) / kThreads, gy), kThreads, 0, s>>>(P, WB, gxw, C);
}

}  // namespace

extern "C" int ecg_tdot_noalloc(int64_t n, int m, const double* const* X, const int* wx, const double* Y, int wy,
                                double* C, void* stream) {
  if (n < 1 || n > 0x7fffffff || m < 1 || m > kNoAllocMaxBlocks || !X || !wx || !Y || !C || width_index(wy) < 0)
    return ECG_EINVAL;
  BlockDesc hd[kNoAllocMaxBlocks];
  int off = 0;
  for (int j = 0; j < m; j++) {
    if (!X[j] || wx[j] < 1 || wx[j] > 128) return ECG_EINVAL;
    hd[j].W = const_cast<double*>(X[j]);
    hd[j].V = const_cast<double*>(X[j]);
    hd[j].w = wx[j];
    hd[j].off = off;
    hd[j].slot = 0;
    hd[j].pad = 0;
    off += wx[j];
  }
  if (off > kNoAllocMaxCols) return ECG_EINVAL;
  NoAllocDevice* d = nullptr;
  int rc = noalloc_setup(&d);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int gy = (off + kChunk - 1) / kChunk;
  const size_t per_cta = (size_t)kChunk * wy;
  int gxw = (4 * d->sms + gy - 1) / gy;
  gxw = std::min<long long>(gxw, (long long)(kNoAllocScratch / (per_cta * gy)));
  gxw = (int)std::max<long long>(1, std::min<long long>(gxw, (n + 31) / 32));
  DevState hs;
  std::memset(&hs, 0, sizeof(hs));
  hs.width = wy;
  hs.nq = m;
  hs.cap = m;
  hs.k = 1;
  CK(cudaMemcpyAsync(d->desc, hd, sizeof(BlockDesc) * m, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d->st, &hs, sizeof(hs), cudaMemcpyHostToDevice, s));
  KP P;
  std::memset(&P, 0, sizeof(P));
  P.n = (int)n;
  P.st = d->st;
  P.desc = d->desc;
  P.part_buf = d->scratch;
  switch (wy) {
    case 1: noalloc_launch<1>(P, Y, gxw, gy, C, s); break;
    case 2: noalloc_launch<2>(P, Y, gxw, gy, C, s); break;
    case 4: noalloc_launch<4>(P, Y, gxw, gy, C, s); break;
    case 8: noalloc_launch<8>(P, Y, gxw, gy, C, s); break;
    case 16: noalloc_launch<16>(P, Y, gxw, gy, C, s); break;
    case 32: noalloc_launch<32>(P, Y, gxw, gy, C, s); break;
    case 64: noalloc_launch<64>(P, Y, gxw, gy, C, s); break;
  }
  CK(cudaGetLastError());
  int fault = 0;  // a bounded wait on a bulk copy ran out
  CK(cudaMemcpyAsync(&fault, &d->st->fault, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return fault ? ECG_ECUDA : ECG_OK;
}
