// batch.cu -- host side of the batched enlarged CG solver (ecg_batch_* in
// include/ecg.h): SELL-C-sigma layout and its autotuner, the CTA groups,
// the refinement rounds captured in a CUDA graph, and the C ABI.
//
// Method: truncated SRE-CG2 (S. Moufawad, "Flexibly Enlarged Conjugate
// Gradient methods", arXiv 2305.19013, Algorithm 1 with the window of
// Section 3) on every system of the batch; see ecg_batch.cuh for the
// persistent kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "ecg.h"
#include "ecg_batch.cuh"

using namespace ecgb;

namespace {

#define BCK(call)                  \
  do {                             \
    cudaError_t e_ = (call);       \
    if (e_ != cudaSuccess) {       \
      cudaGetLastError();          \
      return ECG_ECUDA;            \
    }                              \
  } while (0)

template <typename T>
int balloc(T** p, size_t count) {
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

int balloc_bytes(void** p, size_t bytes) {
  unsigned char* q = nullptr;
  const int rc = balloc(&q, bytes);
  *p = q;
  return rc;
}

template <typename T>
void bfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <typename T>
int bput(T** d, const std::vector<T>& h) {
  int rc = balloc(d, h.size());
  if (rc) return rc;
  if (!h.empty()) BCK(cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return ECG_OK;
}

bool dev_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct HostSys {
  int n = 0;
  std::vector<int64_t> rp;
  std::vector<int> col;  // local columns
  std::vector<double> val;
  std::vector<int> part;
};

// SELL-C-sigma of the whole batch (slots and slices numbered globally,
// every system starting on a slice boundary).
struct Sell {
  int C = 32, sigma = 1;
  std::vector<int> srow, sptr, slen, scol;
  std::vector<double> sval;
  std::vector<int> slot_off, slice_off;  // per system
};

Sell build_sell(const std::vector<HostSys>& sys, const std::vector<int>& off, int C, int sigma) {
  Sell S;
  S.C = C;
  S.sigma = sigma;
  S.sptr.push_back(0);
  for (size_t s = 0; s < sys.size(); s++) {
    const HostSys& h = sys[s];
    S.slot_off.push_back((int)S.srow.size());
    S.slice_off.push_back((int)S.slen.size());
    // rows by decreasing length inside windows of sigma rows (stable)
    std::vector<int> perm(h.n);
    for (int i = 0; i < h.n; i++) perm[i] = i;
    if (sigma > 1)
      for (int w0 = 0; w0 < h.n; w0 += sigma) {
        const int w1 = std::min(h.n, w0 + sigma);
        std::stable_sort(perm.begin() + w0, perm.begin() + w1, [&](int a, int b) {
          return (h.rp[a + 1] - h.rp[a]) > (h.rp[b + 1] - h.rp[b]);
        });
      }
    const int nsl = (h.n + C - 1) / C;
    for (int sl = 0; sl < nsl; sl++) {
      int len = 0;
      for (int l = 0; l < C; l++) {
        const int p = sl * C + l;
        const int row = p < h.n ? perm[p] : -1;
        S.srow.push_back(row < 0 ? -1 : off[s] + row);
        if (row >= 0) len = std::max(len, (int)(h.rp[row + 1] - h.rp[row]));
      }
      S.slen.push_back(len);
      for (int k = 0; k < len; k++)
        for (int l = 0; l < C; l++) {
          const int p = sl * C + l;
          const int row = p < h.n ? perm[p] : -1;
          if (row >= 0 && h.rp[row] + k < h.rp[row + 1]) {
            S.scol.push_back(off[s] + h.col[h.rp[row] + k]);
            S.sval.push_back(h.val[h.rp[row] + k]);
          } else {  // padding: a zero times a valid row of the same system
            S.scol.push_back(off[s] + (row >= 0 ? row : 0));
            S.sval.push_back(0.0);
          }
        }
      S.sptr.push_back((int)S.scol.size());
    }
  }
  return S;
}

}  // namespace

struct ecg_batch {
  int nsys = 0, t = 0, N = 0;
  ecg_batch_opts o;
  int dev = 0, sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<int> n, off;
  int C = 32, sigma = 1, G = 0;
  double spmm_ms = 0.0;
  int nslots = 0;
  std::vector<CtaInfo> cta;
  // device
  int *d_part = nullptr, *d_srow = nullptr, *d_sptr = nullptr, *d_slen = nullptr, *d_scol = nullptr;
  double* d_sval = nullptr;
  float* d_svalf = nullptr;
  CtaInfo* d_cta = nullptr;
  int *d_first = nullptr, *d_gsize = nullptr;
  double *d_x = nullptr, *d_r = nullptr, *d_b = nullptr;
  float *d_xf = nullptr, *d_rf = nullptr;
  void *d_X = nullptr, *d_Y = nullptr, *d_QW = nullptr, *d_QV = nullptr;
  double *d_part_buf = nullptr, *d_part2 = nullptr;
  SysState* d_st = nullptr;
  Outer* d_outer = nullptr;
  unsigned* d_bar = nullptr;
  double *d_rr = nullptr, *d_bb = nullptr;
  int* d_active = nullptr;
  int* h_active = nullptr;  // pinned
  double* d_hist = nullptr;
  int hist_cap = 0;
  bool graph_used = false;  // the last solve replayed a captured graph
  std::vector<double> h_hist;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

namespace {

int width_ok(int t) { return t == 4 || t == 8; }

BatchP make_bp(const ecg_batch* b, bool fp32) {
  BatchP B;
  std::memset(&B, 0, sizeof(B));
  B.nsys = b->nsys;
  B.m = b->o.trunc;
  B.pre = (b->o.ortho == ECG_PRE_CHOLQR) ? 1 : 0;
  B.C = b->C;
  B.cta = b->d_cta;
  B.part = b->d_part;
  B.srow = b->d_srow;
  B.sptr = b->d_sptr;
  B.slen = b->d_slen;
  B.scol = b->d_scol;
  B.sval = fp32 ? (const void*)b->d_svalf : (const void*)b->d_sval;
  B.X = b->d_X;
  B.Y = b->d_Y;
  B.QW = b->d_QW;
  B.QV = b->d_QV;
  B.slot_stride = (long long)b->N * b->t;
  B.x = fp32 ? (void*)b->d_xf : (void*)b->d_x;
  B.r = fp32 ? (void*)b->d_rf : (void*)b->d_r;
  B.part_buf = b->d_part_buf;
  B.st = b->d_st;
  B.bar = b->d_bar;
  B.hist = b->d_hist;
  B.hist_cap = b->hist_cap;
  B.wait_ns = (unsigned long long)(b->o.wait_limit_s * 1e9);
  B.bar_extra = b->o.debug_barrier_extra;
  return B;
}

struct InnerK {
  const void* fn = nullptr;
  int smem = 0;  // dynamic shared memory (bytes)
};

template <typename T, int W, int MM>
InnerK inner_k() {
  InnerK k;
  k.fn = (const void*)k_batch_sre<T, W, MM>;
  k.smem = BGeom<T, W, MM>::SMEM;
  return k;
}

template <typename T, int W>
InnerK inner_kernel(int m) {
  switch (m) {
    case 1: return inner_k<T, W, 1>();
    case 2: return inner_k<T, W, 2>();
    case 3: return inner_k<T, W, 3>();
    case 4: return inner_k<T, W, 4>();
  }
  return InnerK();
}

InnerK inner_kernel_for(bool fp32, int t, int m) {
  switch (t) {
    case 4: return fp32 ? inner_kernel<float, 4>(m) : inner_kernel<double, 4>(m);
    case 8: return fp32 ? inner_kernel<float, 8>(m) : inner_kernel<double, 8>(m);
  }
  return InnerK();
}

// One cooperative launch of the persistent inner solve over G CTAs.
int launch_inner(ecg_batch* b, bool fp32) {
  BatchP B = make_bp(b, fp32);
  void* args[] = {&B};
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  const InnerK k = inner_kernel_for(fp32, b->t, b->o.trunc);
  cfg.gridDim = dim3(b->G);
  cfg.blockDim = dim3(kBThreads);
  cfg.dynamicSmemBytes = (size_t)k.smem;
  cfg.stream = b->stream;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeCooperative;
  attr.val.cooperative = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  BCK(cudaLaunchKernelExC(&cfg, k.fn, args));
  return ECG_OK;
}

template <typename T>
int time_spmm(ecg_batch* b, const Sell& S, double* ms_out) {
  int *srow = nullptr, *sptr = nullptr, *slen = nullptr, *scol = nullptr;
  T* sval = nullptr;
  std::vector<T> v(S.sval.begin(), S.sval.end());
  int rc;
  if ((rc = bput(&srow, S.srow)) || (rc = bput(&sptr, S.sptr)) || (rc = bput(&slen, S.slen)) ||
      (rc = bput(&scol, S.scol)) || (rc = bput(&sval, v))) {
    bfree(srow);
    bfree(sptr);
    bfree(slen);
    bfree(scol);
    bfree(sval);
    return rc;
  }
  BatchP B;
  std::memset(&B, 0, sizeof(B));
  B.C = S.C;
  B.srow = srow;
  B.sptr = sptr;
  B.slen = slen;
  B.scol = scol;
  B.sval = sval;
  B.X = b->d_X;
  B.Y = b->d_Y;
  const int ns = (int)S.srow.size();
  const int grid = std::max(1, std::min(8 * b->sms, (ns + kBThreads - 1) / kBThreads));
  auto launch = [&]() {
    switch (b->t) {
      case 4: k_batch_spmm<T, 4><<<grid, kBThreads, 0, b->stream>>>(B, ns); break;
      default: k_batch_spmm<T, 8><<<grid, kBThreads, 0, b->stream>>>(B, ns); break;
    }
  };
  for (int w = 0; w < 2; w++) launch();
  cudaEventRecord(b->e0, b->stream);
  const int reps = 5;
  for (int w = 0; w < reps; w++) launch();
  cudaEventRecord(b->e1, b->stream);
  cudaError_t e = cudaEventSynchronize(b->e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->e0, b->e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  bfree(srow);
  bfree(sptr);
  bfree(slen);
  bfree(scol);
  bfree(sval);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ECG_ECUDA;
  }
  *ms_out = ms / reps;
  return ECG_OK;
}

// CTA groups: system s gets gsize_s CTAs (at least one) in proportion to
// its expected work, rows times iterations.  The iterations of CG-type
// methods grow like sqrt(kappa), and kappa like n for the 2D diffusion
// systems the batch is built for, so the weight is n^{3/2}: on the 64-system
// workload (n from 16K to 262K) the iteration counts span the same 4-5x as
// sqrt(n).  CTA q of a group owns an even share of its rows and slices.
void place_ctas(ecg_batch* b, const Sell& S) {
  const int ns = b->nsys, G = b->G;
  std::vector<int> gs(ns);
  std::vector<double> w(ns);
  double tot = 0.0;
  for (int s = 0; s < ns; s++) {
    w[s] = (double)b->n[s] * std::sqrt((double)b->n[s]);
    tot += w[s];
  }
  int sum = 0;
  for (int s = 0; s < ns; s++) {
    gs[s] = std::max(1, std::min(b->n[s], (int)((double)G * w[s] / tot)));
    sum += gs[s];
  }
  while (sum > G) {  // take from the system with the least work per CTA
    int best = -1;
    for (int s = 0; s < ns; s++)
      if (gs[s] > 1 && (best < 0 || w[s] / gs[s] < w[best] / gs[best])) best = s;
    gs[best]--;
    sum--;
  }
  while (sum < G) {  // give to the system with the most work per CTA
    int best = -1;
    for (int s = 0; s < ns; s++)
      if (gs[s] < b->n[s] && (best < 0 || w[s] / gs[s] > w[best] / gs[best])) best = s;
    if (best < 0) break;
    gs[best]++;
    sum++;
  }
  b->cta.clear();
  for (int s = 0; s < ns; s++) {
    const int first = (int)b->cta.size();
    const int nsl = (b->n[s] + S.C - 1) / S.C;
    for (int q = 0; q < gs[s]; q++) {
      CtaInfo ci;
      ci.sys = s;
      ci.q = q;
      ci.first = first;
      ci.gsize = gs[s];
      ci.r0 = b->off[s] + (int)((long long)b->n[s] * q / gs[s]);
      ci.r1 = b->off[s] + (int)((long long)b->n[s] * (q + 1) / gs[s]);
      ci.s0 = S.slot_off[s] + S.C * (int)((long long)nsl * q / gs[s]);
      ci.s1 = S.slot_off[s] + S.C * (int)((long long)nsl * (q + 1) / gs[s]);
      b->cta.push_back(ci);
    }
  }
}

void batch_free(ecg_batch* b) {
  bfree(b->d_part);
  bfree(b->d_srow);
  bfree(b->d_sptr);
  bfree(b->d_slen);
  bfree(b->d_scol);
  bfree(b->d_sval);
  bfree(b->d_svalf);
  bfree(b->d_cta);
  bfree(b->d_first);
  bfree(b->d_gsize);
  bfree(b->d_x);
  bfree(b->d_r);
  bfree(b->d_b);
  bfree(b->d_xf);
  bfree(b->d_rf);
  bfree(b->d_X);
  bfree(b->d_Y);
  bfree(b->d_QW);
  bfree(b->d_QV);
  bfree(b->d_part_buf);
  bfree(b->d_part2);
  bfree(b->d_st);
  bfree(b->d_outer);
  bfree(b->d_bar);
  bfree(b->d_rr);
  bfree(b->d_bb);
  bfree(b->d_active);
  bfree(b->d_hist);
  if (b->h_active) cudaFreeHost(b->h_active);
  b->h_active = nullptr;
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  b->e0 = b->e1 = nullptr;
}

// The launches of one round (see k_batch_round_begin): round control,
// [scaling], the persistent inner solve, [x update], the FP64 residual.
int enqueue_round(ecg_batch* b, bool fp32, double tol, int maxit, int max_rounds) {
  cudaStream_t s = b->stream;
  const BatchP B = make_bp(b, fp32);
  const int ns = b->nsys;
  BCK(cudaMemsetAsync(b->d_active, 0, sizeof(int), s));
  k_batch_round_begin<<<(ns + 127) / 128, 128, 0, s>>>(ns, b->d_st, b->d_outer, b->d_rr, tol, b->o.inner_tol, maxit,
                                                       fp32 ? 1 : 0, max_rounds, b->d_active);
  if (fp32) k_batch_scale<<<b->G, kBThreads, 0, s>>>(B, b->d_outer, b->d_r, b->d_rf, b->d_xf);
  BCK(cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned) * ns, s));
  int rc = launch_inner(b, fp32);
  if (rc) return rc;
  if (fp32) k_batch_round_end<<<b->G, kBThreads, 0, s>>>(B, b->d_outer, b->d_x, b->d_xf);
  k_batch_residual<<<b->G, kBThreads, 0, s>>>(B, b->d_sval, b->d_x, b->d_b, b->d_r, b->d_part2);
  k_batch_norms<<<(ns + 127) / 128, 128, 0, s>>>(ns, b->d_first, b->d_gsize, b->d_part2, b->d_rr, b->d_bb);
  BCK(cudaGetLastError());
  return ECG_OK;
}

}  // namespace

extern "C" {

void ecg_batch_default_opts(ecg_batch_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->trunc = 2;
  o->ortho = ECG_PRE_CHOLQR;
  o->precision = ECG_MIXED;
  o->inner_tol = 1e-5;
  o->slice_height = 0;
  o->sort_window = 0;
  o->ctas_per_sm = 0;
  o->wait_limit_s = 1.0;
  o->debug_barrier_extra = 0;
  o->stream = nullptr;
}

void ecg_batch_destroy(ecg_batch* b) {
  if (!b) return;
  cudaSetDevice(b->dev);
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_free(b);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int ecg_batch_create(int nsys, const ecg_csr* A, const int32_t* const* partition, int t, const ecg_batch_opts* opts,
                     ecg_batch** out) {
  if (!out) return ECG_EINVAL;
  *out = nullptr;
  if (nsys < 1 || !A || !partition || !width_ok(t)) return ECG_EINVAL;
  ecg_batch_opts o;
  ecg_batch_default_opts(&o);
  if (opts) o = *opts;
  if (o.trunc < 1 || o.trunc > kBMaxM || (o.ortho != ECG_PRE_CHOLQR && o.ortho != ECG_A_CHOLQR) ||
      (o.precision != ECG_FP64 && o.precision != ECG_MIXED) || !(o.inner_tol > 0.0 && o.inner_tol < 1.0) ||
      (o.slice_height != 0 && o.slice_height != 8 && o.slice_height != 16 && o.slice_height != 32) ||
      o.sort_window < 0 || o.ctas_per_sm < 0 || o.ctas_per_sm > 4 || !(o.wait_limit_s > 0.0) ||
      o.wait_limit_s > 60.0 || o.debug_barrier_extra < 0)
    return ECG_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return ECG_ECUDA;
  }
  // host copies, validated
  std::vector<HostSys> sys(nsys);
  long long N = 0;
  for (int s = 0; s < nsys; s++) {
    const ecg_csr& a = A[s];
    if (!a.rowptr || !a.col || !a.val || !partition[s] || a.n <= 0 || a.nnz < 0) return ECG_EINVAL;
    HostSys& h = sys[s];
    h.n = (int)a.n;
    h.rp.resize(a.n + 1);
    h.col.resize(a.nnz);
    h.val.resize(a.nnz);
    h.part.resize(a.n);
    if (a.on_device) {
      if (cudaMemcpy(h.rp.data(), a.rowptr, sizeof(int64_t) * (a.n + 1), cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(h.col.data(), a.col, sizeof(int32_t) * a.nnz, cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(h.val.data(), a.val, sizeof(double) * a.nnz, cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(h.part.data(), partition[s], sizeof(int32_t) * a.n, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return ECG_ECUDA;
      }
    } else {
      std::memcpy(h.rp.data(), a.rowptr, sizeof(int64_t) * (a.n + 1));
      std::memcpy(h.col.data(), a.col, sizeof(int32_t) * a.nnz);
      std::memcpy(h.val.data(), a.val, sizeof(double) * a.nnz);
      std::memcpy(h.part.data(), partition[s], sizeof(int32_t) * a.n);
    }
    if (h.rp[0] != 0 || h.rp[a.n] != a.nnz) return ECG_EINVAL;
    std::vector<int> cnt(t, 0);
    for (int i = 0; i < h.n; i++) {
      if (h.rp[i + 1] < h.rp[i] || h.part[i] < 0 || h.part[i] >= t) return ECG_EINVAL;
      cnt[h.part[i]]++;
      double d = 0.0;
      for (int64_t p = h.rp[i]; p < h.rp[i + 1]; p++) {
        if (h.col[p] < 0 || h.col[p] >= h.n) return ECG_EINVAL;
        if (h.col[p] == i) d += h.val[p];
      }
      if (!(d > 0.0)) return ECG_ENOTSPD;
    }
    for (int j = 0; j < t; j++)
      if (cnt[j] == 0) return ECG_EINVAL;
    N += h.n;
  }
  if (N > (1LL << 30)) return ECG_EINVAL;

  ecg_batch* b = new (std::nothrow) ecg_batch();
  if (!b) return ECG_ENOMEM;
  b->nsys = nsys;
  b->t = t;
  b->N = (int)N;
  b->o = o;
  auto fail = [&](int code) {
    ecg_batch_destroy(b);
    return code;
  };
  if (cudaGetDevice(&b->dev) != cudaSuccess) return fail(ECG_ECUDA);
  if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev) != cudaSuccess) return fail(ECG_ECUDA);
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->dev) != cudaSuccess || !coop)
    return fail(ECG_ECUDA);
  if (o.stream) {
    b->stream = (cudaStream_t)o.stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(ECG_ECUDA);
    b->own_stream = true;
  }
  if (cudaEventCreate(&b->e0) != cudaSuccess || cudaEventCreate(&b->e1) != cudaSuccess) return fail(ECG_ECUDA);
  // persistent CTAs: as many per SM as the inner solve's kernel fits
  int per_sm = 0;
  {
    const InnerK k = inner_kernel_for(o.precision == ECG_MIXED, t, o.trunc);
    if (cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, kBThreads, (size_t)k.smem) != cudaSuccess) {
      cudaGetLastError();
      return fail(ECG_ECUDA);
    }
  }
  if (per_sm < 1) return fail(ECG_ECUDA);
  const int want = o.ctas_per_sm ? o.ctas_per_sm : std::min(2, per_sm);
  if (want > per_sm) return fail(ECG_EINVAL);
  b->G = want * b->sms;
  if (nsys > b->G) return fail(ECG_EINVAL);
  b->n.resize(nsys);
  b->off.resize(nsys);
  {
    int acc = 0;
    for (int s = 0; s < nsys; s++) {
      b->n[s] = sys[s].n;
      b->off[s] = acc;
      acc += sys[s].n;
    }
  }
  const size_t NW = (size_t)N * t;
  int rc;
  if ((rc = balloc(&b->d_x, (size_t)N)) || (rc = balloc(&b->d_r, (size_t)N)) || (rc = balloc(&b->d_b, (size_t)N)) ||
      (rc = balloc_bytes(&b->d_X, NW * sizeof(double))) || (rc = balloc_bytes(&b->d_Y, NW * sizeof(double))) ||
      (rc = balloc_bytes(&b->d_QW, (size_t)o.trunc * NW * sizeof(double))) ||
      (rc = balloc_bytes(&b->d_QV, (size_t)o.trunc * NW * sizeof(double))) ||
      (rc = balloc(&b->d_part_buf, (size_t)2 * b->G * kBPartStride)) ||
      (rc = balloc(&b->d_part2, (size_t)2 * b->G)) || (rc = balloc(&b->d_st, (size_t)nsys)) ||
      (rc = balloc(&b->d_outer, (size_t)nsys)) || (rc = balloc(&b->d_bar, (size_t)nsys)) ||
      (rc = balloc(&b->d_rr, (size_t)nsys)) || (rc = balloc(&b->d_bb, (size_t)nsys)) ||
      (rc = balloc(&b->d_active, (size_t)1)))
    return fail(rc);
  if (o.precision == ECG_MIXED && ((rc = balloc(&b->d_xf, (size_t)N)) || (rc = balloc(&b->d_rf, (size_t)N))))
    return fail(rc);
  if (cudaMallocHost((void**)&b->h_active, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ECG_ENOMEM);
  }
  if (cudaMemsetAsync(b->d_X, 0, NW * sizeof(double), b->stream) != cudaSuccess) return fail(ECG_ECUDA);
  {
    std::vector<int> part((size_t)N);
    for (int s = 0; s < nsys; s++) std::copy(sys[s].part.begin(), sys[s].part.end(), part.begin() + b->off[s]);
    if ((rc = bput(&b->d_part, part))) return fail(rc);
  }
  // SELL layout: fixed, or the fastest product among the candidates
  std::vector<int> Cs, sigmas;
  if (o.slice_height) Cs.push_back(o.slice_height);
  else Cs = {8, 16, 32};
  if (o.sort_window) sigmas.push_back(o.sort_window);
  else sigmas = {1, 256};
  double best = 1e300;
  int bestC = Cs[0], bestS = sigmas[0];
  if (Cs.size() * sigmas.size() > 1) {
    for (int C : Cs)
      for (int sg : sigmas) {
        const Sell S = build_sell(sys, b->off, C, sg);
        double ms = 0.0;
        rc = (o.precision == ECG_MIXED) ? time_spmm<float>(b, S, &ms) : time_spmm<double>(b, S, &ms);
        if (rc) return fail(rc);
        if (ms < best) {
          best = ms;
          bestC = C;
          bestS = sg;
        }
      }
    b->spmm_ms = best;
  }
  b->C = bestC;
  b->sigma = bestS;
  const Sell S = build_sell(sys, b->off, b->C, b->sigma);
  b->nslots = (int)S.srow.size();
  {
    std::vector<float> vf(S.sval.begin(), S.sval.end());
    if ((rc = bput(&b->d_srow, S.srow)) || (rc = bput(&b->d_sptr, S.sptr)) || (rc = bput(&b->d_slen, S.slen)) ||
        (rc = bput(&b->d_scol, S.scol)) || (rc = bput(&b->d_sval, S.sval)) ||
        (o.precision == ECG_MIXED && (rc = bput(&b->d_svalf, vf))))
      return fail(rc);
  }
  place_ctas(b, S);
  {
    std::vector<int> first(nsys), gsize(nsys);
    for (const CtaInfo& ci : b->cta)
      if (ci.q == 0) {
        first[ci.sys] = ci.first;
        gsize[ci.sys] = ci.gsize;
      }
    if ((rc = bput(&b->d_cta, b->cta)) || (rc = bput(&b->d_first, first)) || (rc = bput(&b->d_gsize, gsize)))
      return fail(rc);
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(ECG_ECUDA);
  *out = b;
  return ECG_OK;
}

int ecg_batch_layout(const ecg_batch* b, int* slice_height, int* sort_window, int* ctas, double* spmm_ms,
                     int* graph) {
  if (!b) return ECG_EINVAL;
  if (graph) *graph = b->graph_used ? 1 : 0;
  if (slice_height) *slice_height = b->C;
  if (sort_window) *sort_window = b->sigma;
  if (ctas) *ctas = b->G;
  if (spmm_ms) *spmm_ms = b->spmm_ms;
  return ECG_OK;
}

int ecg_batch_solve(ecg_batch* b, const double* const* rhs, const double* const* x0, double* const* x_out,
                    double tol, int maxit, ecg_result* res) {
  if (!b || !rhs || !x_out || !(tol >= 0.0) || maxit < 1) return ECG_EINVAL;
  for (int s = 0; s < b->nsys; s++)
    if (!rhs[s] || !x_out[s]) return ECG_EINVAL;
  BCK(cudaSetDevice(b->dev));
  cudaStream_t st = b->stream;
  const bool fp32 = (b->o.precision == ECG_MIXED);
  const int ns = b->nsys;
  // history: maxit + 1 entries per system
  if (b->hist_cap < maxit + 1) {
    bfree(b->d_hist);
    b->hist_cap = 0;
    int rc = balloc(&b->d_hist, (size_t)ns * (maxit + 1));
    if (rc) return rc;
    b->hist_cap = maxit + 1;
  }
  BCK(cudaMemsetAsync(b->d_hist, 0, sizeof(double) * (size_t)ns * b->hist_cap, st));
  // inputs
  const bool dev_in = dev_ptr(rhs[0]);
  for (int s = 0; s < ns; s++) {
    BCK(cudaMemcpyAsync(b->d_b + b->off[s], rhs[s], sizeof(double) * b->n[s],
                        dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (x0 && x0[s]) {
      BCK(cudaMemcpyAsync(b->d_x + b->off[s], x0[s], sizeof(double) * b->n[s],
                          dev_ptr(x0[s]) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    } else {
      BCK(cudaMemsetAsync(b->d_x + b->off[s], 0, sizeof(double) * b->n[s], st));
    }
  }
  BCK(cudaMemsetAsync(b->d_outer, 0, sizeof(Outer) * ns, st));
  {
    std::vector<SysState> s0(ns);
    for (auto& x : s0) {
      std::memset(&x, 0, sizeof(x));
      x.status = B_OK;  // not running until a round starts it
    }
    BCK(cudaMemcpyAsync(b->d_st, s0.data(), sizeof(SysState) * ns, cudaMemcpyHostToDevice, st));
  }
  BCK(cudaEventRecord(b->e0, st));
  {
    const BatchP B = make_bp(b, fp32);
    k_batch_residual<<<b->G, kBThreads, 0, st>>>(B, b->d_sval, b->d_x, b->d_b, b->d_r, b->d_part2);
    k_batch_norms<<<(ns + 127) / 128, 128, 0, st>>>(ns, b->d_first, b->d_gsize, b->d_part2, b->d_rr, b->d_bb);
    BCK(cudaGetLastError());
  }
  // rounds, captured once as a CUDA graph and replayed until no system runs
  // (issued directly when the capture is refused)
  const int max_rounds = fp32 ? 64 : 1;
  cudaGraphExec_t exec = nullptr;
  {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int rc = enqueue_round(b, fp32, tol, maxit, max_rounds);
      const cudaError_t e = cudaStreamEndCapture(st, &g);
      if (rc == ECG_OK && e == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
  }
  int rc = ECG_OK;
  for (int round = 0; round <= max_rounds + 1; round++) {
    const int rr_ = exec ? (cudaGraphLaunch(exec, st) == cudaSuccess ? ECG_OK : ECG_ECUDA)
                         : enqueue_round(b, fp32, tol, maxit, max_rounds);
    if (rr_ != ECG_OK ||
        cudaMemcpyAsync(b->h_active, b->d_active, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      rc = ECG_ECUDA;
      break;
    }
    if (*b->h_active == 0) break;
  }
  b->graph_used = exec != nullptr;
  if (exec) cudaGraphExecDestroy(exec);
  if (rc) return rc;
  BCK(cudaEventRecord(b->e1, st));
  // results
  std::vector<Outer> O(ns);
  std::vector<SysState> S(ns);
  std::vector<double> rr(ns), bb(ns);
  BCK(cudaMemcpyAsync(O.data(), b->d_outer, sizeof(Outer) * ns, cudaMemcpyDeviceToHost, st));
  BCK(cudaMemcpyAsync(S.data(), b->d_st, sizeof(SysState) * ns, cudaMemcpyDeviceToHost, st));
  BCK(cudaMemcpyAsync(rr.data(), b->d_rr, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
  BCK(cudaMemcpyAsync(bb.data(), b->d_bb, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
  b->h_hist.assign((size_t)ns * b->hist_cap, 0.0);
  BCK(cudaMemcpyAsync(b->h_hist.data(), b->d_hist, sizeof(double) * b->h_hist.size(), cudaMemcpyDeviceToHost, st));
  const bool dev_out = dev_ptr(x_out[0]);
  for (int s = 0; s < ns; s++)
    BCK(cudaMemcpyAsync(x_out[s], b->d_x + b->off[s], sizeof(double) * b->n[s],
                        dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->e0, b->e1);
  int worst = ECG_OK;
  for (int s = 0; s < ns; s++) {
    const int status = O[s].done ? O[s].status : ECG_ENOCONV;
    if (worst == ECG_OK && status != ECG_OK) worst = status;
    if (res) {
      ecg_result& r = res[s];
      std::memset(&r, 0, sizeof(r));
      r.iters = O[s].iters;
      r.status = status;
      r.mem_vectors = (int64_t)b->t * (b->o.trunc + 1);
      if (fp32) r.relres = O[s].rho0 > 0.0 ? std::sqrt(rr[s]) / O[s].rho0 : std::sqrt(rr[s]);
      else r.relres = S[s].rho0 > 0.0 ? S[s].rho / S[s].rho0 : S[s].rho;
      r.relres_true = bb[s] > 0.0 ? std::sqrt(rr[s] / bb[s]) : std::sqrt(rr[s]);
      r.device_ms = ms;
      r.history = b->h_hist.data() + (size_t)s * b->hist_cap;
    }
  }
  return worst;
}

}  // extern "C"
