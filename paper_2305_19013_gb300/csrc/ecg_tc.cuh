// ecg_tc.cuh -- FP64 block products of the CGS2 step on the tensor cores
// (tcgen05, sm_103a).
//
// GB300 issues about 1.2 TFLOP/s of FP64 FMA against 6.7 TB/s of HBM, so
// the FP64 CGS2 kernels of ecg_kernels.cuh are bound by FP64 issue (each
// row of the window update W -= Q C costs 2 m t^2 FMAs).  The kernels here
// compute the same FP64 products exactly enough for FP64 results, on the
// FP16 tensor pipe, by the error-free splitting of Ozaki, Ogita, Oishi and
// Rump ("Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer.
// Algorithms 59, 2012), in the fixed-point form used for tensor cores by
// Mukunoki, Ozaki, Ogita and Imamura ("DGEMM using Tensor Cores, and Its
// Accurate and Reproducible Versions", ISC 2020):
//
//   - every row of Q (and every column of C) gets a power-of-two scale from
//     its largest binary exponent, so that each scaled entry lies in (-1, 1);
//   - the scaled entry is truncated to a 64-bit fixed-point fraction U and
//     cut into 8 digits of 8 bits, d_0 (most significant) .. d_7, each an
//     integer in [-255, 255] that FP16 holds exactly;
//   - the MMA multiplies digit matrices: FP16 x FP16 products of such
//     integers are exact, and every FP32 sum in the accumulator stays an
//     integer below 2^24, so the tensor-core accumulation is exact;
//   - digit pairs (p, r) with the same p + r = g share a group accumulator
//     (same binary weight 2^{-8(g+2)}); groups g <= 8 are kept;
//   - the group sums are combined into one 128-bit integer and rounded once
//     to FP64 with integer instructions only; the FP64 pipe does one
//     subtraction per output (X - Q C).
//
// Error.  Each operand is truncated at 2^-64 of its scale and the dropped
// groups (g >= 9) weigh below 2^-64; the computed Q C differs from the
// exact product of the FP64 inputs by less than about 2^-60 x (row scale) x
// (column scale) x window columns, below FP64's own rounding of a dot
// product of that length (2^-53 per term).
//
// Exactness of the accumulator.  Group g sums at most 8 digit pairs over at
// most 32 window columns: |sum| <= 8 * 32 * 255^2 = 16,646,400 < 2^24.  So
// the kernels take windows of at most 32 columns (m t <= 32: the truncated
// methods at t = 16 with two blocks, t = 8 with up to four).
//
// Rounding of non-finite input: a row or column whose scale is Inf/NaN
// gives NaN outputs; subnormal inputs count as zero (below 2^-1022).
#pragma once
#include <cuda_fp16.h>
#include <cstdint>

#include "ecg_kernels.cuh"

namespace ecg {
namespace tc {

// ------------------------------------------------------------ tcgen05 PTX

// Allocate ncols TMEM columns (power of two, 32..512) for this CTA; the
// address is written to *dst (shared memory).  One whole warp executes it.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle: start address, leading
// (K-direction core-matrix) byte offset, stride (M/N-direction 8-row group)
// byte offset; bit 46 is the fixed descriptor version.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor of kind::f16: FP16 A and B (both K-major), FP32 D.
__host__ __device__ constexpr uint32_t idesc_f16(int m, int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// D[tmem] (+)= A * B, issued by one thread.
__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on *bar once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 8 consecutive 32-bit TMEM columns of this warp's 32 lanes (lane quarter
// of the warp) into v; tmem_wait_ld() before use.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 16-byte asynchronous copy global -> shared (both addresses 16-byte
// aligned), cached in L2 only; cp_async16_wait waits for this thread's
// copies.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async16_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Bounded wait on an mbarrier phase (kWaitNs of %globaltimer time).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (long long p = 0; p < kWaitPolls; p += 64) {
    for (int q = 0; q < 64; q++)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// Element (r, k) of a K-major, unswizzled operand tile of R rows and K
// columns (FP16): 8 x 8 core matrices of 128 contiguous bytes, K-direction
// core matrices adjacent (LBO = 128 B), row groups K/8 core matrices apart
// (SBO = K * 16 B).
__device__ __forceinline__ int kmaj(int r, int k, int K) { return ((r >> 3) * (K >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

// ------------------------------------------------------- fixed-point digits

// Biased binary exponent of v (0 for zero and subnormals, 2047 for Inf/NaN).
__device__ __forceinline__ int bexp(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7FF); }

// |v| / 2^(S - 1022) as a 64-bit fraction, truncated: U = floor(|v| 2^(64 -
// (S - 1022))) for the biased scale exponent S >= bexp(v).
__device__ __forceinline__ unsigned long long fixed64(double v, int S) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = S - e;
  return (e == 0 || sh >= 64) ? 0ull : ((m << 11) >> sh);
}

// Digit p (0: most significant) of two fractions u0, u1 as an FP16 pair
// (low half from u0), with signs s0, s1 (0 or 1): the byte is placed under
// the FP16 exponent of 1024 (0x6400 | d = 1024 + d exactly), and
// (1024 + d) * sgn - 1024 * sgn gives +-d exactly.
__device__ __forceinline__ uint32_t digit_pair(unsigned long long u0, unsigned long long u1, int p, __half2 sgn,
                                               __half2 off) {
  const int sh = 56 - 8 * p;
  const uint32_t d0 = (uint32_t)(u0 >> sh) & 0xFFu, d1 = (uint32_t)(u1 >> sh) & 0xFFu;
  const uint32_t raw = 0x64006400u | d0 | (d1 << 16);
  const __half2 h = __hfma2(*reinterpret_cast<const __half2*>(&raw), sgn, off);
  return *reinterpret_cast<const uint32_t*>(&h);
}
// The digits in byte k (0..3, compile time) of the 32-bit words w0 and w1
// as an FP16 pair under the exponent of 1024 (two byte permutations), then
// signed and unbiased by one FP16x2 FMA: (1024 + d) sgn - 1024 sgn = +-d.
__device__ __forceinline__ uint32_t digit_pair_bytes(uint32_t w0, uint32_t w1, int k, __half2 sgn, __half2 off) {
  const uint32_t t = __byte_perm(w0, w1, (uint32_t)(k | ((4 + k) << 4)));  // [w0.k, w1.k, -, -]
  const uint32_t raw = __byte_perm(t, 0x64646464u, 0x4140u);               // [w0.k, 0x64, w1.k, 0x64]
  const __half2 h = __hfma2(*reinterpret_cast<const __half2*>(&raw), sgn, off);
  return *reinterpret_cast<const uint32_t*>(&h);
}
// Digit p (0: most significant) of two 64-bit fractions.
__device__ __forceinline__ uint32_t digit_pair64(unsigned long long u0, unsigned long long u1, int p, __half2 sgn,
                                                 __half2 off) {
  const int byte = 7 - p;
  const uint32_t w0 = byte >= 4 ? (uint32_t)(u0 >> 32) : (uint32_t)u0;
  const uint32_t w1 = byte >= 4 ? (uint32_t)(u1 >> 32) : (uint32_t)u1;
  return digit_pair_bytes(w0, w1, byte & 3, sgn, off);
}
__device__ __forceinline__ void sign_pair(double v0, double v1, __half2& sgn, __half2& off) {
  const __half a = __double_as_longlong(v0) < 0 ? __float2half(-1.f) : __float2half(1.f);
  const __half b = __double_as_longlong(v1) < 0 ? __float2half(-1.f) : __float2half(1.f);
  sgn = __halves2half2(a, b);
  off = __halves2half2(__hmul(a, __float2half(-1024.f)), __hmul(b, __float2half(-1024.f)));
}

// (hi * 2^64 + lo) * 2^E rounded to the nearest double (ties to even), the
// 128-bit integer in two's complement.  Results below 2^-1022 flush to
// zero, results beyond the double range give Inf.
__device__ __forceinline__ double i128_to_double(long long hi, unsigned long long lo, int E) {
  unsigned long long sign = 0;
  unsigned long long uh = (unsigned long long)hi, ul = lo;
  if (hi < 0) {
    sign = 1ull << 63;
    ul = ~ul + 1ull;
    uh = ~uh + (ul == 0ull ? 1ull : 0ull);
  }
  if (uh == 0ull && ul == 0ull) return 0.0;
  int msb = uh ? 127 - __clzll((long long)uh) : 63 - __clzll((long long)ul);
  unsigned long long m;
  int sh = msb - 52;
  if (sh <= 0) {
    m = ul << (-sh);
  } else {  // sh <= 75; the integers here stay below 2^117, so sh < 64
    m = (sh == 0) ? ul : ((uh << (64 - sh)) | (ul >> sh));
    const unsigned long long rem = ul & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) {
      m++;
      if (m == (1ull << 53)) {
        m >>= 1;
        sh++;
      }
    }
  }
  const int be = sh + E + 52 + 1023;
  if (be >= 2047) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
  if (be <= 0) return __longlong_as_double((long long)sign);
  return __longlong_as_double((long long)(sign | ((unsigned long long)be << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

// (hi, lo) += v * 2^sh for an integer v (|v| < 2^31) and 0 <= sh <= 64,
// in 128-bit two's complement.
__device__ __forceinline__ void i128_add_shifted(long long& hi, unsigned long long& lo, long long v, int sh) {
  long long ah;
  unsigned long long al;
  if (sh == 0) {
    ah = v >> 63;
    al = (unsigned long long)v;
  } else if (sh >= 64) {
    ah = v;
    al = 0ull;
  } else {
    ah = v >> (64 - sh);
    al = (unsigned long long)v << sh;
  }
  const unsigned long long s = lo + al;
  hi += ah + (s < lo ? 1ll : 0ll);
  lo = s;
}

// Group sums D_0 .. D_8 (weights 2^{8(8-g)}) as one 128-bit integer.
__device__ __forceinline__ void groups_to_i128(const float (&D)[9], long long& hi, unsigned long long& lo) {
  long long L = 0, H = 0;
#pragma unroll
  for (int g = 8; g >= 4; g--) L += (long long)__float2int_rn(D[g]) << (8 * (8 - g));
#pragma unroll
  for (int g = 3; g >= 0; g--) H += (long long)__float2int_rn(D[g]) << (8 * (3 - g));
  // T = H 2^40 + L
  const unsigned long long hl = (unsigned long long)H << 40;
  lo = hl + (unsigned long long)L;
  const unsigned long long carry = (lo < hl) ? 1ull : 0ull;
  hi = (H >> 24) + (L < 0 ? -1ll : 0ll) + (long long)carry;
}

// ------------------------------------------------------------ CGS update

// Xout = Xsrc - Q C for a window of at most 32 columns and block width W:
// 128-row tiles, the MMA's M = 128 rows, A = the 8 digit slabs of the
// tile's Q rows (K = 8 x 32), B = the digits of C stacked by digit
// (N = 9 W: digit rows r = 0..8, r = 8 zero), slab p accumulating into
// groups p .. 8 (TMEM columns p W ..).
template <int W>
struct UpdTc {
  static constexpr int R = 128;       // rows per tile
  static constexpr int KC = 32;       // window columns (K per digit slab)
  static constexpr int ND = 8;        // digits per operand
  static constexpr int NG = 9;        // groups kept (g = 0..8)
  static constexpr int KA = ND * KC;  // A tile K
  static constexpr int NB = NG * W;   // B rows (digit r = 0..8)
  static constexpr uint32_t TCOLS = (NG * W <= 128) ? 128u : 256u;
  // shared memory: A tile, B tile, scales, barrier
  static constexpr size_t A_BYTES = (size_t)R * KA * 2;
  static constexpr size_t B_BYTES = (size_t)NB * KC * 2;
  static constexpr size_t Q_BYTES = (size_t)R * KC * 8;  // the next tile's window rows (FP64)
  static constexpr size_t SMEM = A_BYTES + B_BYTES + Q_BYTES + 4 * (W + R);  // + column and row scales
};

template <int W>
constexpr size_t smem_update_tc() {
  return UpdTc<W>::SMEM;
}

// True when the tensor-core update applies: FP64, W = 16, and a window of
// at most 32 columns (wcap is the most the launch will see).
template <typename T, int W>
__host__ __device__ constexpr bool update_tc_ok(int wcap) {
  return sizeof(T) == 8 && W == 16 && wcap <= 32;
}

template <int W>
__global__ void __launch_bounds__(256, 2) k_update_tc(KP P, int gw, double* Xio, const double* Cin) {
  static_assert(W == 16, "the epilogue maps two 8-column halves of W = 16 onto the eight warps");
  using U = UpdTc<W>;
  constexpr int R = U::R, KC = U::KC, KA = U::KA, NB = U::NB;
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  const int nq = st->nq;
  if (nq <= 0) return;
  const BlockDesc* D = P.desc;
  const int wtot = D[nq - 1].off + D[nq - 1].w;
  if (wtot > KC) {  // not reached: the host launches this form only for windows of <= 32 columns
    if (threadIdx.x == 0) {
      ((DevState*)st)->status = ST_ECUDA;
      ((DevState*)st)->stop = 1;
    }
    return;
  }
  const double* Xsrc = (P.sre_src && !P.prec && st->gen == GEN_SRE) ? (const double*)D[nq - 1].V : Xio;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __half* sA = (__half*)smem_raw;                         // R x KA, K-major
  __half* sB = (__half*)(smem_raw + U::A_BYTES);          // NB x KC, K-major
  double* sQs = (double*)(smem_raw + U::A_BYTES + U::B_BYTES);  // R x KC staged window rows
  int* sScaleC = (int*)(smem_raw + U::A_BYTES + U::B_BYTES + U::Q_BYTES);  // W column scales of C, then R row scales
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  __shared__ const double* colp[KC];  // column c of the window: pointer to row 0's entry
  __shared__ int cols[KC];            // and its row stride (block width)
  __shared__ int staged;              // 1: window rows arrive by 16-byte cp.async
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // window columns
  if (tid < KC) {
    const double* p = nullptr;
    int w = 0;
    if (tid < wtot) {
      int j = 0;
      while (j + 1 < nq && D[j + 1].off <= tid) j++;
      p = (const double*)D[j].W + (tid - D[j].off);
      w = D[j].w;
    }
    colp[tid] = p;
    cols[tid] = w;
  }
  if (tid == 0) {  // every block 16-byte aligned with an even width: pairs of columns are 16-byte chunks
    int okst = 1;
    for (int j = 0; j < nq; j++) okst &= ((((uintptr_t)D[j].W) & 15) == 0) && ((D[j].w & 1) == 0);
    staged = okst;
  }
  // C's column scales and digits: B[r W + b][a] = digit r of C[a][b] (r < 8),
  // zero for r = 8 and for a >= wtot
  if (tid < W) {
    int s = 0;
    for (int a = 0; a < wtot; a++) s = max(s, bexp(Cin[a * W + tid]));
    sScaleC[tid] = s;
  }
  __syncthreads();
  for (int e = tid; e < NB * (KC / 2); e += blockDim.x) {
    const int n = e / (KC / 2), a = 2 * (e % (KC / 2));
    const int r = n / W, b = n % W;
    uint32_t v = 0;
    if (r < 8 && a < wtot) {
      const double c0 = Cin[a * W + b];
      const double c1 = (a + 1 < wtot) ? Cin[(a + 1) * W + b] : 0.0;
      __half2 sg, of;
      sign_pair(c0, c1, sg, of);
      v = digit_pair(fixed64(c0, sScaleC[b]), fixed64(c1, sScaleC[b]), r, sg, of);
    }
    *reinterpret_cast<uint32_t*>(&sB[kmaj(n, a, KC)]) = v;
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tbase, U::TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  bool cnan = false;
  for (int b = 0; b < W; b++) cnan = cnan || (sScaleC[b] == 2047);

  int r0, r1;
  cta_rows_aligned(P.n, R, r0, r1);
  const int ntiles = (r1 - r0 + R - 1) / R;
  // slicing: thread (row = tid / 2, half = tid % 2) takes window columns
  // [16 half, 16 half + 16) of its row
  const int srow = tid >> 1, shalf = tid & 1;
  const bool use_stage = staged != 0;
  // the window rows of tile i: 16-byte chunks (row, column pair), 8 per thread
  auto stage_tile = [&](int i) {
    const int rb = r0 + i * R, nrr = min(R, r1 - rb);
    for (int ch = tid; ch < R * (KC / 2); ch += blockDim.x) {
      const int rr = ch / (KC / 2), c2 = 2 * (ch % (KC / 2));
      const double* p = colp[c2];
      // 16-byte chunk c2 / 2 of row rr lands at chunk (c2 / 2) ^ (rr % 16): the
      // slicing threads of a warp (16 rows) then read distinct bank groups
      if (p && rr < nrr) cp_async16(&sQs[rr * KC + 2 * ((c2 >> 1) ^ (rr & 15))], p + (long long)(rb + rr) * cols[c2]);
    }
    cp_async16_commit();
  };
  if (use_stage && ntiles > 0) stage_tile(0);
  bool ok = true;
  int it = 0;
  for (; it < ntiles && ok; it++) {
    const int row0 = r0 + it * R;
    const int nr = min(R, r1 - row0);
    if (use_stage) {
      cp_async16_wait();
      __syncthreads();  // tile it is in sQs
    }
    {
      const int grow = row0 + srow;
      double q[16];
      int smax = 0;
#pragma unroll
      for (int c = 0; c < 16; c++) {
        const int col = 16 * shalf + c;
        const double* p = colp[col];
        if (use_stage) q[c] = (p && srow < nr) ? sQs[srow * KC + 2 * ((col >> 1) ^ (srow & 15)) + (col & 1)] : 0.0;
        else q[c] = (p && srow < nr) ? p[(long long)grow * cols[col]] : 0.0;
        smax = max(smax, bexp(q[c]));
      }
      smax = max(smax, __shfl_xor_sync(0xffffffffu, smax, 1));
      if (smax == 2047) {  // a non-finite row: zero digits here, NaN output in the epilogue
#pragma unroll
        for (int c = 0; c < 16; c++) q[c] = 0.0;
      }
      const int S = (smax == 2047) ? 0 : smax;
#pragma unroll
      for (int c = 0; c < 16; c += 2) {
        const unsigned long long u0 = fixed64(q[c], S), u1 = fixed64(q[c + 1], S);
        __half2 sg, of;
        sign_pair(q[c], q[c + 1], sg, of);
#pragma unroll
        for (int p = 0; p < 8; p++)
          *reinterpret_cast<uint32_t*>(&sA[kmaj(srow, p * KC + 16 * shalf + c, KA)]) = digit_pair64(u0, u1, p, sg, of);
      }
      if (shalf == 0) sScaleC[W + srow] = smax;  // the row scale, for the epilogue
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    // every thread has read sQs: bring in the next tile while this one runs
    if (use_stage && it + 1 < ntiles) stage_tile(it + 1);
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      // slab p: A columns [p KC, (p+1) KC), B digit rows r <= 8 - p (all 9
      // for p = 0, so that the first MMA initialises every group column)
      for (int p = 0; p < 8; p++) {
        const int nrows = (p == 0 ? 9 : 9 - p) * W;
        const uint32_t idesc = idesc_f16(R, nrows);
        for (int ks = 0; ks < KC / 16; ks++) {
          const uint64_t ad = sdesc(a0 + (uint32_t)((p * KC + ks * 16) / 8) * 128u, 128u, (uint32_t)(KA / 8) * 128u);
          const uint64_t bd = sdesc(b0 + (uint32_t)(ks * 16 / 8) * 128u, 128u, (uint32_t)(KC / 8) * 128u);
          mma_f16(tmem + (uint32_t)(p * W), ad, bd, idesc, (p > 0 || ks > 0) ? 1u : 0u);
        }
      }
      mma_commit(&bar);
    }
    const bool done = mbar_wait_bounded(&bar, (uint32_t)(it & 1));
    ok = __syncthreads_and(done);
    if (!ok) break;  // it stays the tile whose MMAs did not complete
    tc_fence_after();
    // epilogue: warp w reads rows 32 (w % 4) + lane, columns b in
    // [8 (w / 4), 8 (w / 4) + 8) (W = 16) of the nine groups
    {
      const int row = 32 * (warp & 3) + lane;
      const int bq = 8 * (warp >> 2);
      float g[8][9];
      {
        uint32_t v[9][8];
#pragma unroll
        for (int gi = 0; gi < 9; gi++)
          tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(gi * W + bq), v[gi]);
        tmem_wait_ld();
#pragma unroll
        for (int gi = 0; gi < 9; gi++)
#pragma unroll
          for (int j = 0; j < 8; j++) g[j][gi] = __uint_as_float(v[gi][j]);
      }
      const int Si = sScaleC[W + row];
      if (row < nr) {
        const long long grow = row0 + row;
#pragma unroll
        for (int j = 0; j < 8; j++) {
          const int b = bq + j;
          long long hi;
          unsigned long long lo;
          groups_to_i128(g[j], hi, lo);
          const int Sb = sScaleC[b];
          double pq;
          if (Si == 2047 || cnan) pq = __longlong_as_double(0x7FF8000000000000ll);
          else pq = i128_to_double(hi, lo, (Si - 1022) + (Sb - 1022) - 80);
          Xio[grow * W + b] = Xsrc[grow * W + b] - pq;
        }
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  if (!ok && tid == 0) {
    ((DevState*)st)->fault = 1;
    ((DevState*)st)->status = ST_ECUDA;
    ((DevState*)st)->stop = 1;
    // give the MMAs in flight a second bounded wait before the columns are freed
    mbar_wait_bounded(&bar, (uint32_t)(it & 1));
  }
  cp_async16_wait();  // no copy may still be landing when the CTA exits
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, U::TCOLS);
}

// ------------------------------------------------------- CGS coefficients

// Digit splitting of one scalar type: ND digits of 8 bits of a fraction U
// with FB bits, value = sign * U 2^-FB 2^(S - BIAS) for the biased scale
// exponent S of the value's column tile; digit pairs (p, r) with p + r <=
// GMAX are kept.  FP64: 8 digits (64 bits >= the 53-bit significand),
// pairs up to p + r = 8 (the dropped ones weigh below 2^-80 of the
// scales).  FP32: 3 digits hold the 24-bit significand exactly and every
// pair is kept, so the FP32 product is exact before the FP64 sums.
template <typename T>
struct Digits;
template <>
struct Digits<double> {
  static constexpr int ND = 8, GMAX = 8, BIAS = 1022, FB = 64, EINF = 2047;
  __device__ static int bexp(double v) { return tc::bexp(v); }
  __device__ static unsigned long long fixed(double v, int S) { return fixed64(v, S); }
  __device__ static bool neg(double v) { return __double_as_longlong(v) < 0; }
};
template <>
struct Digits<float> {
  static constexpr int ND = 3, GMAX = 4, BIAS = 126, FB = 24, EINF = 255;
  __device__ static int bexp(float v) { return (int)((__float_as_uint(v) >> 23) & 0xFFu); }
  // |v| / 2^(S - 126) as a 24-bit fraction, truncated (exact when S = bexp(v))
  __device__ static unsigned long long fixed(float v, int S) {
    const uint32_t b = __float_as_uint(v);
    const int e = (int)((b >> 23) & 0xFFu);
    const uint32_t m = (b & 0x7FFFFFu) | 0x800000u;
    const int sh = S - e;
    return (e == 0 || sh >= 24) ? 0ull : (unsigned long long)(m >> sh);
  }
  __device__ static bool neg(float v) { return (__float_as_uint(v) >> 31) != 0u; }
};

// Signs of two values as the FP16 pair (sgn, off) that digit_pair_bytes
// takes.
__device__ __forceinline__ void sign_pair_b(bool n0, bool n1, __half2& sgn, __half2& off) {
  const __half one = __float2half(1.f), mone = __float2half(-1.f);
  const __half m1024 = __float2half(-1024.f), p1024 = __float2half(1024.f);
  sgn = __halves2half2(n0 ? mone : one, n1 ? mone : one);
  off = __halves2half2(n0 ? p1024 : m1024, n1 ? p1024 : m1024);
}
// Digit p of two fractions of scalar type T (FP64: 64 bits, FP32: 24 bits).
template <typename T>
__device__ __forceinline__ uint32_t digit_pair_t(unsigned long long u0, unsigned long long u1, int p, __half2 sgn,
                                                 __half2 off) {
  if constexpr (sizeof(T) == 8) return digit_pair64(u0, u1, p, sgn, off);
  else return digit_pair_bytes((uint32_t)u0, (uint32_t)u1, 2 - p, sgn, off);
}

// Digit pairs (p, r) kept by k_tdot_tc, numbered p by p: slot(p, r) =
// first(p) + r for r <= rmax(p) = min(ND - 1, GMAX - p).
template <typename T>
struct PairSlots {
  using Dg = Digits<T>;
  static constexpr __host__ __device__ int rmax(int p) {
    return (Dg::ND - 1 < Dg::GMAX - p) ? Dg::ND - 1 : Dg::GMAX - p;
  }
  static constexpr __host__ __device__ int first(int p) { return p == 0 ? 0 : first(p - 1) + rmax(p - 1) + 1; }
  static constexpr int COUNT = first(Dg::ND);
};

// Per-CTA partial sums of C = [V_0 .. V_{nq-1}]^T B for a window of at most
// 32 columns and W = 16, over the CTA's rows, into the partial-sum layout of
// k_tdot_window (reduced by k_reduce_C).  128-row tiles are the MMA's K.
// A = the V digits of the tile, M = (digit p, window column a): FP64 256
// rows in two MMAs (p < 4 and p >= 4; the second keeps B digits r <= 4),
// FP32 96 rows in one (rows 96..127 zero).  B = the B digits, N = (digit r,
// column b).  Every accumulator entry sums 128 exact products of at most
// 255^2: 128 * 65025 < 2^23.  The scales are per tile and column, so each
// tile's digit-pair sums are combined into 128-bit integers per (p, a, b),
// summed over p, rounded to FP64 and added to the CTA's FP64 sums.
template <typename T, int W>
struct TdotTc {
  using Dg = Digits<T>;
  static constexpr int ND = Dg::ND;
  static constexpr int R = 128;                              // rows per tile (MMA K)
  static constexpr int KC = 32;                              // window columns
  static constexpr int MA = (ND * KC > 128) ? ND * KC : 128;  // A rows (digit, column), padded
  static constexpr int NB = ND * W;                          // B rows (digit, column)
  static constexpr int N2 = (Dg::GMAX - 4 + 1) * W;           // second MMA (FP64): r <= GMAX - 4
  static constexpr uint32_t TCOLS = (ND * KC > 128) ? 256u : 64u;
  static constexpr size_t A_BYTES = (size_t)MA * R * 2;
  static constexpr size_t B_BYTES = (size_t)NB * R * 2;
  // the int32 digit-pair sums, one slot per kept pair (p, r) and output
  // (b, a), reuse the A and B tiles once the MMAs are done
  static constexpr size_t PART_BYTES = (size_t)PairSlots<T>::COUNT * KC * W * 4;
  static constexpr size_t SMEM = A_BYTES + B_BYTES + 4 * (KC + W);
  static_assert(PART_BYTES <= A_BYTES + B_BYTES, "pair sums alias the A and B tiles");
  static_assert(NB + (ND * KC > 128 ? N2 : 0) <= (int)TCOLS, "accumulator columns");
};

template <typename T, int W>
constexpr size_t smem_tdot_tc() {
  return TdotTc<T, W>::SMEM;
}

template <typename T, int W>
__host__ __device__ constexpr bool tdot_tc_ok(int wcap) {
  return W == 16 && wcap <= 32;
}

// float holding an integer of magnitude below 2^24, to int (exact)
__device__ __forceinline__ int f2i_exact(float f) { return __float2int_rn(f); }

template <typename T, int W>
__global__ void __launch_bounds__(256, 2) k_tdot_tc(KP P, int gw, const T* B) {
  static_assert(W == 16, "16 B columns per tile row");
  using U = TdotTc<T, W>;
  using Dg = typename U::Dg;
  constexpr int R = U::R, KC = U::KC, NB = U::NB, N2 = U::N2, ND = U::ND;
  constexpr bool TWO = (ND * KC > 128);  // FP64: two MMAs per k-step
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  const int nq = st->nq;
  if (nq <= 0) return;
  const BlockDesc* D = P.desc;
  const int wtot = D[nq - 1].off + D[nq - 1].w;
  if (wtot > KC || blockIdx.y != 0) {  // not reached: launched only for windows of <= 32 columns
    if (threadIdx.x == 0 && wtot > KC) {
      ((DevState*)st)->status = ST_ECUDA;
      ((DevState*)st)->stop = 1;
    }
    return;
  }
  if (P.sre_src && !P.prec && st->gen == GEN_SRE) B = (const T*)D[nq - 1].V;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __half* sA = (__half*)smem_raw;                          // MA x R, K-major
  __half* sB = (__half*)(smem_raw + U::A_BYTES);           // NB x R, K-major
  int* sSv = (int*)(smem_raw + U::A_BYTES + U::B_BYTES);  // KC column scales of V
  int* sSx = sSv + KC;                                     // W column scales of B
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  __shared__ const T* colp[KC];
  __shared__ int cols[KC];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < KC) {
    const T* p = nullptr;
    int w = 0;
    if (tid < wtot) {
      int j = 0;
      while (j + 1 < nq && D[j + 1].off <= tid) j++;
      p = (const T*)D[j].V + (tid - D[j].off);
      w = D[j].w;
    }
    colp[tid] = p;
    cols[tid] = w;
  }
  if constexpr (ND * KC < U::MA) {  // padding rows of A stay zero
    for (int e = tid; e < (U::MA - ND * KC) * R / 2; e += blockDim.x)
      reinterpret_cast<uint32_t*>(sA + (size_t)ND * KC * R)[e] = 0u;
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tbase, U::TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;

  int r0, r1;
  cta_rows_aligned(P.n, R, r0, r1);
  const int ntiles = (r1 - r0 + R - 1) / R;
  // loading and slicing.  V: column va = tid % 8 + 8 (warp % 4), row pairs
  // kp = (tid / 8) % 4 + 4 (warp / 4 + 2 j), j < 8; B: column xb = tid % 8 +
  // 8 (warp % 2), row pairs (tid / 8) % 4 + 4 (warp / 2 + 4 j), j < 4.  A
  // warp then covers 8 columns x 4 row pairs, and its 32 digit-pair stores
  // hit 32 different banks of the K-major core matrices.
  const int kpl = (tid >> 3) & 3;
  const int va = (tid & 7) + 8 * (warp & 3), vg = warp >> 2;
  const int xb = (tid & 7) + 8 * (warp & 1), xg = warp >> 1;
  // outputs of this thread: (a, b) = (tid % 32, tid / 32) and (tid % 32, tid / 32 + 8)
  double acc0 = 0.0, acc1 = 0.0;
  bool ok = true;
  int it = 0;
  for (; it < ntiles && ok; it++) {
    const int row0 = r0 + it * R;
    const int nr = min(R, r1 - row0);
    if (tid < KC + W) sSv[tid] = 0;  // sSx follows sSv
    __syncthreads();
    T v[8][2], x[4][2];
    {
      const T* p = colp[va];
      const long long cs = cols[va];
      int mx = 0;
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const int rr = 2 * (kpl + 4 * (vg + 2 * j));
#pragma unroll
        for (int u = 0; u < 2; u++) {
          v[j][u] = (p && rr + u < nr) ? p[(long long)(row0 + rr + u) * cs] : T(0);
          mx = max(mx, Dg::bexp(v[j][u]));
        }
      }
      // lanes with the same column differ in bits 3 and 4
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
      if (kpl == 0) atomicMax(&sSv[va], mx);
      int mb = 0;
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const int rr = 2 * (kpl + 4 * (xg + 4 * j));
#pragma unroll
        for (int u = 0; u < 2; u++) {
          x[j][u] = (rr + u < nr) ? B[(long long)(row0 + rr + u) * W + xb] : T(0);
          mb = max(mb, Dg::bexp(x[j][u]));
        }
      }
      mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, 8));
      mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, 16));
      if (kpl == 0) atomicMax(&sSx[xb], mb);
    }
    __syncthreads();
    {
      const bool vinf = sSv[va] == Dg::EINF;  // non-finite column: zero digits, NaN output below
      const int Sv = vinf ? 0 : sSv[va];
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const T a0 = vinf ? T(0) : v[j][0], a1 = vinf ? T(0) : v[j][1];
        const unsigned long long u0 = Dg::fixed(a0, Sv), u1 = Dg::fixed(a1, Sv);
        __half2 sg, of;
        sign_pair_b(Dg::neg(a0), Dg::neg(a1), sg, of);
        const int k = 2 * (kpl + 4 * (vg + 2 * j));
#pragma unroll
        for (int p = 0; p < ND; p++)
          *reinterpret_cast<uint32_t*>(&sA[kmaj(p * KC + va, k, R)]) = digit_pair_t<T>(u0, u1, p, sg, of);
      }
      const bool xinf = sSx[xb] == Dg::EINF;
      const int Sx = xinf ? 0 : sSx[xb];
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const T b0 = xinf ? T(0) : x[j][0], b1 = xinf ? T(0) : x[j][1];
        const unsigned long long u0 = Dg::fixed(b0, Sx), u1 = Dg::fixed(b1, Sx);
        __half2 sg, of;
        sign_pair_b(Dg::neg(b0), Dg::neg(b1), sg, of);
        const int k = 2 * (kpl + 4 * (xg + 4 * j));
#pragma unroll
        for (int r = 0; r < ND; r++)
          *reinterpret_cast<uint32_t*>(&sB[kmaj(r * W + xb, k, R)]) = digit_pair_t<T>(u0, u1, r, sg, of);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      const uint32_t sbo = (uint32_t)(R / 8) * 128u;
      for (int ks = 0; ks < R / 16; ks++) {
        const uint32_t ko = (uint32_t)(ks * 16 / 8) * 128u;
        const uint64_t bd = sdesc(b0 + ko, 128u, sbo);
        // FP64: digits p < 4 in A rows [0, 128) x all B rows, p >= 4 in A
        // rows [128, 256) x B digit rows r <= GMAX - 4; FP32: one MMA
        mma_f16(tmem, sdesc(a0 + ko, 128u, sbo), bd, idesc_f16(128, NB), ks > 0 ? 1u : 0u);
        if constexpr (TWO)
          mma_f16(tmem + (uint32_t)NB, sdesc(a0 + (uint32_t)(128 / 8) * sbo + ko, 128u, sbo), bd,
                  idesc_f16(128, N2), ks > 0 ? 1u : 0u);
      }
      mma_commit(&bar);
    }
    const bool done = mbar_wait_bounded(&bar, (uint32_t)(it & 1));
    ok = __syncthreads_and(done);
    if (!ok) break;
    tc_fence_after();
    // drain: warp w holds digit p = 4 (w / 4) + w % 4 (FP64; FP32: p = w for
    // w < 3) of window column a = lane; every kept digit-pair sum D_{p r}[a][b]
    // (an exact integer below 2^23) goes to its int32 slot
    {
      const int region = warp >> 2, q = warp & 3;
      const int p = TWO ? 4 * region + q : (region == 0 ? q : ND);
      // the MMAs have completed (barrier above): the A and B tiles are free
      int* slots = reinterpret_cast<int*>(smem_raw);
      if (p < ND) {  // uniform over the warp
        const int rmax = PairSlots<T>::rmax(p), s0 = PairSlots<T>::first(p);
        const uint32_t base = tmem + ((uint32_t)(32 * q) << 16) + (region ? (uint32_t)NB : 0u);
        for (int r = 0; r <= rmax; r++) {
          uint32_t t0[8], t1[8];
          tmem_ld8(base + (uint32_t)(r * W), t0);
          tmem_ld8(base + (uint32_t)(r * W + 8), t1);
          tmem_wait_ld();
          int* dst = slots + (s0 + r) * (KC * W) + lane;  // [slot][b][a]
#pragma unroll
          for (int j = 0; j < 8; j++) {
            dst[j * KC] = f2i_exact(__uint_as_float(t0[j]));
            dst[(8 + j) * KC] = f2i_exact(__uint_as_float(t1[j]));
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    {
#pragma unroll
      for (int h = 0; h < 2; h++) {
        // output (a, b) = (tid % 32, tid / 32 + 8 h): a warp reads 32 consecutive slots
        const int a = tid & 31, b = (tid >> 5) + 8 * h;
        const int* slots = reinterpret_cast<const int*>(smem_raw);
        // group sums in int32 (at most 8 pairs x 2^23 < 2^31), then one
        // 128-bit combine T = sum_g G_g 2^{8 (GMAX - g)}
        int G[Dg::GMAX + 1];
#pragma unroll
        for (int g = 0; g <= Dg::GMAX; g++) G[g] = 0;
#pragma unroll
        for (int p = 0; p < ND; p++)
#pragma unroll
          for (int r = 0; r <= PairSlots<T>::rmax(p); r++)
            G[p + r] += slots[(PairSlots<T>::first(p) + r) * (KC * W) + b * KC + a];
        long long hi = 0;
        unsigned long long lo = 0;
#pragma unroll
        for (int g = 0; g <= Dg::GMAX; g++) i128_add_shifted(hi, lo, (long long)G[g], 8 * (Dg::GMAX - g));
        double val;
        if (sSv[a] == Dg::EINF || sSx[b] == Dg::EINF) val = __longlong_as_double(0x7FF8000000000000ll);
        else val = i128_to_double(hi, lo, (sSv[a] - Dg::BIAS) + (sSx[b] - Dg::BIAS) - 8 * (Dg::GMAX + 2));
        if (h == 0) acc0 += val;
        else acc1 += val;
      }
    }
    __syncthreads();
  }
  if (!ok && tid == 0) {
    ((DevState*)st)->fault = 1;
    ((DevState*)st)->status = ST_ECUDA;
    ((DevState*)st)->stop = 1;
    mbar_wait_bounded(&bar, (uint32_t)(it & 1));
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, U::TCOLS);
  if (!ok) return;
  double* out = P.part_buf + (long long)blockIdx.x * (kChunk * W);
  const int a0 = tid & 31, b0 = tid >> 5;
  if (a0 < wtot) {
    out[a0 * W + b0] = acc0;
    out[a0 * W + b0 + 8] = acc1;
  }
}

// ------------------------------------------------------------ final update

// W_k = X R^{-1} and V_k = Y R^{-1} into the window slot, x += W_k alpha,
// r -= V_k alpha, per-CTA partial ||r||^2 and (MSDO-CG) beta partials
// V_k^T r: the FP64 k_final with its two triangular transforms on the tensor
// cores (Algorithm 1, the A-orthonormalised block and the x/r updates).
// Per 128-row tile: A_X and A_Y = the 8 digit slabs of the X and Y rows
// (row scales), B = the digits of R^{-1} by column scale, stacked by digit;
// slab p accumulates into groups p .. 7 (8 groups: pairs p + r <= 7; the
// dropped ones weigh below 2^-57 of row scale x column scale).  X's groups
// take TMEM columns [0, 128), Y's [128, 256).  Each group sum is at most
// 8 * 16 * 255^2 < 2^23.  The dot products with alpha, the residual norm and
// beta stay FP64, one FMA per entry as in k_final.
template <int W>
struct FinTc {
  static constexpr int R = 128;      // rows per tile
  static constexpr int ND = 8;       // digits
  static constexpr int NG = 8;       // groups kept
  static constexpr int KA = ND * W;  // A tile K (digit, column)
  static constexpr int NB = NG * W;  // B rows (digit r = 0..7, column b)
  static constexpr uint32_t TCOLS = 256;
  static constexpr size_t A_BYTES = (size_t)R * KA * 2;  // one of A_X, A_Y
  static constexpr size_t B_BYTES = (size_t)NB * W * 2;
  static constexpr size_t S_BYTES = (size_t)2 * R * W * 8;  // the next tile's X and Y rows (FP64)
  static constexpr size_t SMEM = 2 * A_BYTES + B_BYTES + S_BYTES + 4 * (W + 2 * R) + 8 * (2 * W);
};

template <int W>
constexpr size_t smem_final_tc() {
  return FinTc<W>::SMEM;
}

template <typename T, int W>
__host__ __device__ constexpr bool final_tc_ok() {
  return sizeof(T) == 8 && W == 16;
}

template <int W>
__global__ void __launch_bounds__(256, 2) k_final_tc(KP P, int gw, const double* Xin, const double* Yin,
                                                     double* Wout, double* Vout, double* xio, double* rio) {
  static_assert(W == 16, "one 16-column row per slicing thread");
  using U = FinTc<W>;
  constexpr int R = U::R, KA = U::KA, NB = U::NB;
  const DevState* st = P.st;
  if (skip(st, gw)) return;
  if (Wout == nullptr) {  // the solver's window slot
    const long long sl = st->next_slot;
    Wout = (double*)P.slotW + sl * P.slot_stride;
    Vout = (double*)P.slotV + sl * P.slot_stride;
  }
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __half* sAX = (__half*)smem_raw;                                 // R x KA
  __half* sAY = (__half*)(smem_raw + U::A_BYTES);                  // R x KA
  __half* sB = (__half*)(smem_raw + 2 * U::A_BYTES);               // NB x W
  double* sXs = (double*)(smem_raw + 2 * U::A_BYTES + U::B_BYTES);  // R x W staged X rows, then R x W Y rows
  int* sSc = (int*)(smem_raw + 2 * U::A_BYTES + U::B_BYTES + U::S_BYTES);  // W column scales of R^{-1}
  int* sSr = sSc + W;                                               // 2 R row scales (X rows, Y rows)
  double* sal = (double*)(sSr + 2 * R);                             // W: alpha
  double* sbeta = sal + W;                                          // W: beta partial sums
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  __shared__ double sred[8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double* Ri = P.small + kSmallRi;
  if (tid < W) {
    int sc = 0;
    for (int a = 0; a < W; a++) sc = max(sc, bexp(Ri[a * W + tid]));
    sSc[tid] = sc;
    sal[tid] = P.block ? 0.0 : P.small[kSmallAl + tid];  // block-residual mode updates x, r elsewhere
    sbeta[tid] = 0.0;
  }
  __syncthreads();
  for (int e = tid; e < NB * (W / 2); e += blockDim.x) {
    const int n = e / (W / 2), a = 2 * (e % (W / 2));
    const int r = n / W, b = n % W;
    const double c0 = Ri[a * W + b], c1 = Ri[(a + 1) * W + b];
    __half2 sg, of;
    sign_pair(c0, c1, sg, of);
    *reinterpret_cast<uint32_t*>(&sB[kmaj(n, a, W)]) =
        digit_pair(fixed64(c0, sSc[b]), fixed64(c1, sSc[b]), r, sg, of);
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tbase, U::TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  bool cnan = false;
  for (int b = 0; b < W; b++) cnan = cnan || (sSc[b] == 2047);

  int r0, r1;
  cta_rows_aligned(P.n, R, r0, r1);
  const int ntiles = (r1 - r0 + R - 1) / R;
  // slicing: thread (row = tid / 2, which = tid % 2) takes the X (0) or Y (1) row
  const int srow = tid >> 1, which = tid & 1;
  // X and Y rows arrive by 16-byte cp.async one tile ahead when both blocks
  // are 16-byte aligned (their rows are 128 bytes)
  const bool use_stage = ((((uintptr_t)Xin) | ((uintptr_t)Yin)) & 15) == 0;
  auto stage_tile = [&](int i) {
    const int rb = r0 + i * R, nrr = min(R, r1 - rb);
    for (int ch = tid; ch < 2 * R * (W / 2); ch += blockDim.x) {
      const int y = ch / (R * (W / 2)), e = ch % (R * (W / 2));
      const int rr = e / (W / 2), c2 = 2 * (e % (W / 2));
      // chunk c2 / 2 of a row lands at chunk (c2 / 2) ^ (rr % 8) (bank groups)
      if (rr < nrr)
        cp_async16(&sXs[(y * R + rr) * W + 2 * ((c2 >> 1) ^ (rr & 7))], (y ? Yin : Xin) + (long long)(rb + rr) * W + c2);
    }
    cp_async16_commit();
  };
  if (use_stage && ntiles > 0) stage_tile(0);
  // epilogue: warp w reads rows 32 (w % 4) + lane of X's (w < 4) or Y's groups
  const int erow = 32 * (warp & 3) + lane, ey = warp >> 2;
  double rho_acc = 0.0;
  double bacc[W];
#pragma unroll
  for (int b = 0; b < W; b++) bacc[b] = 0.0;
  bool ok = true;
  int it = 0;
  for (; it < ntiles && ok; it++) {
    const int row0 = r0 + it * R;
    const int nr = min(R, r1 - row0);
    if (use_stage) {
      cp_async16_wait();
      __syncthreads();  // tile it is in sXs
    }
    {
      const double* src = which ? Yin : Xin;
      __half* sA = which ? sAY : sAX;
      double q[W];
      int smax = 0;
#pragma unroll
      for (int c = 0; c < W; c++) {
        if (use_stage) q[c] = (srow < nr) ? sXs[(which * R + srow) * W + 2 * ((c >> 1) ^ (srow & 7)) + (c & 1)] : 0.0;
        else q[c] = (srow < nr) ? src[(long long)(row0 + srow) * W + c] : 0.0;
        smax = max(smax, bexp(q[c]));
      }
      if (smax == 2047) {
#pragma unroll
        for (int c = 0; c < W; c++) q[c] = 0.0;
      }
      const int S = (smax == 2047) ? 0 : smax;
#pragma unroll
      for (int c = 0; c < W; c += 2) {
        const unsigned long long u0 = fixed64(q[c], S), u1 = fixed64(q[c + 1], S);
        __half2 sg, of;
        sign_pair(q[c], q[c + 1], sg, of);
#pragma unroll
        for (int p = 0; p < 8; p++)
          *reinterpret_cast<uint32_t*>(&sA[kmaj(srow, p * W + c, KA)]) = digit_pair64(u0, u1, p, sg, of);
      }
      sSr[which * R + srow] = smax;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (use_stage && it + 1 < ntiles) stage_tile(it + 1);  // every thread has read sXs
    if (tid == 0) {
      tc_fence_after();
      const uint32_t b0 = smem_u32(sB);
      const uint64_t bd = sdesc(b0, 128u, (uint32_t)(W / 8) * 128u);
      for (int y = 0; y < 2; y++) {
        const uint32_t a0 = smem_u32(y ? sAY : sAX);
        for (int p = 0; p < 8; p++) {
          const uint64_t ad = sdesc(a0 + (uint32_t)(p * W / 8) * 128u, 128u, (uint32_t)(KA / 8) * 128u);
          mma_f16(tmem + (uint32_t)(y * NB + p * W), ad, bd, idesc_f16(R, (8 - p) * W), p > 0 ? 1u : 0u);
        }
      }
      mma_commit(&bar);
    }
    const bool done = mbar_wait_bounded(&bar, (uint32_t)(it & 1));
    ok = __syncthreads_and(done);
    if (!ok) break;
    tc_fence_after();
    // epilogue: rows of W_k (ey = 0) or V_k (ey = 1)
    {
      // T_b = sum_g D_g 2^{8 (8 - g)}, accumulated group by group
      long long hia[W];
      unsigned long long loa[W];
#pragma unroll
      for (int b = 0; b < W; b++) {
        hia[b] = 0;
        loa[b] = 0;
      }
#pragma unroll
      for (int gi = 0; gi < 8; gi++) {
        uint32_t v0[8], v1[8];
        const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(ey * NB + gi * W);
        tmem_ld8(ta, v0);
        tmem_ld8(ta + 8u, v1);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; j++) {
          i128_add_shifted(hia[j], loa[j], (long long)f2i_exact(__uint_as_float(v0[j])), 8 * (8 - gi));
          i128_add_shifted(hia[8 + j], loa[8 + j], (long long)f2i_exact(__uint_as_float(v1[j])), 8 * (8 - gi));
        }
      }
      const int Si = sSr[ey * R + erow];
      double dsum = 0.0;
      double vk[W];
#pragma unroll
      for (int b = 0; b < W; b++) {
        const long long hi = hia[b];
        const unsigned long long lo = loa[b];
        double val;
        if (Si == 2047 || cnan) val = __longlong_as_double(0x7FF8000000000000ll);
        else val = i128_to_double(hi, lo, (Si - 1022) + (sSc[b] - 1022) - 80);
        vk[b] = val;
        dsum += val * sal[b];
      }
      if (erow < nr) {
        const long long i = row0 + erow;
        double* out = ey ? Vout : Wout;
#pragma unroll
        for (int b = 0; b < W; b++) out[i * W + b] = vk[b];
        if (ey == 0) {
          xio[i] += dsum;
        } else {
          const double rn = rio[i] - dsum;
          rio[i] = rn;
          rho_acc += rn * rn;
          if (P.want_beta) {
#pragma unroll
            for (int b = 0; b < W; b++) bacc[b] = fma(vk[b], rn, bacc[b]);
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  if (!ok && tid == 0) {
    ((DevState*)st)->fault = 1;
    ((DevState*)st)->status = ST_ECUDA;
    ((DevState*)st)->stop = 1;
    mbar_wait_bounded(&bar, (uint32_t)(it & 1));
  }
  cp_async16_wait();  // no copy may still be landing when the CTA exits
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, U::TCOLS);
  if (!ok) return;
  // fixed-order CTA sums: warp shuffles, then the warps in order
  double v = rho_acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sred[warp] = v;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int w = 0; w < 8; w++) tot += sred[w];
    P.rho_part[blockIdx.x] = tot;
  }
  if (P.want_beta) {
#pragma unroll
    for (int b = 0; b < W; b++) {
      double bv = bacc[b];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bv += __shfl_xor_sync(0xffffffffu, bv, o);
      __syncthreads();
      if (lane == 0) sred[warp] = bv;
      __syncthreads();
      if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; w++) tot += sred[w];
        P.beta_part[(long long)blockIdx.x * 64 + b] = tot;
      }
    }
  }
}

}  // namespace tc
}  // namespace ecg
