// nn.cu -- sm_103a kernels of the warm-start network (include/ecg_nn.h):
// direct K x K convolutions on bf16 NHWC activations with FP32
// accumulation, their input and weight gradients, pooling, upsampling, the
// loss and the Adam step.  The network and its training loop live in
// paper_2305_19013_gb300/warmstart.py; this file holds every arithmetic
// step they run.
//
// The convolution kernels tile a CTA over 16 x 16 pixels of one image and
// 16 channels, stage the input halo and a weight slice in shared memory in
// FP32, and give every thread one pixel and 16 accumulators.  Reductions
// (weight and bias gradients, the loss) go through per-CTA partials summed
// in a fixed order, so training is reproducible run to run.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "ecg.h"
#include "ecg_nn.h"

namespace ecgnn {

typedef __nv_bfloat16 bf16;

constexpr int kTS = 16;   // pixel tile side
constexpr int kCT = 16;   // channels per CTA (outputs in forward / dgrad)
constexpr int kCC = 8;    // channels per staged chunk (reduction dimension)
constexpr int kWG = 64;   // CTAs over pixels in the weight gradient

__device__ __forceinline__ float bf(const bf16 v) { return __bfloat162float(v); }

// Forward: out = act(conv_K(concat(A, B)) + bias).
template <int K, bool OUT32>
__global__ void __launch_bounds__(256) k_conv(const bf16* A, int Ca, const bf16* B, int Cb, const bf16* w,
                                              const float* bias, void* out, int H, int W, int Cout, int relu) {
  constexpr int R = K / 2, HT = kTS + K - 1;
  __shared__ float sIn[kCC * HT * HT];           // [c][hy][hx]
  __shared__ __align__(16) float sW[K * K * kCC * kCT];  // [tap][c][co]
  const int tiles_x = (W + kTS - 1) / kTS;
  const int tx0 = (blockIdx.x % tiles_x) * kTS, ty0 = (blockIdx.x / tiles_x) * kTS;
  const int co0 = blockIdx.y * kCT, n = blockIdx.z;
  const int Cin = Ca + Cb;
  const int px = threadIdx.x % kTS, py = threadIdx.x / kTS;
  float acc[kCT];
#pragma unroll
  for (int co = 0; co < kCT; co++) acc[co] = 0.f;
  for (int ci0 = 0; ci0 < Cin; ci0 += kCC) {
    for (int e = threadIdx.x; e < kCC * HT * HT; e += blockDim.x) {
      const int c = e / (HT * HT), q = e - c * HT * HT, hy = q / HT, hx = q - hy * HT;
      const int y = ty0 + hy - R, x = tx0 + hx - R, ci = ci0 + c;
      float v = 0.f;
      if (y >= 0 && y < H && x >= 0 && x < W && ci < Cin) {
        const long long pix = ((long long)n * H + y) * W + x;
        v = (ci < Ca) ? bf(A[pix * Ca + ci]) : bf(B[pix * Cb + (ci - Ca)]);
      }
      sIn[e] = v;
    }
    for (int e = threadIdx.x; e < K * K * kCC * kCT; e += blockDim.x) {
      const int co = e % kCT, q = e / kCT, c = q % kCC, tap = q / kCC;
      const int ci = ci0 + c, cg = co0 + co;
      sW[e] = (ci < Cin && cg < Cout) ? bf(w[((long long)tap * Cin + ci) * Cout + cg]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int tap = 0; tap < K * K; tap++) {
      const int ky = tap / K, kx = tap - ky * K;
#pragma unroll
      for (int c = 0; c < kCC; c++) {
        const float v = sIn[(c * HT + py + ky) * HT + px + kx];
        const float4* wp = reinterpret_cast<const float4*>(&sW[(tap * kCC + c) * kCT]);
#pragma unroll
        for (int q = 0; q < kCT / 4; q++) {
          const float4 w4 = wp[q];
          acc[4 * q] = fmaf(v, w4.x, acc[4 * q]);
          acc[4 * q + 1] = fmaf(v, w4.y, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(v, w4.z, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(v, w4.w, acc[4 * q + 3]);
        }
      }
    }
    __syncthreads();
  }
  const int y = ty0 + py, x = tx0 + px;
  if (y >= H || x >= W) return;
  const long long pix = ((long long)n * H + y) * W + x;
#pragma unroll
  for (int co = 0; co < kCT; co++) {
    const int cg = co0 + co;
    if (cg < Cout) {
      float v = acc[co] + (bias ? bias[cg] : 0.f);
      if (relu) v = fmaxf(v, 0.f);
      if (OUT32) ((float*)out)[pix * Cout + cg] = v;
      else ((bf16*)out)[pix * Cout + cg] = __float2bfloat16_rn(v);
    }
  }
}

// Input gradient: din[p][ci] = sum over taps and co of
// dout[p + R - ky, q + R - kx][co] * w[ky][kx][ci][co].
template <int K>
__global__ void __launch_bounds__(256) k_conv_dgrad(const float* dout, const bf16* w, float* dA, int Ca, float* dB,
                                                    int Cb, int H, int W, int Cout, int accumulate) {
  constexpr int R = K / 2, HT = kTS + K - 1;
  __shared__ float sD[kCC * HT * HT];                    // [c(co)][hy][hx]
  __shared__ __align__(16) float sW[K * K * kCC * kCT];  // [tap][c(co)][ci]
  const int tiles_x = (W + kTS - 1) / kTS;
  const int tx0 = (blockIdx.x % tiles_x) * kTS, ty0 = (blockIdx.x / tiles_x) * kTS;
  const int ci0 = blockIdx.y * kCT, n = blockIdx.z;
  const int Cin = Ca + Cb;
  const int px = threadIdx.x % kTS, py = threadIdx.x / kTS;
  float acc[kCT];
#pragma unroll
  for (int c = 0; c < kCT; c++) acc[c] = 0.f;
  for (int co0 = 0; co0 < Cout; co0 += kCC) {
    // halo rows y = ty0 - R + hy: the pixels that tap (ky, kx) of the output
    // tile reads are hy = py + 2R - ky, hx = px + 2R - kx
    for (int e = threadIdx.x; e < kCC * HT * HT; e += blockDim.x) {
      const int c = e / (HT * HT), q = e - c * HT * HT, hy = q / HT, hx = q - hy * HT;
      const int y = ty0 + hy - R, x = tx0 + hx - R, co = co0 + c;
      float v = 0.f;
      if (y >= 0 && y < H && x >= 0 && x < W && co < Cout) v = dout[(((long long)n * H + y) * W + x) * Cout + co];
      sD[e] = v;
    }
    for (int e = threadIdx.x; e < K * K * kCC * kCT; e += blockDim.x) {
      const int ci = e % kCT, q = e / kCT, c = q % kCC, tap = q / kCC;
      const int cig = ci0 + ci, co = co0 + c;
      sW[e] = (cig < Cin && co < Cout) ? bf(w[((long long)tap * Cin + cig) * Cout + co]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int tap = 0; tap < K * K; tap++) {
      const int ky = tap / K, kx = tap - ky * K;
#pragma unroll
      for (int c = 0; c < kCC; c++) {
        const float v = sD[(c * HT + py + 2 * R - ky) * HT + px + 2 * R - kx];
        const float4* wp = reinterpret_cast<const float4*>(&sW[(tap * kCC + c) * kCT]);
#pragma unroll
        for (int q = 0; q < kCT / 4; q++) {
          const float4 w4 = wp[q];
          acc[4 * q] = fmaf(v, w4.x, acc[4 * q]);
          acc[4 * q + 1] = fmaf(v, w4.y, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(v, w4.z, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(v, w4.w, acc[4 * q + 3]);
        }
      }
    }
    __syncthreads();
  }
  const int y = ty0 + py, x = tx0 + px;
  if (y >= H || x >= W) return;
  const long long pix = ((long long)n * H + y) * W + x;
#pragma unroll
  for (int c = 0; c < kCT; c++) {
    const int cig = ci0 + c;
    if (cig >= Cin) continue;
    float* dst = (cig < Ca) ? &dA[pix * Ca + cig] : &dB[pix * Cb + (cig - Ca)];
    *dst = accumulate ? *dst + acc[c] : acc[c];
  }
}

// Weight gradient partials: CTA g of kWG sums over the pixel tiles
// g, g + kWG, ... for a 16 x 16 block of (ci, co), every tap; one thread per
// (ci, co) pair.
template <int K>
__global__ void __launch_bounds__(256) k_conv_wgrad(const bf16* A, int Ca, const bf16* B, int Cb, const float* dout,
                                                    float* part, int N, int H, int W, int Cout) {
  constexpr int R = K / 2, HT = kTS + K - 1;
  __shared__ float sIn[HT * HT * kCT];   // [hy][hx][ci]
  __shared__ float sD[kTS * kTS * kCT];  // [py][px][co]
  const int Cin = Ca + Cb;
  const int ci0 = blockIdx.y * kCT, co0 = blockIdx.z * kCT;
  const int cl = threadIdx.x / kCT, ol = threadIdx.x % kCT;
  const int tiles_x = (W + kTS - 1) / kTS, tiles_y = (H + kTS - 1) / kTS;
  const int ntiles = N * tiles_x * tiles_y;
  float acc[K * K];
#pragma unroll
  for (int t = 0; t < K * K; t++) acc[t] = 0.f;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int n = tile / (tiles_x * tiles_y), tq = tile - n * tiles_x * tiles_y;
    const int tx0 = (tq % tiles_x) * kTS, ty0 = (tq / tiles_x) * kTS;
    for (int e = threadIdx.x; e < HT * HT * kCT; e += blockDim.x) {
      const int c = e % kCT, q = e / kCT, hx = q % HT, hy = q / HT;
      const int y = ty0 + hy - R, x = tx0 + hx - R, ci = ci0 + c;
      float v = 0.f;
      if (y >= 0 && y < H && x >= 0 && x < W && ci < Cin) {
        const long long pix = ((long long)n * H + y) * W + x;
        v = (ci < Ca) ? bf(A[pix * Ca + ci]) : bf(B[pix * Cb + (ci - Ca)]);
      }
      sIn[e] = v;
    }
    for (int e = threadIdx.x; e < kTS * kTS * kCT; e += blockDim.x) {
      const int c = e % kCT, q = e / kCT, px = q % kTS, py = q / kTS;
      const int y = ty0 + py, x = tx0 + px, co = co0 + c;
      sD[e] = (y < H && x < W && co < Cout) ? dout[(((long long)n * H + y) * W + x) * Cout + co] : 0.f;
    }
    __syncthreads();
    for (int py = 0; py < kTS; py++)
      for (int px = 0; px < kTS; px++) {
        const float d = sD[(py * kTS + px) * kCT + ol];
#pragma unroll
        for (int tap = 0; tap < K * K; tap++) {
          const int ky = tap / K, kx = tap - ky * K;
          acc[tap] = fmaf(sIn[((py + ky) * HT + px + kx) * kCT + cl], d, acc[tap]);
        }
      }
    __syncthreads();
  }
  const int ci = ci0 + cl, co = co0 + ol;
  if (ci < Cin && co < Cout)
#pragma unroll
    for (int tap = 0; tap < K * K; tap++)
      part[((long long)blockIdx.x * K * K * Cin + (long long)tap * Cin + ci) * Cout + co] = acc[tap];
}

// Bias gradient partials: CTA g sums dout[.][co] over pixels g, g + G, ...
__global__ void __launch_bounds__(256) k_bias_grad(const float* dout, float* part, long long npix, int Cout) {
  __shared__ float s[256];
  for (int co = 0; co < Cout; co++) {
    float a = 0.f;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (long long)gridDim.x * blockDim.x)
      a += dout[p * Cout + co];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)blockIdx.x * Cout + co] = s[0];
    __syncthreads();
  }
}

// out[e] = sum over g < G of part[g * count + e].
__global__ void k_sum_parts(const float* part, float* out, long long count, int G) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int g = 0; g < G; g++) s += part[(long long)g * count + e];
    out[e] = s;
  }
}

__global__ void k_relu_bwd(const bf16* out, float* dout, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    if (!(bf(out[i]) > 0.f)) dout[i] = 0.f;
}

__global__ void k_pool2(const bf16* in, bf16* out, int N, int H, int W, int C) {
  const int Ho = H / 2, Wo = W / 2;
  const long long total = (long long)N * Ho * Wo * C;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    long long q = e / C;
    const int x = (int)(q % Wo);
    q /= Wo;
    const int y = (int)(q % Ho);
    const int n = (int)(q / Ho);
    const long long p = ((long long)n * H + 2 * y) * W + 2 * x;
    const float s = bf(in[p * C + c]) + bf(in[(p + 1) * C + c]) + bf(in[(p + W) * C + c]) +
                    bf(in[(p + W + 1) * C + c]);
    out[e] = __float2bfloat16_rn(0.25f * s);
  }
}

__global__ void k_pool2_bwd(const float* dout, float* din, int N, int H, int W, int C) {
  const long long total = (long long)N * H * W * C;
  const int Wo = W / 2, Ho = H / 2;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    long long q = e / C;
    const int x = (int)(q % W);
    q /= W;
    const int y = (int)(q % H);
    const int n = (int)(q / H);
    din[e] += 0.25f * dout[(((long long)n * Ho + y / 2) * Wo + x / 2) * C + c];
  }
}

__global__ void k_up2(const bf16* in, bf16* out, int N, int H, int W, int C) {
  const long long total = (long long)N * (2 * H) * (2 * W) * C;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    long long q = e / C;
    const int x = (int)(q % (2 * W));
    q /= (2 * W);
    const int y = (int)(q % (2 * H));
    const int n = (int)(q / (2 * H));
    out[e] = in[(((long long)n * H + y / 2) * W + x / 2) * C + c];
  }
}

__global__ void k_up2_bwd(const float* dout, float* din, int N, int H, int W, int C) {
  const long long total = (long long)N * H * W * C;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    long long q = e / C;
    const int x = (int)(q % W);
    q /= W;
    const int y = (int)(q % H);
    const int n = (int)(q / H);
    const long long p = ((long long)n * (2 * H) + 2 * y) * (2 * W) + 2 * x;
    din[e] = dout[p * C + c] + dout[(p + 1) * C + c] + dout[(p + 2 * W) * C + c] + dout[(p + 2 * W + 1) * C + c];
  }
}

// MSE partials: CTA g sums (pred - target)^2 over e = g*256 + tid, strided.
__global__ void __launch_bounds__(256) k_mse(const float* pred, const float* target, float* dpred, double* part,
                                             long long count) {
  __shared__ double s[256];
  double a = 0.0;
  const float inv = 2.0f / (float)count;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const float d = pred[e] - target[e];
    dpred[e] = inv * d;
    a += (double)d * (double)d;
  }
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_mse_final(const double* part, int G, double* loss, long long count) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int g = 0; g < G; g++) s += part[g];
    *loss = s / (double)count;
  }
}

__global__ void k_adam(float* w32, bf16* w16, const float* g, float* m, float* v, long long count, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w32[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w32[i] = wi;
    if (w16) w16[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void k_to_bf16(const float* in, bf16* out, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

__global__ void k_pack(const double* logk, const double* b, double mu, double s, double sb, bf16* out, int npix) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x) {
    out[2 * i] = __float2bfloat16_rn((float)((logk[i] - mu) / s));
    out[2 * i + 1] = __float2bfloat16_rn((float)(b[i] / sb));
  }
}

__global__ void k_unpack(const float* pred, const int32_t* perm, double scale, double* x0, int n) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    x0[r] = scale * (double)pred[perm ? perm[r] : r];
}

// Energy-norm loss of a 2D diffusion problem on an N x side x side batch:
// e = pred - target, (A e)_c = sum over the four faces of f (e_c - e_nb),
// f the harmonic mean of the two cells' coefficients (the cell's own
// coefficient and e_nb = 0 on the Dirichlet boundary), the stencil of
// workloads.diffusion2d; loss = sum_n w_n e_n^T A_n e_n, dpred = 2 w_n A_n e_n.
__global__ void __launch_bounds__(256) k_energy(const float* pred, const float* target, const float* kappa,
                                                const float* wn, float* dpred, double* part, int N, int side) {
  __shared__ double s[256];
  double a = 0.0;
  const long long npix = (long long)side * side, total = npix * N;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(e / npix);
    const int q = (int)(e - (long long)n * npix), y = q / side, x = q - y * side;
    const long long base = (long long)n * npix;
    const float kc = kappa[e];
    const float ec = pred[e] - target[e];
    float ae = 0.f;
    const int dy[4] = {0, 0, -1, 1}, dx[4] = {-1, 1, 0, 0};
#pragma unroll
    for (int f = 0; f < 4; f++) {
      const int yy = y + dy[f], xx = x + dx[f];
      if (yy < 0 || yy >= side || xx < 0 || xx >= side) {
        ae += kc * ec;
      } else {
        const long long nb = base + (long long)yy * side + xx;
        const float kn = kappa[nb];
        ae += (2.f * kc * kn / (kc + kn)) * (ec - (pred[nb] - target[nb]));
      }
    }
    dpred[e] = 2.f * wn[n] * ae;
    a += (double)wn[n] * (double)ec * (double)ae;
  }
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_sum_double(const double* part, int G, double* out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int g = 0; g < G; g++) s += part[g];
    *out = s;
  }
}

int grid_for(long long count) {
  long long g = (count + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

int status() {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ECG_OK : ECG_ECUDA;
}

bool dims_ok(int N, int H, int W, int C) { return N >= 1 && H >= 1 && W >= 1 && C >= 1 && C <= 128; }

}  // namespace ecgnn

using namespace ecgnn;

extern "C" {

int ecg_nn_conv(const uint16_t* A, int Ca, const uint16_t* B, int Cb, const uint16_t* w, const float* bias,
                void* out, int out_fp32, int N, int H, int W, int Cout, int K, int relu, void* stream) {
  if (!A || !w || !out || Ca < 1 || Cb < 0 || (Cb > 0 && !B) || !dims_ok(N, H, W, Ca + Cb) ||
      !dims_ok(N, H, W, Cout) || (K != 1 && K != 3))
    return ECG_EINVAL;
  const dim3 grid(((W + kTS - 1) / kTS) * ((H + kTS - 1) / kTS), (Cout + kCT - 1) / kCT, N);
  cudaStream_t s = (cudaStream_t)stream;
  const bf16* a = (const bf16*)A;
  const bf16* b = (const bf16*)B;
  const bf16* ww = (const bf16*)w;
  if (K == 3) {
    if (out_fp32) k_conv<3, true><<<grid, 256, 0, s>>>(a, Ca, b, Cb, ww, bias, out, H, W, Cout, relu);
    else k_conv<3, false><<<grid, 256, 0, s>>>(a, Ca, b, Cb, ww, bias, out, H, W, Cout, relu);
  } else {
    if (out_fp32) k_conv<1, true><<<grid, 256, 0, s>>>(a, Ca, b, Cb, ww, bias, out, H, W, Cout, relu);
    else k_conv<1, false><<<grid, 256, 0, s>>>(a, Ca, b, Cb, ww, bias, out, H, W, Cout, relu);
  }
  return status();
}

int ecg_nn_conv_dgrad(const float* dout, const uint16_t* w, float* dA, int Ca, float* dB, int Cb, int N, int H,
                      int W, int Cout, int K, int accumulate, void* stream) {
  if (!dout || !w || !dA || Ca < 1 || Cb < 0 || (Cb > 0 && !dB) || !dims_ok(N, H, W, Ca + Cb) ||
      !dims_ok(N, H, W, Cout) || (K != 1 && K != 3))
    return ECG_EINVAL;
  const dim3 grid(((W + kTS - 1) / kTS) * ((H + kTS - 1) / kTS), (Ca + Cb + kCT - 1) / kCT, N);
  cudaStream_t s = (cudaStream_t)stream;
  if (K == 3) k_conv_dgrad<3><<<grid, 256, 0, s>>>(dout, (const bf16*)w, dA, Ca, dB, Cb, H, W, Cout, accumulate);
  else k_conv_dgrad<1><<<grid, 256, 0, s>>>(dout, (const bf16*)w, dA, Ca, dB, Cb, H, W, Cout, accumulate);
  return status();
}

size_t ecg_nn_wgrad_scratch(int Cin, int Cout, int K) {
  const size_t w = (size_t)kWG * K * K * Cin * Cout;
  const size_t b = (size_t)kWG * Cout;
  return w > b ? w : b;
}

int ecg_nn_conv_wgrad(const uint16_t* A, int Ca, const uint16_t* B, int Cb, const float* dout, float* dw,
                      float* dbias, float* scratch, int N, int H, int W, int Cout, int K, void* stream) {
  if (!A || !dout || !dw || !scratch || Ca < 1 || Cb < 0 || (Cb > 0 && !B) || !dims_ok(N, H, W, Ca + Cb) ||
      !dims_ok(N, H, W, Cout) || (K != 1 && K != 3))
    return ECG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int Cin = Ca + Cb;
  const dim3 grid(kWG, (Cin + kCT - 1) / kCT, (Cout + kCT - 1) / kCT);
  const bf16* a = (const bf16*)A;
  const bf16* b = (const bf16*)B;
  if (K == 3) k_conv_wgrad<3><<<grid, 256, 0, s>>>(a, Ca, b, Cb, dout, scratch, N, H, W, Cout);
  else k_conv_wgrad<1><<<grid, 256, 0, s>>>(a, Ca, b, Cb, dout, scratch, N, H, W, Cout);
  const long long nw = (long long)K * K * Cin * Cout;
  k_sum_parts<<<grid_for(nw), 256, 0, s>>>(scratch, dw, nw, kWG);
  if (dbias) {
    k_bias_grad<<<kWG, 256, 0, s>>>(dout, scratch, (long long)N * H * W, Cout);
    k_sum_parts<<<grid_for(Cout), 256, 0, s>>>(scratch, dbias, Cout, kWG);
  }
  return status();
}

int ecg_nn_relu_bwd(const uint16_t* out, float* dout, int64_t count, void* stream) {
  if (!out || !dout || count < 0) return ECG_EINVAL;
  k_relu_bwd<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>((const bf16*)out, dout, count);
  return status();
}

int ecg_nn_pool2(const uint16_t* in, uint16_t* out, int N, int H, int W, int C, void* stream) {
  if (!in || !out || !dims_ok(N, H, W, C) || (H & 1) || (W & 1)) return ECG_EINVAL;
  k_pool2<<<grid_for((long long)N * H * W * C / 4), 256, 0, (cudaStream_t)stream>>>((const bf16*)in, (bf16*)out, N, H,
                                                                                   W, C);
  return status();
}

int ecg_nn_pool2_bwd(const float* dout, float* din, int N, int H, int W, int C, void* stream) {
  if (!dout || !din || !dims_ok(N, H, W, C) || (H & 1) || (W & 1)) return ECG_EINVAL;
  k_pool2_bwd<<<grid_for((long long)N * H * W * C), 256, 0, (cudaStream_t)stream>>>(dout, din, N, H, W, C);
  return status();
}

int ecg_nn_up2(const uint16_t* in, uint16_t* out, int N, int H, int W, int C, void* stream) {
  if (!in || !out || !dims_ok(N, H, W, C)) return ECG_EINVAL;
  k_up2<<<grid_for((long long)N * 4 * H * W * C), 256, 0, (cudaStream_t)stream>>>((const bf16*)in, (bf16*)out, N, H,
                                                                                 W, C);
  return status();
}

int ecg_nn_up2_bwd(const float* dout, float* din, int N, int H, int W, int C, void* stream) {
  if (!dout || !din || !dims_ok(N, H, W, C)) return ECG_EINVAL;
  k_up2_bwd<<<grid_for((long long)N * H * W * C), 256, 0, (cudaStream_t)stream>>>(dout, din, N, H, W, C);
  return status();
}

int ecg_nn_mse(const float* pred, const float* target, float* dpred, double* loss, int64_t count, void* stream) {
  if (!pred || !target || !dpred || !loss || count < 1) return ECG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // loss[1 .. 256] hold the per-CTA partial sums (see ecg_nn.h)
  const int G = 256;
  k_mse<<<G, 256, 0, s>>>(pred, target, dpred, loss + 1, count);
  k_mse_final<<<1, 32, 0, s>>>(loss + 1, G, loss, count);
  return status();
}

int ecg_nn_energy_loss(const float* pred, const float* target, const float* kappa, const float* weights,
                       float* dpred, double* loss, int N, int side, void* stream) {
  if (!pred || !target || !kappa || !weights || !dpred || !loss || N < 1 || side < 1) return ECG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int G = 256;
  k_energy<<<G, 256, 0, s>>>(pred, target, kappa, weights, dpred, loss + 1, N, side);
  k_sum_double<<<1, 32, 0, s>>>(loss + 1, G, loss);
  return status();
}

int ecg_nn_adam(float* w32, uint16_t* w16, const float* g, float* m, float* v, int64_t count, float lr, float beta1,
                float beta2, float eps, int step, void* stream) {
  if (!w32 || !g || !m || !v || count < 0 || step < 1) return ECG_EINVAL;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>(w32, (bf16*)w16, g, m, v, count, lr, beta1, beta2, eps,
                                                             c1, c2);
  return status();
}

int ecg_nn_to_bf16(const float* in, uint16_t* out, int64_t count, void* stream) {
  if (!in || !out || count < 0) return ECG_EINVAL;
  k_to_bf16<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>(in, (bf16*)out, count);
  return status();
}

int ecg_nn_pack(const double* logk, const double* b, double mu, double s, double sb, uint16_t* out, int side,
                void* stream) {
  if (!logk || !b || !out || side < 1 || !(s > 0.0) || !(sb > 0.0)) return ECG_EINVAL;
  const int npix = side * side;
  k_pack<<<grid_for(npix), 256, 0, (cudaStream_t)stream>>>(logk, b, mu, s, sb, (bf16*)out, npix);
  return status();
}

int ecg_nn_unpack(const float* pred, const int32_t* perm, double scale, double* x0, int n, void* stream) {
  if (!pred || !x0 || n < 1) return ECG_EINVAL;
  k_unpack<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(pred, perm, scale, x0, n);
  return status();
}

}  // extern "C"
