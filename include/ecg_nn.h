/*
 * ecg_nn.h -- C ABI of the small convolutional network that proposes the
 * initial iterate x_0 of an enlarged CG solve from (coefficient field,
 * right-hand side) on a 2D grid.
 *
 * The paper has no counterpart: its solves start from x_0 = 0 (Section 5).
 * The network is an addition beside the method; ecg_solve with
 * ECG_STOP_B (stop when ||r_k|| <= tol ||b||) measures its proposals, and the
 * plain x_0 = 0 solve is always available as the fallback.
 *
 * Conventions.  Activations are NHWC (image, row, column, channel), bf16
 * (__nv_bfloat16 bit patterns, passed as uint16_t), weights of a K x K
 * convolution are [K][K][Cin][Cout] bf16 with an FP32 master copy, biases
 * and every gradient are FP32, and all products accumulate in FP32.  All
 * pointers are device pointers; `stream` is a cudaStream_t (NULL: the
 * default stream).  Calls are asynchronous on the stream.  Every function
 * returns 0 or ECG_EINVAL / ECG_ECUDA (ecg.h).  Sizes: 1 <= N, 1 <= H, W;
 * channels 1..128; K in {1, 3} (zero padding K/2, stride 1).
 */
#ifndef ECG_NN_H
#define ECG_NN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* out = act(conv_K(concat(A, B)) + bias): A has Ca channels, B (may be
 * NULL, Cb = 0) Cb channels, concatenated in that order.  bias may be NULL.
 * relu: 1 applies max(0, .).  out is bf16 (out_fp32 = 0) or FP32
 * (out_fp32 = 1), N x H x W x Cout. */
int ecg_nn_conv(const uint16_t* A, int Ca, const uint16_t* B, int Cb, const uint16_t* w, const float* bias,
                void* out, int out_fp32, int N, int H, int W, int Cout, int K, int relu, void* stream);

/* Input gradients of that convolution: d(concat(A, B)) = conv_K^T(dout)
 * with the same weights; dA (Ca channels) and dB (Cb channels, may be NULL)
 * are FP32 and are overwritten (accumulate = 0) or added to
 * (accumulate = 1).  dout is FP32, already multiplied by the activation's
 * derivative. */
int ecg_nn_conv_dgrad(const float* dout, const uint16_t* w, float* dA, int Ca, float* dB, int Cb, int N, int H,
                      int W, int Cout, int K, int accumulate, void* stream);

/* Weight and bias gradients: dw[ky][kx][ci][co] = sum over images and
 * pixels of concat(A, B)[p + offset] * dout[p][co], dbias[co] = sum of
 * dout[.][co] (dbias may be NULL).  Both overwritten, summed in a fixed
 * order.  scratch: FP32 device memory of ecg_nn_wgrad_scratch(...)
 * elements. */
size_t ecg_nn_wgrad_scratch(int Cin, int Cout, int K);
int ecg_nn_conv_wgrad(const uint16_t* A, int Ca, const uint16_t* B, int Cb, const float* dout, float* dw,
                      float* dbias, float* scratch, int N, int H, int W, int Cout, int K, void* stream);

/* dout[i] = 0 where out[i] <= 0 (ReLU backward, in place on FP32 dout). */
int ecg_nn_relu_bwd(const uint16_t* out, float* dout, int64_t count, void* stream);

/* 2 x 2 average pooling (H, W even): out is N x H/2 x W/2 x C; backward
 * din += 0.25 * dout spread over each 2 x 2 window (din FP32, added to). */
int ecg_nn_pool2(const uint16_t* in, uint16_t* out, int N, int H, int W, int C, void* stream);
int ecg_nn_pool2_bwd(const float* dout, float* din, int N, int H, int W, int C, void* stream);

/* Nearest 2x upsampling: out is N x 2H x 2W x C; backward din = sum of the
 * four dout values of each input pixel (din FP32, overwritten). */
int ecg_nn_up2(const uint16_t* in, uint16_t* out, int N, int H, int W, int C, void* stream);
int ecg_nn_up2_bwd(const float* dout, float* din, int N, int H, int W, int C, void* stream);

/* Mean squared error over count values: loss[0] = sum (pred - target)^2 /
 * count, summed in a fixed order; loss is a device array of 257 doubles
 * (loss[1..256] hold partial sums).  dpred (FP32) = 2 (pred - target) /
 * count. */
int ecg_nn_mse(const float* pred, const float* target, float* dpred, double* loss, int64_t count,
               void* stream);

/* Energy-norm loss for the 2D diffusion problems of a batch (N images of
 * side x side cells, grid order): with e = pred - target and A_n the
 * 5-point operator of the cell coefficients kappa (harmonic means on
 * interior faces, the cell's own coefficient on the Dirichlet boundary),
 * loss[0] = sum_n weights[n] e_n^T A_n e_n and dpred = 2 weights[n] A_n e_n.
 * The energy norm is what CG reduces, so the loss weighs each error
 * component as the solve will have to; loss is a device array of 257
 * doubles (loss[1..256] hold partial sums). */
int ecg_nn_energy_loss(const float* pred, const float* target, const float* kappa, const float* weights,
                       float* dpred, double* loss, int N, int side, void* stream);

/* One Adam step on count parameters (w32 FP32 master, w16 its bf16 copy,
 * g gradient, m and v moments; step >= 1 for the bias correction). */
int ecg_nn_adam(float* w32, uint16_t* w16, const float* g, float* m, float* v, int64_t count, float lr, float beta1,
                float beta2, float eps, int step, void* stream);

/* Round FP32 values to bf16 (count values). */
int ecg_nn_to_bf16(const float* in, uint16_t* out, int64_t count, void* stream);

/* Network input of one grid problem: out (1 x side x side x 2 bf16) holds
 * ((log kappa - mu) / s, b / sb) in grid order (row index y * side + x). */
int ecg_nn_pack(const double* logk, const double* b, double mu, double s, double sb, uint16_t* out, int side,
                void* stream);

/* x0[r] = scale * pred[perm[r]] (FP64): the network's grid-ordered output
 * scaled back and permuted into the solver's row order (perm may be NULL:
 * identity). */
int ecg_nn_unpack(const float* pred, const int32_t* perm, double scale, double* x0, int n, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ECG_NN_H */
