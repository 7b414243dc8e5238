/*
 * evx_nn.h - C-ABI of the learned surrogate's GPU kernels (sm_103a).
 *
 * The paper motivates embedding the solver in learning pipelines: neural
 * surrogates trained on solver data, with gradients through the whole
 * pipeline (Statement of Need, on differentiable physics and neural surrogate
 * training; Summary, on machine learning integrated with simulation). It
 * gives no architecture. The surrogate here is a 3D residual CNN that maps
 * c_n to c_{n+s} (a block of s solver steps):
 *   lift conv 1 -> 32 (input padded to 16 channels), 4 residual blocks
 *   [conv 32 -> 32, GELU, conv 32 -> 32] + skip, projection conv 32 -> 1
 *   (output padded to 16 channels, channel 0 used), correction made zero-mean
 *   per sample in FP64 (the scheme conserves mass), c_{n+s} = c_n + correction.
 * All convolutions are 3x3x3 with periodic wrap, BF16 operands, FP32
 * accumulation on the tensor cores.
 *
 * Layouts: activations BF16 channels-last [B][X][Y][Z][C] (C = 16 or 32);
 * weights BF16 (master copies FP32) [27][Cout][Cin], tap t = 9 (dx+1) +
 * 3 (dy+1) + (dz+1); biases FP32 [Cout]; fields FP32 [B][X][Y][Z].
 * Sizes: Y even, Z a multiple of 64. All pointers are device pointers the
 * caller owns; calls are asynchronous on `stream` (a cudaStream_t, NULL =
 * legacy default stream) and return EVX_ERR_ARG / EVX_ERR_SIZE for invalid
 * arguments, EVX_ERR_CUDA if a launch fails (message: evx_nn_last_error).
 */
#ifndef EVX_NN_H
#define EVX_NN_H

#include <stddef.h>

#include "evx.h"

#ifdef __cplusplus
extern "C" {
#endif

/* conv epilogues: out(v, co) = acc(v, co) + bias(co), then */
enum {
    EVX_NN_EPI_PLAIN = 0,    /* out (BF16) = value */
    EVX_NN_EPI_GELU = 1,     /* pre (BF16) = value (not stored if pre is NULL, e.g. in inference);
                              * out (BF16) = GELU(value) (erf form) */
    EVX_NN_EPI_RESID = 2,    /* out (BF16) = res + value */
    EVX_NN_EPI_GELU_BWD = 3, /* out (BF16) = value * GELU'(pre) (pre read, not written) */
    EVX_NN_EPI_FIELD = 4,    /* out (FP32 field) = value of channel 0 */
    EVX_NN_EPI_RESID32 = 5   /* FP32 residual stream: pre (FP32 [..][cout]) += value, updated in
                              * place; out (BF16) = the new pre (the next convolution's input) */
};

/* Periodic 3x3x3 convolution in (BF16, cin channels) -> out, weights w
 * [27][cout][cin], bias (may be NULL), epilogue as above. cin, cout in
 * {16, 32}. With flipped weights (evx_nn_flip_weights) the same call computes
 * the data gradient of a convolution. */
evx_status evx_nn_conv3d(const void *in, const void *w, const float *bias, void *out, void *pre,
                         const void *res, int B, int X, int Y, int Z, int cin, int cout, int epilogue,
                         void *stream);

/* The network's lift and projection as direct sums (CUDA cores): a convolution
 * whose input (lift) or output (projection) is a single field would spend
 * 15/16 of a 16-channel tensor-core GEMM on zero padding.
 * evx_nn_lift: out(v, co) = bias(co) + sum_t w[t][co][0] BF16(scale f(v + off_t))
 *   for co < cout = 32; w is the [27][cout][cin] weight of the padded lift
 *   (only input channel 0 used); f FP32 field, out BF16 [..][32]. Equals
 *   evx_nn_field_to_act + evx_nn_conv3d(EPI_PLAIN) up to FP32 summation order.
 * evx_nn_project: out(v) = bias(0) + sum_t sum_ci w[t][0][ci] h(v + off_t, ci)
 *   with cin = 32; w [27][cout][32] (output channel 0 used); h BF16, out FP32
 *   field. Equals evx_nn_conv3d(EPI_FIELD) up to summation order.
 * Any B, X, Y, Z >= 1 (periodic). */
evx_status evx_nn_lift(const float *f, float scale, const void *w, int cin, int cout, const float *bias, void *out,
                       int B, int X, int Y, int Z, void *stream);
evx_status evx_nn_project(const void *h, const void *w, int cin, int cout, const float *bias, float *out, int B,
                          int X, int Y, int Z, void *stream);
/* The same two with an FP32 residual stream (EVX_NN_EPI_RESID32): evx_nn_lift32
 * writes the lift both as FP32 out32 [..][32] and as its BF16 copy out;
 * evx_nn_project32 reads the FP32 stream h32 [..][32]. The stream keeps FP32
 * precision between the blocks; only the convolutions' operands are BF16. */
evx_status evx_nn_lift32(const float *f, float scale, const void *w, int cin, int cout, const float *bias,
                         void *out, float *out32, int B, int X, int Y, int Z, void *stream);
evx_status evx_nn_project32(const float *h32, const void *w, int cin, int cout, const float *bias, float *out,
                            int B, int X, int Y, int Z, void *stream);

/* Weight gradient of out = conv(x, W): dw[t][co][ci] = sum_v dy(v, co) x(v + off_t, ci)
 * (FP32). partials: device scratch of partial_floats floats (at least
 * 27 * cin * cout; more allows more CTAs), reduced in a fixed order. */
evx_status evx_nn_conv3d_wgrad(const void *dy, const void *x, float *dw, float *partials,
                               size_t partial_floats, int B, int X, int Y, int Z, int cin, int cout,
                               void *stream);

/* Bias gradient db[co] = sum_v dy(v, co) (FP64 partials: nparts * c doubles; fixed
 * summation order). c = 16 or 32 with dy 16-byte aligned: one pass over dy; other
 * cases: one pass per channel. */
evx_status evx_nn_bias_grad(const void *dy, long long nvox, int c, double *partials, int nparts, float *db,
                            void *stream);

/* Data-gradient weights: wt[26 - t][ci][co] = w[t][co][ci] (BF16). */
evx_status evx_nn_flip_weights(const void *w, int cout, int cin, void *wt, void *stream);

/* FP32 field -> BF16 activation with c channels (channel 0 = scale * f, others 0). */
evx_status evx_nn_field_to_act(const float *f, long long nvox, int c, float scale, void *act, void *stream);

/* Per sample s: out = base + (d - mean_s(d)) (base may be NULL), mean in FP64;
 * partials: nsamples * nparts doubles. */
evx_status evx_nn_zero_mean_add(const float *base, const float *d, int nsamples, long long V, double *partials,
                                int nparts, float *out, void *stream);

/* As evx_nn_zero_mean_add with the correction scaled per sample:
 * out = base + scale[s] (d - mean_s(d)), scale a device array of nsamples doubles. */
evx_status evx_nn_zero_mean_add_scaled(const float *base, const float *d, const double *scale, int nsamples,
                                       long long V, double *partials, int nparts, float *out, void *stream);

/* Relative strength of the nonlinear remainder of c^3 - c about each sample's
 * mean (the part the block propagator of evx_ch_block freezes over a block):
 *   scale[s] = min(1, ||N||_2 / ||d||_2),  d = c - mean(c),  N = d^2 (3 mean(c) + d),
 * FP64, fixed summation order; 0 for a uniform sample. It is the learned
 * surrogate's output scale (the network's correction cannot exceed what the
 * nonlinearity can produce). nsamples <= 32 fields of V values, contiguous;
 * partials: 3 nsamples nparts doubles; scale: nsamples device doubles. */
evx_status evx_nn_nl_scale(const float *c, int nsamples, long long V, double *partials, int nparts, double *scale,
                           void *stream);

/* d_sum = sum |x| over n values in FP64 (device double), fixed summation order
 * (nparts partials, then one sum); the guard's L1 norm of a sample, against which
 * the mass drift of a surrogate block is measured. */
evx_status evx_nn_abs_sum(const float *x, long long n, double *partials, int nparts, double *d_sum, void *stream);

/* d_sum = sum (p - t)^2 in FP64 (device double); grad (may be NULL) = grad_scale (p - t). */
evx_status evx_nn_mse(const float *p, const float *t, long long n, float grad_scale, float *grad,
                      double *partials, int nparts, double *d_sum, void *stream);

/* Adam step (step >= 1) on FP32 master parameters; refreshes the BF16 copy wbf
 * if non-NULL. */
evx_status evx_nn_adam(float *w, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                       float eps, int step, void *wbf, void *stream);

/* BF16 copy of an FP32 array. */
evx_status evx_nn_f32_to_bf16(const float *a, int n, void *b, void *stream);

/* Convolution engines for the 32 -> 32 layers (Z a multiple of 64):
 * TCGEN05 (default) issues tcgen05.mma from shared-memory operands into a
 * tensor-memory accumulator; MMA_SYNC uses warp-level mma.sync fragments.
 * Other channel pairs always use MMA_SYNC. Process-wide setting. */
enum { EVX_NN_ENGINE_TCGEN05 = 0, EVX_NN_ENGINE_MMA_SYNC = 1 };
evx_status evx_nn_set_conv_engine(int engine);
int evx_nn_conv_engine(void);

/* Synchronizes the device and reports whether a tensor-core pipeline wait
 * ran past its bound since the last check (EVX_ERR_CUDA; the flag is then
 * cleared). Such a kernel returns early and leaves its outputs invalid. */
evx_status evx_nn_check(void);

/* Message of the last failed evx_nn_* call of this thread. */
const char *evx_nn_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* EVX_NN_H */
