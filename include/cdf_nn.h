/*
 * cdf_nn.h -- C ABI of the BF16 kernels of the convolutional surrogate that
 * predicts steady moment fields to warm-start cdf_lb_run_to_steady.
 *
 * The paper (Zhan, Chai & Shi, arXiv:2101.03055) has no learned component: the
 * network is a systems addition whose only role is a better initial state for
 * the paper's steady solves (Sec. 3.2 cavity); the lattice Boltzmann residual
 * still decides convergence.
 *
 * Conventions: activations are NHWC BF16 arrays [N][H][W][C] on the device,
 * C a multiple of 16; 3x3 weights are BF16 [Cout][3][3][Cin]; biases, head
 * weights, gradients of weights and optimiser state are FP32.  Every call
 * enqueues work on `stream` (cudaStream_t, NULL = legacy default) and returns
 * without synchronising; pointers are the caller's.  Calls return CDF_NN_OK,
 * CDF_NN_EINVAL for bad shapes (nothing is launched) or CDF_NN_ECUDA when the
 * launch failed; cdf_nn_last_error() has the message.
 */
#ifndef CDF_NN_H
#define CDF_NN_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { CDF_NN_OK = 0, CDF_NN_EINVAL = 1, CDF_NN_ECUDA = 2 } cdf_nn_status;

/* y[p][co] = act(sum_{ky,kx,ci} x[p + (ky-1, kx-1)][ci] w[co][ky][kx][ci] + bias[co]),
 * zero padding; act = ReLU if relu != 0.  Tensor cores, FP32 accumulation, BF16 out.
 * Cin % 16 == 0, Cout % 32 == 0; bias may be NULL. */
cdf_nn_status cdf_nn_conv3x3_fwd(const void *x, const void *w, const float *bias, void *y, int N, int H, int W,
                                 int Cin, int Cout, int relu, void *stream);
/* dx = gradient of the convolution above with respect to x (before any ReLU):
 * dx[p][ci] = sum_{t,co} dy[p + d(t)][co] w[co][8 - t][ci]. */
cdf_nn_status cdf_nn_conv3x3_bwd_data(const void *dy, const void *w, void *dx, int N, int H, int W, int Cin, int Cout,
                                      void *stream);
/* dw[co][t][ci] += sum_p dy[p][co] x[p + d(t)][ci] and db[co] += sum_p dy[p][co]
 * (FP32, accumulated: zero them first).  db may be NULL.  On the tensor-core path
 * the pixels are split over the GPU for dw and, separately, for db; each split's
 * partial sums go to `workspace` (device memory of at least
 * cdf_nn_conv3x3_bwd_weight_workspace() bytes, owned by the caller, contents
 * overwritten) and are added in a fixed order: the result is the same bits on
 * every run.  The warp-level MMA path adds its partial sums
 * atomically (order-dependent) and ignores the workspace. */
cdf_nn_status cdf_nn_conv3x3_bwd_weight(const void *x, const void *dy, float *dw, float *db, int N, int H, int W,
                                        int Cin, int Cout, void *workspace, long long workspace_bytes, void *stream);
/* Bytes of workspace cdf_nn_conv3x3_bwd_weight needs for this shape; -1 for a bad shape. */
long long cdf_nn_conv3x3_bwd_weight_workspace(int N, int H, int W, int Cin, int Cout);
/* d[i] = 0 where y[i] <= 0 (ReLU backward through the layer's output y), n elements. */
cdf_nn_status cdf_nn_relu_bwd(void *d, const void *y, long long n, void *stream);
/* 2x2 average pooling [N][H][W][C] -> [N][H/2][W/2][C] and its backward (H, W even). */
cdf_nn_status cdf_nn_avgpool2_fwd(const void *x, void *y, int N, int H, int W, int C, void *stream);
cdf_nn_status cdf_nn_avgpool2_bwd(const void *dy, void *dx, int N, int H, int W, int C, void *stream);
/* Nearest 2x upsampling of x [N][H][W][C] into channels [coff, coff + C) of
 * y [N][2H][2W][Cy]; backward sums the four covering values. */
cdf_nn_status cdf_nn_upsample2_fwd(const void *x, void *y, int N, int H, int W, int C, int Cy, int coff, void *stream);
cdf_nn_status cdf_nn_upsample2_bwd(const void *dy, void *dx, int N, int H, int W, int C, int Cy, int coff, void *stream);
/* y[p][dst_off + c] (+)= x[p][src_off + c], c < count, p < P (skip concatenation / split). */
cdf_nn_status cdf_nn_copy_channels(const void *x, void *y, long long P, int Cx, int Cy, int src_off, int dst_off,
                                   int count, int accumulate, void *stream);
/* 1x1 output head in FP32: out[p][o] = sum_c x[p][c] w[o][c] + b[o]; backward gives
 * dx (BF16) and accumulates dw, db (zero them first). */
cdf_nn_status cdf_nn_head_fwd(const void *x, const float *w, const float *b, float *out, long long P, int C, int O,
                              void *stream);
cdf_nn_status cdf_nn_head_bwd(const void *x, const float *w, const float *dout, void *dx, float *dw, float *db,
                              long long P, int C, int O, void *stream);
/* Mean squared error over n values: *loss += mean((pred - target)^2) (zero it first),
 * grad = 2 (pred - target) / n. */
cdf_nn_status cdf_nn_mse(const float *pred, const float *target, float *grad, float *loss, long long n, void *stream);
/* One Adam step (Kingma & Ba) on FP32 weights w with gradient g and moments m, v;
 * step >= 1 sets the bias corrections; w_bf16 (may be NULL) receives the BF16 copy. */
cdf_nn_status cdf_nn_adam(float *w, const float *g, float *m, float *v, void *w_bf16, long long n, float lr, float b1,
                          float b2, float eps, long long step, void *stream);
const char *cdf_nn_last_error(void);
/* Tensor-core path of the convolutions above.  1 (the default): the 5th-generation
 * tensor cores (tcgen05.mma, accumulators in tensor memory) with the faster operand
 * staging for the layer's depth -- for a forward pass whose image rows are whole
 * 128-pixel tiles with 16, 32 or 64 input channels, the kernel without im2col copy
 * (each tile's three input rows staged once; every tap's operand is the same rows
 * seen through a shifted descriptor; persistent CTAs); otherwise tiles copied by
 * cp.async through three stage buffers when the GEMM input has at least 128
 * channels, two buffers filled by ordinary loads below that (more CTAs per SM hide
 * more latency at short K); 4: the kernel without im2col copy where the shape
 * allows it, else as 1;
 * 2: tcgen05 with the two-buffer staging for every layer; 3: the forward pass on a
 * persistent warp-specialised tcgen05 kernel (producer warps, one MMA thread, epilogue
 * warps, two accumulators; slower than 1 at the surrogate's layer shapes, where one
 * CTA per SM leaves too few warps to hide latency), the backward pass as in 1;
 * 0: the warp-level MMA kernels.  The weight gradient runs on tcgen05 for 1 to 4.
 * Process-wide; all give the same results up to the order of the FP32 accumulation
 * (1 to 4 issue the same MMAs in the same order: the same bits). */
cdf_nn_status cdf_nn_set_tensor_path(int tcgen05);
/* *out = 1 if a bounded wait of a tcgen05 convolution ever ran out (its output is
 * then undefined), else 0.  Synchronises with the device. */
cdf_nn_status cdf_nn_error_flag(int *out);

#ifdef __cplusplus
}
#endif
#endif /* CDF_NN_H */
