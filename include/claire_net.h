/*
 * libclaire network kernels: the learned warm start of the registration.
 *
 * The paper (Sec. 2.2, Sec. 4) solves every registration from v = 0 or from
 * a coarser-grid solution.  This part adds a small 3D convolutional network
 * (a U-Net over periodic volumes) that maps an image pair (m0, m1) to an
 * initial velocity and, optionally, to a pointwise weight of the data term of
 * the two-level preconditioner's coarse operator; Gauss-Newton-Krylov from
 * that guess remains the solver and corrects whatever error the guess has.  The paper has no network: these entry points
 * are building blocks of that extension, with no counterpart in it.
 *
 * Conventions, for every entry point below:
 *   - All array pointers are DEVICE pointers owned by the caller; nothing is
 *     allocated, freed or retained.  Work is queued on `stream` (a
 *     cudaStream_t, NULL = legacy default stream) and returns without
 *     synchronising.
 *   - Activations are BF16, channels-last [B][D][H][W][C] (C contiguous).  A
 *     tensor may be a channel slice of a wider buffer: `*_stride` is the
 *     channel stride (elements between consecutive voxels), the pointer is
 *     the slice's first channel.  Strides and slice offsets must be
 *     multiples of 8 channels and pointers 16-byte aligned.
 *   - vol[4] = {B, D, H, W}: batch and grid of the tensor the operation
 *     produces (for pool2/up2 and their backward passes: of the COARSE grid).
 *     Boundaries are periodic (wrap-around), like the registration domain.
 *   - 3x3x3 conv weights are BF16 [Cout][27][Cin], tap = kd*9 + kh*3 + kw
 *     with offset (kd-1, kh-1, kw-1); biases FP32 [Cout].
 *   - Errors: CLAIRE_EINVAL for a shape, stride or alignment the kernels do
 *     not support (nothing is launched), CLAIRE_ECUDA for a failed launch;
 *     the message is available from claire_net_last_error() (per thread).
 */
#ifndef CLAIRE_NET_H
#define CLAIRE_NET_H

#include <stddef.h>

#include "claire.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Y = act(bias + conv3x3x3(X, W)): act 0 = identity, 1 = leaky ReLU with
 * `slope` for negative inputs.  Cin a multiple of 16, Cout one of 16, 32,
 * 48, 64, 96, 128, 192;
 * D, H, W powers of two >= 4 with D*H*W >= 64 (any bias may be NULL).
 * BF16 inputs and outputs, FP32 accumulation on the tensor cores: grids with
 * H a multiple of 16 and W of 8 run on tcgen05 (accumulators in TMEM, one
 * CTA per 1 x 16 x 8 brick); smaller grids on mma.sync.  A tcgen05 CTA whose
 * completion wait gives up (it never should) counts an error that
 * claire_net_device_errors reports; its outputs are then unspecified. */
claire_status claire_net_conv3d(const void* x, int x_stride, int cin, const void* w, const float* bias,
                                float slope, int act, void* y, int y_stride, int cout, const int vol[4],
                                void* stream);

/* Weights of the adjoint convolution: wf[ci][tap][co] = w[co][26 - tap][ci]
 * (BF16, Cin*27*Cout elements).  claire_net_conv3d(dY, wf) is then the
 * input gradient dX of the convolution (no bias, no activation). */
claire_status claire_net_conv3d_flip(const void* w, int cout, int cin, void* wf, void* stream);

/* Number of voxel chunks the weight gradient is split into (fixed by the
 * shapes and the device's SM count): `part` needs chunks*Cout*27*Cin floats
 * and `part_bias` chunks*Cout floats. */
claire_status claire_net_conv3d_wgrad_chunks(int cin, int cout, const int vol[4], int* chunks);

/* Weight gradient of Y = conv3x3x3(X, W) for the output gradient dY (the
 * pre-activation gradient): dw[co][tap][ci] = sum_p dY[p][co] X[p+off][ci]
 * and db[co] = sum_p dY[p][co] (FP32; db may be NULL).  Per-chunk partials
 * are summed in a fixed order, so the result is deterministic.  Volumes with
 * H % 16 == 0 and W % 8 == 0 run on the tcgen05 tensor cores (voxels as the
 * reduction dimension, accumulators in TMEM); others on mma.sync. */
claire_status claire_net_conv3d_wgrad(const void* x, int x_stride, int cin, const void* dy, int dy_stride,
                                      int cout, const int vol[4], int chunks, float* part, float* part_bias,
                                      float* dw, float* db, void* stream);

/* 2x2x2 average pooling: y (coarse vol) = mean of the 8 children of x. */
claire_status claire_net_pool2(const void* x, int x_stride, int c, void* y, int y_stride, const int vol[4],
                               void* stream);
/* Its backward: dx (fine) = dy / 8, plus add (fine, may be NULL). */
claire_status claire_net_pool2_bwd(const void* dy, int dy_stride, const void* add, int add_stride, int c, void* dx,
                                   int dx_stride, const int vol[4], void* stream);
/* Nearest 2x upsampling: every child of a coarse voxel gets its value. */
claire_status claire_net_up2(const void* x, int x_stride, int c, void* y, int y_stride, const int vol[4],
                             void* stream);
/* Its backward: dx (coarse) = sum of dy over the 8 children. */
claire_status claire_net_up2_bwd(const void* dy, int dy_stride, int c, void* dx, int dx_stride, const int vol[4],
                                 void* stream);
/* Leaky ReLU backward through its output y: dp = dy * (y > 0 ? 1 : slope). */
claire_status claire_net_leaky_bwd(const void* dy, int dy_stride, const void* y, int y_stride, int c, float slope,
                                   void* dp, int dp_stride, const int vol[4], void* stream);

/* Network input: x[p] = (a0*m0[p], a1*m1[p], 0, ..., 0) over `stride`
 * channels (even, >= 2); m0, m1 FP32 [nvox]. */
claire_status claire_net_pack(const float* m0, const float* m1, float a0, float a1, size_t nvox, void* x,
                              int stride, void* stream);

/* Output head, a 1x1x1 conv to nout channels (3: the velocity; 4: the
 * velocity and, as channel 3, the logit o of the coarse preconditioner weight,
 * see claire_net_pcw_weight):
 * v[b][c][p] = scale * (bh[c] + sum_ci x[b,p][ci] wh[c][ci]); v FP32
 * [B][nout][D][H][W] (channels 0..2 in physical units, the layout of
 * claire_transport's v for each sample); wh FP32 [nout][cin], cin 16 or 32. */
claire_status claire_net_head(const void* x, int x_stride, int cin, int nout, const float* wh, const float* bh,
                              float scale, void* v, const int vol[4], void* stream);
/* Partial blocks of claire_net_head_bwd: `part` needs blocks*(nout*cin+nout) floats. */
claire_status claire_net_head_bwd_blocks(const int vol[4], int* blocks);
/* Head backward for dv (FP32, layout of v): dx[b,p][ci] = scale sum_c
 * dv[b][c][p] wh[c][ci] (BF16, dx may be NULL) and dwb = [dwh (nout*cin),
 * dbh (nout)] (FP32, fixed-order reduction). */
claire_status claire_net_head_bwd(const void* x, int x_stride, int cin, int nout, const float* wh, float scale,
                                  const float* dv, void* dx, int dx_stride, const int vol[4], int blocks,
                                  float* part, float* dwb, void* stream);

/* One Adam step (bias-corrected, step >= 1) on FP32 master weights w with
 * gradient gscale*g; m, s are the moment buffers; wb (may be NULL) receives
 * the updated weights as BF16. */
claire_status claire_net_adam(float* w, const float* g, float* m, float* s, size_t n, float lr, float beta1,
                              float beta2, float eps, int step, float gscale, void* wb, void* stream);

/* Training loss pieces (FP32 arrays of n values, `sum` one device double
 * that is ADDED to, may be NULL; its rounding may differ between runs since
 * blocks add their partials atomically):
 * velocity term dv = a (v - vstar) + b gv (gv may be NULL), sum += |v - vstar|^2;
 * residual r = x - y (r may be NULL), sum += |x - y|^2. */
claire_status claire_net_vel_loss(const float* v, const float* vstar, const float* gv, float a, float b, size_t n,
                                  float* dv, double* sum, void* stream);
claire_status claire_net_residual(const float* x, const float* y, size_t n, float* r, double* sum, void* stream);

/* Coarse preconditioner correction (the network's second output).  The
 * two-level preconditioner (Sec. 2.2, "Optimization") inverts on a coarse
 * grid the zero-velocity operator S + gbar gbar^T; the correction is a
 * pointwise weight w >= 0 of its data term, S + gbar w gbar^T (w = 1: the
 * paper's operator; claire_set_pc_weight installs it).  The network predicts
 * o with w = softplus(o) = log(1 + e^o); its training target is the
 * least-squares fit of that model to the data term of the true Gauss-Newton
 * matvec on probe fields p, pooled over 2 x 2 x 2 cells.
 *
 * Fit statistics, added to num and den (FP32 [n]): with a = gbar . p,
 * num += a (gbar . (hp - sp)), den += a^2 |gbar|^2, where gbar is the mean
 * state gradient (claire_mean_state_gradient), hp = H p the Gauss-Newton
 * matvec and sp = S p the regulariser (claire_spectral); vector fields FP32
 * [3][n]. */
claire_status claire_net_pcw_stats(const float* gbar, const float* p, const float* hp, const float* sp, size_t n,
                                   float* num, float* den, void* stream);
/* Training loss of w = softplus(o) (o, num, den, dout FP32 on the grid
 * grid[0] x grid[1] x grid[2], even extents): with A and B the sums of den
 * and num over the voxel's 2 x 2 x 2 cell and T the sum of den,
 * L = sum_x (A w^2 - 2 B w + B^2 / A) / (8 T) (cells with A > 0), minimised by
 * w = B / A; dout = scale dL/do.  sums: two device doubles; sums[0] must be 0
 * on entry and receives T, sums[1] += L. */
claire_status claire_net_pcw_loss(const float* o, const float* num, const float* den, const int grid[3],
                                  float scale, float* dout, double* sums, void* stream);
/* Preconditioner weight from the network's logit: w = softplus(o), FP32 [n]. */
claire_status claire_net_pcw_weight(const float* o, float* w, size_t n, void* stream);

/* Tiling of the tcgen05 convolution for this process: bricks of bdc x 16 x 8
 * voxels (bdc 1, 2 or 4: D planes sharing one staged halo) and nstage 1 or 2
 * shared-memory stages (2: the next channel slice is staged while the tensor
 * cores work).  0 restores the automatic choice (the deepest brick that
 * leaves two waves of CTAs, one stage).  A forced setting that does not fit a
 * shape (D % bdc, TMEM or shared memory) makes that call fail with
 * CLAIRE_ECUDA.  Meant for tuning and tests; not thread-safe. */
claire_status claire_net_set_conv_tiling(int bdc, int nstage);

/* Input channels per CTA of the tcgen05 weight gradient for this process:
 * nc 16, 32, 48 or 64 (0 = automatic, 16).  Each CTA accumulates three taps
 * x nc channels per MMA and as many (kd, kw) tap triples as TMEM holds; a
 * larger nc means wider MMAs but more passes over each brick.  A forced nc
 * that does not divide Cin leaves that shape to the mma.sync kernel.  Meant
 * for tuning and tests; not thread-safe.  Fails with CLAIRE_EINVAL for any
 * other nc. */
claire_status claire_net_set_wgrad_tiling(int nc);

/* Number of tcgen05 CTAs whose bounded completion wait gave up since the
 * last reset (reset != 0 clears it).  Synchronises the device.  A CTA that
 * gives up agrees on it block-wide, writes no output, and releases its
 * tensor memory only after a final commit shows that its MMAs have drained. */
claire_status claire_net_device_errors(int* count, int reset);

/* Failure-detection hook of the tcgen05 kernels (the paper has no
 * counterpart; for tests).  spin_limit: polls of every bounded mbarrier wait
 * (0 restores the default, 2^22).  stall != 0: every CTA of the tcgen05
 * kernels launched afterwards first waits on a completion phase that nothing
 * signals, before it stages data or issues an MMA; that wait runs out after
 * spin_limit polls and the CTA gives up (counted by claire_net_device_errors,
 * outputs unspecified) and returns with its tensor memory released.  stall = 0
 * switches the hook off.  tmem_kept (nullable) receives the number of CTAs
 * that gave up and could not confirm that their MMAs had drained, which
 * therefore returned without releasing their tensor-memory columns (0 unless
 * the tensor cores stop completing work).  Synchronises the device; call it
 * only while no network kernel is running. */
claire_status claire_net_set_wait_test(unsigned int spin_limit, int stall, int* tmem_kept);

/* Message of the last failing claire_net_* call on this thread. */
const char* claire_net_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CLAIRE_NET_H */
