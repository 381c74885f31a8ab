/* libternelbm -- learned surrogate kernels (C ABI).
 *
 * The paper has no surrogate.  These entry points are the learned part built
 * on top of the method: a small convolutional encoder-decoder that advances
 * the density, composition and velocity fields of a D2Q9 lattice k steps at
 * a time, trained on snapshots of the lattice update itself, with the plain
 * update as its fallback and as the reference its error is measured
 * against.  Each entry point is one kernel
 * (or a short fixed sequence) issued on `stream` (a cudaStream_t, NULL = the
 * legacy default stream); all pointers are DEVICE pointers owned by the
 * caller, nothing is allocated or retained.  Return 0 on success,
 * TEL_EINVAL (-1) for a shape the kernels do not support (checked on the
 * host before any launch), TEL_ECUDA (-3) for a launch error.
 *
 * Conventions.
 *   Activations: NHWC bf16 [B][H][W][C] on a periodic H x W grid, C in
 *     {16, 32, 64, 128}.  B*H*W must be a multiple of 128 and H, W even
 *     where pooling is used.
 *   Conv weights: bf16 [9][Cout][Cin] (tap t = 3 (dy+1) + (dx+1), the input
 *     channel innermost); their FP32 gradients have the same layout.
 *   A 3x3 convolution is the periodic cross-correlation
 *     y[b,h,w,o] = bias[o] + sum_t sum_i x[b,(h+dy)%H,(w+dx)%W,i] W[t][o][i]
 *   with FP32 accumulation, optionally followed by ReLU, stored as bf16.
 *   Fields: normalised FP32 [B][H][W][4] = (rho/rho_l, phi/chi, u_x/U, u_y/U).
 */
#ifndef TERNELBM_SUR_H
#define TERNELBM_SUR_H

#ifdef __cplusplus
extern "C" {
#endif

/* y = relu?(conv3x3(x, w) + bias).  bias: FP32 [Cout] or NULL (zero).  The
 * tensor-core (mma.sync bf16, FP32 accumulate) implicit GEMM: M = B*H*W
 * pixels, N = Cout, K = 9*Cin. */
int tel_sur_conv3x3(const void *x, const void *w, const float *bias, void *y, int B, int H, int W, int cin,
                    int cout, int relu, void *stream);

/* The same convolution on the 5th-generation tensor cores (tcgen05.mma,
 * accumulator in tensor memory); err (device, may be NULL) is OR-ed with 1
 * if a bounded wait for the tensor cores timed out, in which case y is not
 * written. */
int tel_sur_conv3x3_tc(const void *x, const void *w, const float *bias, void *y, int B, int H, int W, int cin,
                       int cout, int relu, unsigned *err, void *stream);

/* Inference form of the tensor-memory convolution for rows of whole
 * 128-pixel segments (W a multiple of 128, H of 4): with up_input != 0, x is
 * the (H/2) x (W/2) grid read through 2x2 nearest upsampling, which saves
 * materialising the upsampled tensor; skip (bf16
 * [B][H][W][cout], may be NULL) is added to the output, rounded as a
 * separate tel_sur_add of the rounded output would be.  Other shapes:
 * TEL_EINVAL. */
int tel_sur_conv3x3_tc_fused(const void *x, const void *w, const float *bias, void *y, int B, int H, int W, int cin,
                             int cout, int relu, int up_input, const void *skip, unsigned *err, void *stream);

/* Weights for the input gradient: the input gradient of a conv is the conv
 * of its output gradient with w_t[s][i][o] = w[8-s][o][i].  Writes w_t
 * (bf16 [9][Cin][Cout]) from w (bf16 [9][Cout][Cin]). */
int tel_sur_flip_weights(const void *w, void *w_t, int cin, int cout, void *stream);

/* dz = dy * (y > 0) (the ReLU mask from the layer's own output), bf16, n
 * elements; dz may alias dy. */
int tel_sur_relu_bwd(const void *y, const void *dy, void *dz, long long n, void *stream);

/* Weight and bias gradients of a conv, ACCUMULATED into dw (FP32
 * [9][Cout][Cin]) and db (FP32 [Cout], may be NULL):
 *   dw[t][o][i] += sum_p dz[p][o] x[p + d_t][i],  db[o] += sum_p dz[p][o].
 * dz is the gradient at the pre-activation (after tel_sur_relu_bwd).  FP32
 * atomics combine pixel chunks, so the summation order is not fixed. */
int tel_sur_conv3x3_wgrad(const void *x, const void *dz, float *dw, float *db, int B, int H, int W, int cin,
                          int cout, void *stream);

/* 2x2 mean pooling, its adjoint (dx = dy/4 on each of the 4 inputs), 2x2
 * nearest upsampling and its adjoint (sum of the 4 copies).  H, W are the
 * FINE grid's sizes in all four. */
int tel_sur_pool2(const void *x, void *y, int B, int H, int W, int C, void *stream);
int tel_sur_pool2_bwd(const void *dy, void *dx, int B, int H, int W, int C, void *stream);
int tel_sur_up2(const void *x, void *y, int B, int H, int W, int C, void *stream);
int tel_sur_up2_bwd(const void *dy, void *dx, int B, int H, int W, int C, void *stream);

/* y = a + b (bf16, n elements; y may alias a or b). */
int tel_sur_add(const void *a, const void *b, void *y, long long n, void *stream);

/* Normalised fields of B lattices of H x W nodes from FP64 SoA fields
 * (rho[B][H*W], phi[B][H*W], u[B][2][H*W]) into f32 (FP32 [B][H][W][4])
 * and/or x16 (network input, bf16 [B][H][W][16], channels 4..15 zero);
 * norm = {1/rho_l, 1/chi, 1/U} per case (FP32 [B][3]). */
int tel_sur_pack(const double *rho, const double *phi, const double *u, const float *norm, float *f32, void *x16,
                 int B, int H, int W, void *stream);

/* The inverse of tel_sur_pack for the first three outputs (FP64 SoA fields
 * for handing the state back to the lattice update). */
int tel_sur_unpack(const float *f32, const float *norm, double *rho, double *phi, double *u, int B, int H, int W,
                   void *stream);

/* Training batch from a snapshot store (FP32 [S][H][W][4]): for sample k,
 * input = store[src[k]] (written to f32 [B][H][W][4] and x16) and target
 * = (store[dst[k]] - store[src[k]]) / scale (FP32 [B][H][W][4]).  sym
 * (may be NULL; square lattices only) gives per sample an element of the
 * lattice's symmetry group applied to input and target alike: bit 0 mirrors
 * x (u_x -> -u_x), bit 1 mirrors y (u_y -> -u_y), bit 2 transposes first
 * (u_x <-> u_y); mirror images of a lattice trajectory are trajectories of
 * the same update, so they augment the training set. */
int tel_sur_gather(const float *store, const int *src, const int *dst, const int *sym, const float *scale,
                   float *f32, void *x16, float *target, int B, int H, int W, void *stream);

/* Head and loss.  The prediction is the network output's channels 0..3 with
 * the spatial mean of channels 0 and 1 removed per sample (mass-conserving
 * projection P).  loss[0] += mean((P(out) - target)^2) (FP32; the caller
 * zeroes it) and dout (bf16 [B][H][W][16]) = P(2 (P(out) - target) / n),
 * zero on channels 4..15.  work: FP32 scratch of 4*B floats. */
int tel_sur_loss(const void *out, const float *target, void *dout, float *loss, float *work, int B, int H, int W,
                 void *stream);

/* Inference step: f32_next = f32 + scale * P(out) (FP32 [B][H][W][4]) and
 * x16_next (may be NULL) the matching network input; mass[2B] (FP64, the
 * caller zeroes it) receives per sample the sums of channel 0 and 1 of
 * f32_next for the mass-residual check.  work: FP32 scratch of 4*B floats. */
int tel_sur_advance(const float *f32, const void *out, const float *scale, float *f32_next, void *x16_next,
                    double *mass, float *work, int B, int H, int W, void *stream);

/* Relative field errors against a reference state (both FP32 [B][H][W][4]):
 * acc[3B*2] (FP64, caller zeroes) receives per sample sum (pred-ref)^2 and
 * sum ref^2 for rho, phi and u (u over both components). */
int tel_sur_errors(const float *pred, const float *ref, double *acc, int B, int H, int W, void *stream);

/* sums[2B] (FP64, overwritten) = per sample the sums of channels 0 and 1
 * (density and composition) of FP32 fields [B][H][W][4]. */
int tel_sur_sums(const float *f32, double *sums, int B, int H, int W, void *stream);

/* One Adam step (bias-corrected, step t >= 1) on n FP32 master weights w32
 * with gradient g and moments m, v; w16 (bf16, may be NULL) receives the
 * updated weights rounded to bf16.  grad_scale multiplies g first. */
int tel_sur_adam(float *w32, void *w16, const float *g, float *m, float *v, long long n, float lr, float beta1,
                 float beta2, float eps, int t, float grad_scale, void *stream);

/* Gradient-norm clipping without a host round trip: scale[0] (device FP32)
 * = min(1, clip / ||g||_2) over n values (norm accumulated in FP64 in
 * work[0], device); tel_sur_adam_scaled is tel_sur_adam with the gradient
 * multiplied by scale[0] read on the device. */
int tel_sur_clip_scale(const float *g, long long n, float clip, double *work, float *scale, void *stream);
int tel_sur_adam_scaled(float *w32, void *w16, const float *g, float *m, float *v, long long n, float lr, float beta1,
                        float beta2, float eps, int t, const float *scale, void *stream);

/* Zero n FP32 values (cudaMemsetAsync). */
int tel_sur_zero(float *p, long long n, void *stream);

/* w16 = bf16(w32), n elements. */
int tel_sur_to_bf16(const float *w32, void *w16, long long n, void *stream);

#ifdef __cplusplus
}
#endif
#endif
