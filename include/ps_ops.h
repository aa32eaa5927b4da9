/*
 * ps_ops.h -- operator-level C-ABI of the F-BMP library: each step of the
 * hot path on its own, on device pointers, for callers that compose the
 * method themselves and for step-by-step parity checks.
 *
 * Conventions are those of ps.h (layouts, kernel storage, ownership, stream
 * order, host-side argument checks, [0, 255] scale). Band-batched operators
 * take N bands stored back to back (N x H x W or N x h x w).
 */
#ifndef PS_OPS_H
#define PS_OPS_H

#include <stddef.h>

#include "ps.h"

#ifdef __cplusplus
extern "C" {
#endif

/* v_b = D B(u) z_b for every band b (Sec. II-A, Eq. objective0).
 * d_z: N x H x W, d_v: N x (H/c) x (W/c). */
ps_status ps_op_blur_decimate(const float *d_z, int N, int H, int W,
                              int ratio, const float *d_kernel, int R,
                              float *d_v, void *stream);

/* z_b = B(u)^T D^T v_b (the adjoint of the above; with v = X it is the
 * right-hand side of Eq. Z_ini_matting). d_v: N x h x w, d_z: N x H x W. */
ps_status ps_op_blur_decimate_adj(const float *d_v, int N, int H, int W,
                                  int ratio, const float *d_kernel, int R,
                                  float *d_z, void *stream);

/* PAN window statistics (Algorithm 2, step 3): I = L Y with L the 5-point
 * Laplacian of Eq. reg2; per (2r+1)^2 torus window centred at each pixel,
 * mu = mean of I and s = 1 / (var + eps), var the population variance,
 * accumulated in FP64. All outputs H x W float32. */
ps_status ps_op_pan_stats(const float *d_pan, int H, int W, int r, float eps,
                          float *d_I, float *d_mu, float *d_s, void *stream);

/* diag(A) of the operator A = B^T D^T D B + lambda L^T M L of
 * Eq. Z_ini_matting (the same for every band), H x W into d_diag: the sum of
 * u(i, j)^2 over the taps that meet the pixel at an LR site, plus lambda
 * times the sum over the pixel's 5-point stencil pairs (a, b) of
 * L_ma L_mb M_ab, M_ab from Eq. matting_matrix (denominator sigma^2 + eps)
 * with (I, mu, s) as from ps_op_pan_stats. Its inverse is the Jacobi
 * preconditioner of ps_hrms_params.precond = 3. Workspace:
 * ps_op_workspace_size(1, H, W, ratio, R). */
ps_status ps_op_jacobi_diag(int H, int W, int ratio, const float *d_kernel, int R,
                            const float *d_I, const float *d_mu, const float *d_s, int r,
                            float lambda, float *d_diag, void *d_ws, size_t ws_bytes,
                            void *stream);

/* out_b = (B^T D^T D B + lambda L^T M L) z_b, the operator of
 * Eq. Z_ini_matting, with M the matting matrix of I (Eq. matting_matrix,
 * denominator sigma^2 + eps) applied matrix-free from (I, mu, s).
 * Workspace: ps_op_workspace_size(N, H, W, ratio). */
ps_status ps_op_apply_z0(const float *d_z, int N, int H, int W, int ratio,
                         const float *d_kernel, int R, const float *d_I,
                         const float *d_mu, const float *d_s, int r,
                         float lambda, float *d_out, void *d_ws,
                         size_t ws_bytes, void *stream);

/* Guided filter of q_b with guide I (Eq. ac_h_compute): per window
 * a = (mean(I q) - mu mean(q)) s, c = mean(q) - a mu; out = mean(a) I +
 * mean(c), means over the windows containing each pixel. N x H x W.
 * Workspace: at least 16 H W bytes, 256-byte aligned. */
ps_status ps_op_guided_filter(const float *d_q, int N, int H, int W,
                              const float *d_I, const float *d_mu,
                              const float *d_s, int r, float *d_out,
                              void *d_ws, size_t ws_bytes, void *stream);

/* Z step of Algorithm 2 (Eq. Z_solution) for every band, given Z0:
 * L-hat = guided filter of L Z0_b, then Z_b solves
 * (B^T D^T D B + lambda' L^T L) Z_b = B^T D^T X_b + lambda' L L-hat exactly
 * (FFT, per-alias-group rank-one solve). lambda' = lambda, or
 * lambda (2r+1)^2 when exact_weight. Workspace: ps_op_workspace_size. */
ps_status ps_op_zstep(const float *d_lrms, const float *d_z0, int N, int H,
                      int W, int ratio, const float *d_kernel, int R,
                      const float *d_I, const float *d_mu, const float *d_s,
                      int r, float lambda, int exact_weight, float *d_z,
                      void *d_ws, size_t ws_bytes, void *stream);

/* Preconditioner of the Z0 CG (an extension: the paper runs plain CG):
 * z_b = P^{-1} r_b with P = B^T D^T D B + lambda_gamma L^T L, the operator of
 * Eq. Z_solution at weight lambda_gamma, solved exactly in the Fourier domain
 * per alias group of ratio^2 frequencies, FP32. N x H x W in and out (device,
 * caller-owned, not aliased). H, W of the form 2^a 3^b. The passes are those
 * ps_set_tuning recorded for (N, H, W, ratio, r = 1) (prec_impl, prec_rows),
 * else the defaults. Workspace: ps_op_workspace_size. */
ps_status ps_op_precond(const float *d_r, int N, int H, int W, int ratio,
                        const float *d_kernel, int R, float lambda_gamma,
                        float *d_z, void *d_ws, size_t ws_bytes, void *stream);

/* Bicubic x ratio upsampling of N LR bands (h = H / ratio, w = W / ratio),
 * the warm start of the Z0 solve: Keys' cubic convolution (a = -1/2), HR
 * pixel ratio k + phi on LR coordinate k + phi / ratio, circular boundary.
 * d_lrms N x h x w in, d_out N x H x W out (device, caller-owned, 16-byte
 * aligned). No workspace. */
ps_status ps_op_bicubic_up(const float *d_lrms, int N, int H, int W, int ratio,
                           float *d_out, void *stream);

/* One 3 x 3 convolution of the warm-start network with 32 input and 32
 * output channels on the tensor cores (BF16 operands, FP32 accumulation),
 * circular boundary. d_in and d_out: N x H x W x 32 BF16 (NHWC, device,
 * 16-byte aligned, not aliased). d_weight: 32 x 32 x 3 x 3 FP32 as
 * (out, in, dy + 1, dx + 1); d_bias: 32 FP32 or NULL. mode 0: out =
 * ReLU(conv(in) + bias); 1: out = conv(in) + bias; 2: the adjoint in the
 * input (backward data), out = conv^T(in), times (d_mask > 0) elementwise
 * when d_mask (N x H x W x 32 BF16) is given. Workspace: 18688 bytes.
 * Synchronises the stream; PS_ERR_TIMEOUT if a bounded wait gave up. */
ps_status ps_op_cnn_conv32(const void *d_in, int N, int H, int W,
                           const float *d_weight, const float *d_bias,
                           const void *d_mask, int mode, void *d_out,
                           void *d_ws, size_t ws_bytes, void *stream);

/* Spectral weights of Eq. objective3 in closed form: the normal equations
 * of || B(u1) X omega - D B(u2) Y ||^2 + lambda_omega ||G omega||^2,
 * accumulated in FP64; u1 the (2l+1)^2 unit box on the LR grid, u2 the
 * (2cl+1)^2 unit box on the HR grid, G first differences. Out: d_omega (N). */
ps_status ps_op_omega(const float *d_lrms, const float *d_pan, int N, int H,
                      int W, int ratio, int l, float lambda_omega,
                      float *d_omega, void *d_ws, size_t ws_bytes,
                      void *stream);

/* E^T E (n^2 x n^2, FP64, full symmetric) and E^T f (n^2, FP64) of
 * Eq. z_solution, with E = D C(Y) (row q holds Y(c q - a) for every tap a)
 * and f = sum_b omega_b X_b. Workspace: ps_op_workspace_size. */
ps_status ps_op_kernel_normal_eq(const float *d_lrms, const float *d_pan,
                                 const float *d_omega, int N, int H, int W,
                                 int ratio, int R, double *d_EtE,
                                 double *d_Etf, void *d_ws, size_t ws_bytes,
                                 void *stream);

/* The ADMM loop of Algorithm 1 given E^T E and E^T f (FP64, as above).
 * Out: d_kernel (n x n, in the simplex). */
ps_status ps_op_admm(const double *d_EtE, const double *d_Etf, int R,
                     const ps_kernel_params *h_params, float *d_kernel,
                     ps_kernel_info *h_info, void *d_ws, size_t ws_bytes,
                     void *stream);

/* Workspace bytes for the operator entry points above at these sizes
 * (the largest any of them needs). */
size_t ps_op_workspace_size(int N, int H, int W, int ratio, int R);

/* Size of the scratch array the library defines for
 * ps_op_kernel_normal_eq_noalloc (on every GPU that loads the library). */
#define PS_NOALLOC_SCRATCH_BYTES (4u << 20)

/* ps_op_kernel_normal_eq without a workspace. The paper has no counterpart:
 * this entry point is for callers that cannot allocate device memory on
 * their call path, such as plugins whose host application owns all device
 * memory and passes in only inputs and outputs, or real-time code that cannot
 * accept cudaMalloc's possible implicit synchronisation or failure. Inputs,
 * outputs and results are those of ps_op_kernel_normal_eq.
 * Scratch: a fixed array of PS_NOALLOC_SCRATCH_BYTES defined by the library
 * on every GPU that loads it, kept until the process exits. A call uses
 * (h w 4 bytes, rounded up to 256) + c^2 (4R+1)^2 8 bytes of it, with
 * h w = (H/ratio)(W/ratio); when that exceeds the array the call returns
 * PS_ERR_UNSUPPORTED before launching anything.
 * Sizes: the limits of ps_op_kernel_normal_eq (same status codes), then the
 * array's.
 * All calls share the one array: calls that overlap on the GPU (on different
 * streams, or from different host threads) race on it and must be serialised
 * by the caller. The array has one device address per CUDA context; the
 * first call in a context (the device's primary context, or a context the
 * caller made current through the driver API) looks that address up and
 * caches it under the context's ID. Make that first call before any stream
 * capture. */
ps_status ps_op_kernel_normal_eq_noalloc(const float *d_lrms,
                                         const float *d_pan,
                                         const float *d_omega, int N, int H,
                                         int W, int ratio, int R,
                                         double *d_EtE, double *d_Etf,
                                         void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PS_OPS_H */
