/*
 * Learned warm start of the Z0 solve (an extension: the paper's solve starts
 * from zeros). A small CNN predicts a band's Z0 from the bicubic upsampling of
 * its LRMS band and the PAN:
 *   x = (up / 255, pan / 255);  a1 = ReLU(conv0(x));  a(l+1) = ReLU(conv_l(a_l)),
 *   l = 1..4;  z = 255 (x_0 + conv5(a5))
 * with circular 3 x 3 cross-correlations, widths 2 -> 32 -> 32 -> 32 -> 32 ->
 * 32 -> 1. The 32 -> 32 layers run on the tensor cores (tcgen05, BF16
 * operands, FP32 accumulation); hidden activations are BF16. Training
 * minimises the mean squared error of z / 255 against target / 255 (the
 * method's own Z0) with Adam (Kingma & Ba 2015).
 *
 * Parameters: one FP32 vector of ps_cnn_param_count() values, layer by
 * layer, each layer's weights (out, in, 3, 3) then its biases.
 * Images: B bands of H x W, FP32, device, caller-owned; pan_stride is the
 * element distance between the PAN of consecutive bands (0: one PAN for all).
 * W % 4 == 0, H >= 3, W >= 3. All calls are stream-ordered and asynchronous;
 * argument errors return before any launch. A bounded device-side wait that
 * gives up is reported by ps_cnn_sync_status.
 */
#ifndef PS_CNN_H
#define PS_CNN_H

#include <stddef.h>

#include "ps.h"

#ifdef __cplusplus
extern "C" {
#endif

int ps_cnn_param_count(void);

/* Workspace bytes for B x H x W: training = 0 for ps_cnn_forward, 1 for
 * ps_cnn_loss_grad (it keeps every activation). */
size_t ps_cnn_workspace_size(int B, int H, int W, int training);

/* z (B x H x W) = the network on (d_up, d_pan). */
ps_status ps_cnn_forward(const float *d_params, const float *d_up, const float *d_pan,
                         size_t pan_stride, int B, int H, int W, float *d_z,
                         void *d_ws, size_t ws_bytes, void *stream);

/* Loss sum_p ((z - target) / 255)^2 / (B H W) into *d_loss (one FP64, device)
 * and its gradient with respect to every parameter into d_grad
 * (ps_cnn_param_count() FP32, overwritten). */
ps_status ps_cnn_loss_grad(const float *d_params, const float *d_up, const float *d_pan,
                           size_t pan_stride, const float *d_target, int B, int H, int W,
                           float *d_grad, double *d_loss, void *d_ws, size_t ws_bytes,
                           void *stream);

/* The same with a per-pixel weight w >= 0 (B x H x W FP32, device; NULL:
 * w = 1): loss sum_p w_p ((z - target) / 255)^2 / (B H W). This trains the
 * diagonal network of ps_hrms_params.diag_params, whose target and weight
 * turn the one-step fit of the diagonal into this form. */
ps_status ps_cnn_loss_grad_weighted(const float *d_params, const float *d_up,
                                    const float *d_pan, size_t pan_stride, const float *d_target,
                                    const float *d_weight, int B, int H, int W, float *d_grad,
                                    double *d_loss, void *d_ws, size_t ws_bytes, void *stream);

/* One Adam step (t = step >= 1) on d_params with moments d_m, d_v (FP32,
 * ps_cnn_param_count() each, zero before the first step). */
ps_status ps_cnn_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int step,
                      float lr, float beta1, float beta2, float eps, void *stream);

/* Synchronises the stream; PS_ERR_TIMEOUT if a wait of the last forward or
 * loss_grad call on this workspace gave up (the flag is then cleared). */
ps_status ps_cnn_sync_status(void *d_ws, int B, int H, int W, int training, void *stream);

#ifdef __cplusplus
}
#endif

#endif
