// Internal launch interface between the kernels and the C-ABI layer.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace ps {

// api.cu: the band count, sizes, ratio and kernel radius every image entry
// point accepts (PS_ERR_INVALID_ARG, PS_ERR_SHAPE or PS_ERR_UNSUPPORTED).
ps_status check_dims(int N, int H, int W, int c, int R);

enum LlpMode { LLP_APPLY = 0, LLP_ZRHS = 1, LLP_GF = 2, LLP_CGQ = 3 };

struct LlpArgs {
    const float *in;    // p (APPLY), Z0 (ZRHS) or q (GF); N x H x W
    const float *lr;    // D B p (APPLY) or X (ZRHS); N x h x w
    const float4 *st4;  // packed PAN statistics (I, mu, s, -) per pixel
    const float *u;
    int R, c, H, W, N;
    float lam;
    float *out;         // N x H x W (APPLY, GF)
    double2 *cout;      // packed complex images (ZRHS), FP64 for the forward FFT;
                        // NULL: ZRHS writes real bands to out
    CgBand *bands;      // CG mode of APPLY: p^T A p and alpha
    const CgGlobal *g;
    int cg;
    int ty;             // CG mode: output rows per warp (0: default)
    int pf;             // CG mode: rows the loads run ahead (2, 4 or 6 in registers,
                        // 8: a ring of 8 rows in shared memory; 0: 2)
    int nbd;            // CG mode: bands per CTA (1 or 2; 0: 1)
    int form;           // CG mode: 0 or 1 the general walk; for r = 1 and one band
                        // per CTA, 2 the lean two-column walk, 4 four columns a
                        // lane (W % 4 == 0); the lean walks take pf 2 or 4
};

// operators.cu
void launch_pan_stats(const float *Y, int H, int W, int r, float eps, float *I, float *mu,
                      float *s, float4 *st4, cudaStream_t st);
void launch_pack_stats(const float *I, const float *mu, const float *s, size_t n, float4 *st4,
                       cudaStream_t st);
// impl: the blur-decimate variant of cg_fast.cu (0 or 1: one load per sample
// and LR site; 2: four sites a thread from register runs)
void launch_db(const float *src, const float *rsrc, float *pdst, const CgBand *bands,
               const CgGlobal *g, int cg, int N, int H, int W, int c, const float *u, int R,
               float *v, cudaStream_t st, int impl = 0);
void launch_adj(const float *v, int N, int H, int W, int c, const float *u, int R, float *z,
                cudaStream_t st);
void launch_llp(const LlpArgs &a, int mode, int r, int N, cudaStream_t st);
void launch_cg_reset(CgBand *bands, CgGlobal *g, int N, double tol, int max_iter, int precond,
                     int rule, cudaStream_t st);
void launch_cg_init(const float *bvec, const float *ax0, const float *x0, float *x, float *r,
                    int N, size_t HW, CgBand *bands, CgGlobal *g, cudaStream_t st);
void launch_cg_update(float *x, float *r, const float *p, const float *q, const float *v,
                      const float *u, int R, int c, int N, int H, int W, CgBand *bands,
                      const CgGlobal *g, cudaStream_t st);
void launch_stamp(unsigned long long *t, cudaStream_t st);
void launch_cg_control(CgBand *bands, CgGlobal *g, int N, int use_cond,
                       cudaGraphConditionalHandle handle, cudaStream_t st);
cudaError_t operators_set_attrs();
size_t db_smem_bytes(int c, int R);
size_t llp_smem_bytes(int r);

// cg_fast.cu: compile-time (ratio, radius) versions of db and cg_update;
// return false when no specialisation covers (c, R)
bool launch_db_fast(const float *src, const float *rsrc, float *pdst, CgBand *bands,
                    const CgGlobal *g, int cg, int N, int H, int W, int c, const float *u, int R,
                    float *v, cudaStream_t st, int impl);
bool launch_cg_update_fast(float *x, float *r, const float *p, const float *q, const float *v,
                           const float *u, int R, int c, int N, int H, int W, CgBand *bands,
                           const CgGlobal *g, cudaStream_t st);
cudaError_t cg_fast_set_attrs();
// the same for ratio 4 and radii 12, 14, 16 (cg_fast_wide.cu)
bool launch_db_fast_wide(const float *src, const float *rsrc, float *pdst, CgBand *bands,
                         const CgGlobal *g, int cg, int N, int H, int W, int c, const float *u,
                         int R, float *v, cudaStream_t st, int impl);
bool launch_cg_update_fast_wide(float *x, float *r, const float *p, const float *q,
                                const float *v, const float *u, int R, int c, int N, int H,
                                int W, CgBand *bands, const CgGlobal *g, cudaStream_t st);
cudaError_t cg_fast_set_attrs_wide();

// fft.cu
struct FftPlan {
    int L;
    int npass;
    int radix[16];
};
bool fft_make_plan(int L, FftPlan *plan);
void launch_fft_twiddles(int L, float2 *tw32, double2 *tw64, cudaStream_t st);
void launch_fft_rows32(float2 *data, const FftPlan &plan, int rows, const float2 *tw,
                       int inverse, float *unpack, int N, size_t HW, cudaStream_t st);
void launch_fft_rows64(double2 *data, const FftPlan &plan, int rows, const double2 *tw,
                       cudaStream_t st);
void launch_transpose32(const float2 *in, float2 *out, int rows, int cols, int batch,
                        cudaStream_t st);
void launch_transpose64(const double2 *in, double2 *out, int rows, int cols, int batch,
                        cudaStream_t st);
void launch_kernel_embed(const float *u, int R, int H, int W, double2 *out, cudaStream_t st);
void launch_kernel_spectrum(const float *u, int R, int H, int W, const double2 *twW,
                            const double2 *twH, double2 *out, cudaStream_t st);
void launch_alias_solve(const double2 *spec, const double2 *bspec, float2 *sol, int nimg, int H,
                        int W, int c, float lam, cudaStream_t st, const double *tsym = nullptr);
cudaError_t fft_set_attrs();

// diag.cu: the diagonal preconditioner z = s r (per-band r^T z, beta) and the
// head s = max((zd - up) / 255, floor) of the diagonal network
void launch_diag_precond(const float *r, const float *s, float *z, int N, size_t HW,
                         CgBand *bands, cudaStream_t st);
// diag(A) of the Z0 operator (or its inverse), N copies of H x W
void launch_jacobi_diag(const float4 *st4, const float *u, int R, int c, int H, int W, int r,
                        float lam, int N, int invert, float *out, cudaStream_t st);
void launch_diag_head(const float *zd, float *s, size_t n, float floor_, cudaStream_t st);

// prior.cu: the alternative cross-channel priors
int prior_filter_radius(int prior, int R);
int prior_filter_count(int prior);
void launch_prior_filters(const float *u, int R, int prior, float *f0, float *f1,
                          cudaStream_t st);
void launch_guide_stats(const float *G, int H, int W, int r, float eps, float4 *st4,
                        cudaStream_t st);
void launch_prior_window(const float *alpha, const float4 *st4, int N, int H, int W, int r,
                         int gf, float *ta, float *tb, float *out, const CgBand *bands,
                         const CgGlobal *g, cudaStream_t st);
void launch_prior_combine(const float *t0, const float *t1, const float *p, float *q, int N,
                          size_t HW, float lam, CgBand *bands, const CgGlobal *g,
                          cudaStream_t st);
void launch_symbol_add(const double2 *fh, double *T, size_t n, int first, cudaStream_t st);
void launch_prior_pack(const float *b, const float *acc, float lam, int N, size_t HW,
                       double2 *out, cudaStream_t st);

// precond.cu: z = P^{-1} r, P = B^T D^T D B + lam L^T L (lam = lambda gamma)
struct PrecArgs {
    const float *r;       // N x H x W
    float *z;             // N x H x W
    float2 *spec;         // ceil(N/2) x W x H complex scratch
    const float2 *bh;     // kernel spectrum B^, layout [kx][ky]
    const float2 *twW, *twH;
    FftPlan pw, ph;
    int N, H, W, c;
    float lam;
    CgBand *bands;        // NULL: plain operator (no r^T z, no skipping)
    const CgGlobal *g;
    int rows;             // rows per CTA of the row passes (0: the plan's choice)
    int impl;             // 0: register-resident passes where supported, else the
                          // shared-memory ones; 1: shared-memory; 2: register-resident
};
bool precond_supported(int H, int W, int c);
// precond_reg.cu: the register-resident passes (power-of-two sides 256..4096,
// ratios 2 and 4); launch_precond_reg returns false for other sizes
bool precond_reg_supported(int H, int W, int c);
// the shared-memory passes with the column pass over two-CTA clusters
bool precond_cluster_supported(int H, int W, int c);
bool launch_precond_reg(const PrecArgs &a, cudaStream_t st);
cudaError_t precond_reg_set_attrs();
bool precond_rows_ok(int H, int W, int c, int tr);
void launch_precond(const PrecArgs &a, cudaStream_t st);
void launch_spectrum_to_f32(const double2 *in, float2 *out, size_t n, cudaStream_t st);
cudaError_t precond_set_attrs();
// precond_wide.cu: the column pass's 512- and 1024-thread shapes (C = 2, 4)
void launch_prec_cols_wide(int C, int shape, const PrecArgs &a, bool p2, int col_per, int col_tpr,
                           int col_ld, size_t col_smem, float scale, cudaStream_t st);
cudaError_t precond_set_attrs_wide();

// cnn.cu: 3 x 3 convolutions with 32 in / 32 out channels on tcgen05
enum { CONV_PLAIN = 0, CONV_LAST = 2 };
struct Conv32Args {
    const __nv_bfloat16 *in;    // N x H x W x 32, NHWC
    __nv_bfloat16 *out;         // N x H x W x 32 (CONV_PLAIN)
    const void *wpack;          // B operand from launch_pack_w32 (18432 bytes)
    const float *bias;          // 32, or NULL
    const __nv_bfloat16 *mask;  // NULL, or out = conv * (mask > 0) (before the bias)
    int N, H, W;
    int relu;                   // bias then ReLU
    int rpi;                    // output rows per work item
    int *err;                   // set to 1 when a bounded wait gives up
    int mode;                   // CONV_*
    // CONV_LAST: the output is z = up + 255 (conv5(ReLU(conv + bias)) + b5)
    // with w5 (32 x 9 weights, then the bias); z is N x H x W FP32
    const float *up;
    const float *w5;
    float *z;
};
size_t conv32_smem_bytes();
void launch_pack_w32(const float *w, void *out, int adjoint, cudaStream_t st);
void launch_conv32(const Conv32Args &a, int num_sms, cudaStream_t st);
cudaError_t cnn_set_attrs();

// cnn_core.cu: the network's CUDA-core parts
void cnn_layout(int *w_off, int *b_off);  // w_off[6] = parameter count
void launch_cnn_first(const float *up, const float *pan, size_t pan_stride, const float *prm,
                      int B, int H, int W, __nv_bfloat16 *a1, cudaStream_t st);
void launch_cnn_last(const __nv_bfloat16 *a5, const float *up, const float *prm5, int B, int H,
                     int W, float *z, const float *target, const float *weight, float *d5,
                     double *loss, cudaStream_t st);
void launch_cnn_last_bwd(const __nv_bfloat16 *a5, const float *d5, const float *prm5, int B,
                         int H, int W, __nv_bfloat16 *D4, float *g5, cudaStream_t st);
void launch_cnn_wgrad32(const __nv_bfloat16 *act, const __nv_bfloat16 *D, int B, int H, int W,
                        float *gw, float *gb, int num_sms, cudaStream_t st);
void launch_cnn_wgrad_first(const float *up, const float *pan, size_t pan_stride,
                            const __nv_bfloat16 *D0, int B, int H, int W, float *g0,
                            cudaStream_t st);
void launch_cnn_adam(float *p, const float *g, float *m, float *v, int n, int step, float lr,
                     float b1, float b2, float eps, cudaStream_t st);

// llp2.cu: q = lam L M L p and p^T q inside the CG loop, two pixels per lane;
// rows per warp from LlpArgs::ty (llp_cgq2_rows(r, 0) long, (r, 1) short)
void launch_llp_cgq2(const LlpArgs &a, int r, int N, cudaStream_t st);
int llp_cgq2_rows(int r, int which);
// the lean walks (form 2, 4): whether one applies, and their rows per warp
bool llp_lean_supported(int form, int r, int W);
int llp_lean_rows(int which);

// tune.cu: launch choices of the tunable kernels per problem size
struct Tuning {
    int prec_rows;  // rows per CTA of the preconditioner's row passes (0: default)
    int llp_rows;   // output rows per warp of the CG-loop LLP kernel (0: default)
    int split;      // parallel branches of the CG iteration (0: default)
    int llp_pf;     // rows the LLP kernel's loads run ahead (0: default)
    int llp_bands;  // bands per CTA of the CG-loop LLP kernel (0: 1)
    int prec_impl;  // preconditioner passes: 0 default, 1 shared-memory, 2 register-resident
    int db_impl;    // blur-decimate of the CG loop: 0 default, 1 per-site loads, 2 register runs
    int llp_form;   // CG-loop LLP kernel: 0 default (1), 1 general, 2 lean two-column, 4 four-column
};
Tuning tuning_get(int dev, int N, int H, int W, int c, int r);
void launch_fill(float *p, size_t n, float v, cudaStream_t st);
void tuning_set(int dev, int N, int H, int W, int c, int r, const Tuning &t);

// warm.cu
void launch_bicubic_up(const float *X, int N, int h, int w, int c, float *out,
                       cudaStream_t st);

// kest.cu
// The LRMS channels X' of Eq. objective1 a kernel estimate reads: n band
// indices in increasing order (all N when the mask is 0).
struct BandSel {
    int n;
    unsigned char idx[kMaxBands];
};
BandSel band_sel(unsigned long long mask, int N);
void launch_box_lr(const float *X, const BandSel &sel, int h, int w, int l, float *out,
                   cudaStream_t st);
void launch_box_hr_dec(const float *Y, int H, int W, int c, int half, float *out,
                       cudaStream_t st);
void launch_omega_normal(const float *A, const float *bv, int N, int hw, double *G,
                         cudaStream_t st);
void launch_omega_solve(double *G, const BandSel &sel, int N, float lambda_omega, float *omega,
                        cudaStream_t st);
void launch_omega_mask(const float *in, unsigned long long mask, int N, float *out,
                       cudaStream_t st);
void launch_combine_f(const float *X, const float *omega, int N, int hw, float *f,
                      cudaStream_t st);
void launch_ete_lags(const float *Y, int H, int W, int c, int R, double *lags,
                     cudaStream_t st);
void launch_ete_assemble(const double *lags, int c, int R, double *EtE, cudaStream_t st);
void launch_etf(const float *Y, int H, int W, int c, int R, const float *f, double *Etf,
                cudaStream_t st);
void launch_cholesky(double *A, int n, float mu3, cudaStream_t st);
void launch_chol_solve(const double *L, const double *b, int n, double *x, cudaStream_t st);
void launch_chol_inverse(const double *L, int n, float scale, float *Q, double *tmp,
                         cudaStream_t st);
void launch_admm(const float *Q, const double *zf, int R, const ps_kernel_params &p,
                 float *kernel_out, int *info_iters, int *info_status, double *info_change,
                 cudaStream_t st);
size_t admm_smem_bytes(int R);
cudaError_t kest_set_attrs();

}  // namespace ps
