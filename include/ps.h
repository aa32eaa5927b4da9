/*
 * ps.h -- C-ABI of the GB300 (sm_103a) F-BMP blind pansharpening library.
 *
 * Method: L. Yu, D. Liu, H. Mansour, P. T. Boufounos, "Fast and High-Quality
 * Blind Multi-Spectral Image Pansharpening", arXiv 2103.09943.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Images are float32, row-major, band-planar: the LRMS X is N x h x w, the
 *   PAN Y and every HRMS band are H x W, with H = c h and W = c w for the
 *   resolution ratio c >= 2 (Sec. II-A, "Notation").
 * - The blur kernel u is n x n float32, n = 2R + 1; tap (i, j) in [-R, R]^2
 *   is stored at u[(i + R) n + (j + R)]. B(u) is circular convolution,
 *   (B(u) z)(y, x) = sum_{i,j} u(i, j) z(y - i, x - j) with indices modulo
 *   H and W (Sec. II-A); D keeps the samples (c k, c l).
 * - All image, kernel and workspace pointers are DEVICE pointers owned by the
 *   caller; host pointers are marked h_. The library allocates nothing: the
 *   scratch it needs lives in a caller-provided workspace (d_ws, ws_bytes),
 *   256-byte aligned, sized by the matching *_workspace_size call.
 * - Calls are stream-ordered on `stream` (a cudaStream_t passed as void*;
 *   NULL is the legacy default stream). Argument and shape errors are
 *   detected on the host and returned before anything is launched. A call
 *   given a non-NULL h_info blocks until its work on `stream` has finished
 *   and then fills h_info; with h_info == NULL the call returns as soon as
 *   its work is enqueued.
 * - Intensities are expected on the [0, 255] scale: the paper states its
 *   images on that scale (Sec. IV-C) and its parameter values assume it.
 * - No C++ exception crosses this interface. Calls from several host
 *   threads at once are not supported: besides the workspace, the library
 *   keeps per-device side streams, events and cached CUDA graphs that its
 *   calls share.
 */
#ifndef PS_H
#define PS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ps_status {
    PS_OK = 0,
    PS_ERR_INVALID_ARG = 1,   /* NULL pointer, bad parameter value          */
    PS_ERR_SHAPE = 2,         /* H != c h, kernel larger than the LR grid... */
    PS_ERR_CUDA = 3,          /* a CUDA runtime call failed                  */
    PS_ERR_WORKSPACE = 4,     /* workspace too small or not 256-B aligned    */
    PS_ERR_NOT_CONVERGED = 5, /* iteration cap reached; result still written */
    PS_ERR_NONFINITE = 6,     /* NaN or Inf met in a reduction               */
    PS_ERR_BREAKDOWN = 7,     /* CG met p^T A p <= 0                         */
    PS_ERR_UNSUPPORTED = 8,   /* size outside what the kernels support       */
    PS_ERR_TIMEOUT = 9        /* a bounded device-side wait gave up          */
} ps_status;

/* Parameters of Algorithm 1 (blur kernel estimation). Defaults
 * (ps_default_kernel_params) are the values of Sec. IV-F. */
typedef struct ps_kernel_params {
    float lambda_omega; /* weight of ||G omega||^2 in Eq. objective3 (10)     */
    int l;              /* half-width of the LR box u1 of Eq. objective3;
                           the HR box u2 has half-width c*l. Not given by the
                           paper; default 2                                   */
    float alpha1;       /* TGV^2 weight of ||grad u - p||_{2,1}, Eq. reg1 (1) */
    float alpha2;       /* TGV^2 weight of ||E(p)||_{2,1}, Eq. reg1 (0.006)   */
    float mu1, mu2, mu3;/* penalties of Eq. Lagrangian (100 each)             */
    float rho;          /* multiplier step of Eq. subproblems (0.5)           */
    int t_max;          /* iteration cap of Algorithm 1 (10000)               */
    float th;           /* stop when ||u^t - u^{t+1}|| / ||u^{t+1}|| < th (1e-5) */
    unsigned long long band_mask; /* the LRMS channels X' of Eq. objective1,
                           those spectrally overlapped with the PAN (Sec. II,
                           N' <= N): bit b set takes band b. 0 (default)
                           takes all N bands. Bits at or above N are an
                           error (PS_ERR_INVALID_ARG).                        */
} ps_kernel_params;

/* Cross-channel prior of Algorithm 2 (Sec. IV-D, Table III): the filter F_d
 * whose local affine relation to F_d Y is regularised. */
typedef enum ps_prior {
    PS_PRIOR_LLP = 0, /* the 5-point Laplacian (the paper's method)        */
    PS_PRIOR_LPF = 1, /* the blur kernel u (low-pass)                      */
    PS_PRIOR_HPF = 2, /* delta - u (high-pass)                             */
    PS_PRIOR_LPP = 3, /* delta (the pixels)                                */
    PS_PRIOR_LGC = 4  /* horizontal and vertical first differences, each
                         with its own affine model (Eq. reg2_lgc)          */
} ps_prior;

/* Parameters of Algorithm 2 (per-band HRMS solve). */
typedef struct ps_hrms_params {
    float lambda;       /* LLP weight of Eq. pansharp (2e-4, Sec. IV-F)        */
    int r;              /* window radius of Eq. reg2, windows (2r+1)^2 (1)     */
    float eps;          /* epsilon of Eq. reg2; not given by the paper;
                           default 1.0 on the [0, 255] scale                   */
    float tol;          /* CG for Eq. Z_ini_matting stops when the recursive
                           residual ||b - A z|| / ||b|| <= tol (default 1e-6) */
    int max_iter;       /* CG iteration cap (default 5000)                     */
    int exact_weight;   /* 0: the Z step of Eq. Z_solution uses lambda as
                           printed; 1: lambda (2r+1)^2, the exact minimiser of
                           Eq. pansharp for fixed A, C                         */
    int host_loop;      /* 0: the CG loop runs on the device as one CUDA graph
                           with a conditional while node (default); 1: the
                           host launches the same iteration kernels itself and
                           reads the stop flag every 8 iterations, for tools
                           that cannot look inside conditional graphs
                           (profilers). Results are identical.              */
    int precond;        /* preconditioner of the Z0 CG. 0: none, plain CG as in
                           the paper. 1 (default): P = B^T D^T D B
                           + lambda gamma L^T L, the Z-step operator of
                           Eq. Z_solution with M of Eq. Z_ini_matting replaced
                           by gamma I, applied exactly by FFT and a per-alias-
                           group solve (FP32). The solution and the stop rule
                           are unchanged; the iteration count drops.
                           2: diagonal, P^{-1} = diag(s) with s > 0 per pixel
                           and band, from precond_diag or from the learned
                           diagonal network diag_params.
                           3: Jacobi, P^{-1} = diag(A)^{-1} with A the Z0
                           operator itself (its exact diagonal, computed
                           once per solve; see ps_op_jacobi_diag).         */
    float precond_gamma; /* gamma of P (default 4; any value in [1, 8] gives
                           about the same iteration counts)                   */
    int warm;           /* start point of the Z0 CG when d_z_init is NULL.
                           0 (default): zeros, as in the paper. 1: bicubic
                           x ratio upsampling of the LRMS band (Keys, a = -1/2,
                           phase 0, circular). 2: the learned warm start of
                           include/ps_cnn.h on (bicubic, PAN), parameters
                           cnn_params. The stop rule is the same for all. */
    const float *cnn_params; /* device, ps_cnn_param_count() FP32 values;
                           read only when warm == 2                        */
    int stop_rule;      /* stop test of the Z0 CG. 0 (default): the recursive
                           residual ||b - A z|| / ||b|| <= tol, independent of
                           the start point. 1: the paper's rule (Sec. IV-F):
                           the relative change of the iterate in the
                           Frobenius norm, ||z_k+1 - z_k|| / ||z_k+1|| < tol
                           (the paper's tol is 5e-5); it depends on the start
                           point and on the preconditioner.              */
    int zstep_fp32;     /* Z step of Eq. Z_solution: 0 (default) forward FFT and
                           group solve in FP64, inverse in FP32 (rel-L2 to the
                           exact solve ~1e-7); 1 all in FP32 through the
                           preconditioner's register FFTs (~1e-5), for the
                           mixed-precision form whose bar is 1e-3. LLP only;
                           sizes the preconditioner does not take use FP64. */
    int prior;          /* ps_prior (default PS_PRIOR_LLP). The alternatives
                           replace L by their filters in Eq. Z_ini_matting,
                           the guided filter and Eq. Z_solution; they take
                           the plain CG (precond must be 0) and one branch
                           per iteration.                                */
    const float *precond_diag; /* precond == 2: the diagonal s of P^{-1}
                           (device, N x H x W FP32, every value > 0 and
                           finite, caller-owned, read during the solve).
                           NULL: s comes from diag_params. Not accepted by
                           ps_pansharpen_batched (one diagonal per scene). */
    const float *diag_params; /* precond == 2 without precond_diag: device,
                           ps_cnn_param_count() FP32 values of the diagonal
                           network, the architecture of include/ps_cnn.h on
                           (bicubic, PAN); s = max((net - bicubic) / 255,
                           1/64). It is trained (ps_cnn_loss_grad_weighted)
                           so that z_w + kappa s r_0 fits the solution from
                           a warm start z_w with residual r_0; PCG does not
                           depend on the scale kappa.                      */
} ps_hrms_params;

/* Per-band result of the Z0 conjugate-gradient solve. */
typedef struct ps_band_info {
    int status;          /* PS_OK, PS_ERR_NOT_CONVERGED, _NONFINITE, _BREAKDOWN */
    int iters;           /* CG iterations taken                                */
    double rel_residual; /* final recursive ||r|| / ||b||                      */
    float ms;            /* device time of this band's Z0 solve: from the
                            solve's initialisation to the end of the CG
                            iteration in which the band stopped (the
                            device's global timer). The bands of a call run
                            together, so their times overlap.              */
} ps_band_info;

/* Result of the kernel estimate. */
typedef struct ps_kernel_info {
    int status;          /* PS_OK or PS_ERR_NOT_CONVERGED                      */
    int iters;           /* ADMM iterations taken                              */
    double last_change;  /* ||u^t - u^{t+1}|| / ||u^{t+1}|| at exit            */
} ps_kernel_info;

void ps_default_kernel_params(ps_kernel_params *h_params);
void ps_default_hrms_params(ps_hrms_params *h_params);
const char *ps_status_string(int status);

/* Statuses the device detects (a band's CG not converged, non-finite or in
 * breakdown; the kernel estimate not converged) land in h_info when a call
 * is given one, and are also recorded as a sticky status: the first such
 * status since the last ps_sync_status in the current CUDA context. This
 * call waits for the work queued on `stream`, returns that status (PS_OK
 * when none, PS_ERR_CUDA when the wait fails) and clears it, so that calls
 * made without h_info (which return before their work runs) can be checked
 * afterwards. Waits that give up inside the warm-start network are reported
 * by ps_cnn_sync_status. */
ps_status ps_sync_status(void *stream);

/* Launch choices of the tunable kernels of ps_solve_hrms for one size, and
 * the times (microseconds, one launch on the workload's sizes) that picked
 * them; 0 marks a candidate that was not valid. */
typedef struct ps_tuning {
    int prec_rows;       /* rows per CTA of the preconditioner's row FFTs   */
    int llp_rows;        /* output rows per warp of the CG loop's LLP kernel */
    int llp_pf;          /* rows its loads run ahead (2, 3, 4 in registers;
                            8: a ring of 8 rows filled by asynchronous
                            copies into shared memory)                      */
    float prec_us[4];    /* candidates 1, 2, 4, 8 rows                      */
    float llp_us[6];     /* candidates: long walk with 2, 3, 4 rows ahead,
                            then the short walk                             */
    int split;           /* parallel branches of a CG iteration (1, 2, 4)    */
    float split_us[3];   /* two CG iterations, candidates 1, 2, 4 branches   */
    int llp_bands;       /* bands per CTA of that LLP kernel (1, 2)          */
    float llp2_us[2];    /* two bands per CTA: long, short walk (2 ahead)    */
    int prec_impl;       /* preconditioner passes: 1 shared-memory (any size;
                            for power-of-two columns too long for one CTA,
                            e.g. 8192 at ratio 4, the column pass splits each
                            alias-group set over a cluster of two CTAs),
                            2 register-resident (power-of-two sides 256 ..
                            4096, 384, 768, 1536; ratios 2 and 4), 3 the
                            shared-memory passes with that cluster column
                            pass at any power-of-two size with an even ratio
                            (not timed by the autotuner); 0 the default (2
                            where it applies)                               */
    float prec_impl_us[2]; /* one application: candidates 1 (its best row
                            count), 2                                        */
    int db_impl;         /* blur-decimate D B p of the CG loop: 1 one load
                            per sample and LR site, 2 four LR sites a thread
                            from register runs of the phase planes; 0 the
                            default (1)                                      */
    float db_impl_us[2]; /* one launch: candidates 1, 2                      */
    float llp_ring_us[2]; /* LLP kernel with the ring: long, short walk      */
    int llp_form;        /* form of that LLP kernel: 1 the general walk (two
                            columns a lane, any r); for r = 1 only, with one
                            band per CTA, 2 or 4 rows ahead and 64 or 32 rows
                            a warp: 2 the lean two-column walk, 4 four columns
                            a lane (W % 4 == 0); 0 the default (1)           */
    float llp_lean_us[8]; /* the lean walks: form 2 long walk with 2, 4 rows
                            ahead, short walk with 2, 4; then form 4 alike    */
} ps_tuning;

/* Autotuner: times every candidate of each tunable kernel on N bands of
 * H x W (CUDA events on `stream`, zeroed scratch in the caller's workspace
 * of ps_workspace_size) and records the fastest for this device and sizes;
 * later ps_solve_hrms / ps_pansharpen calls with the same sizes use it.
 * With a scene (d_lrms, d_pan, d_kernel as for ps_solve_hrms; all NULL to
 * skip) it also times whole solves of 20 CG iterations for each number of
 * parallel branches. Synchronises the stream. h_out may be NULL. */
ps_status ps_autotune(int N, int H, int W, int ratio, int R, int r,
                      const float *d_lrms, const float *d_pan, const float *d_kernel,
                      void *d_ws, size_t ws_bytes, void *stream, ps_tuning *h_out);

/* The launch choices recorded for these sizes on the current device (all
 * zero: the defaults), and their replacement, e.g. with choices an earlier
 * process's ps_autotune found. Only the choice fields (prec_rows, llp_rows,
 * llp_pf, split, llp_bands, prec_impl, db_impl, llp_form) are read or
 * written; 0 keeps a default. */
ps_status ps_get_tuning(int N, int H, int W, int ratio, int r, ps_tuning *h_out);
ps_status ps_set_tuning(int N, int H, int W, int ratio, int r, const ps_tuning *h_in);

/* Workspace bytes needed by ps_pansharpen (covers ps_estimate_kernel and
 * ps_solve_hrms for the same sizes; h_hrms may be NULL, and with warm == 2
 * the network's workspace is included). 0 when a size is invalid. */
size_t ps_workspace_size(int N, int H, int W, int ratio, int R,
                         const ps_hrms_params *h_hrms);

/*
 * Algorithm 1 (Sec. III-A): blur kernel estimation.
 *   omega: spectral weights of Eq. objective3 over the bands X' that
 *          h_params->band_mask selects (all N when it is 0), in closed form,
 *          unless d_omega_in is non-NULL (N floats, used as given; entries
 *          of bands outside X' are ignored);
 *   E^T E, E^T f of Eq. z_solution with E = D C(Y), f = X' omega,
 *          accumulated in FP64, and the Cholesky factor of E^T E + mu3 I;
 *   the generalized ADMM of Eq. subproblems until
 *          ||u^t - u^{t+1}|| / ||u^{t+1}|| < th or t_max iterations.
 * Out: d_kernel (n x n, in the simplex of Eq. simplex), d_omega_out (N floats,
 * may be NULL): the weight of every band of X', 0 for the other bands.
 */
ps_status ps_estimate_kernel(const float *d_lrms, const float *d_pan, int N,
                             int H, int W, int ratio, int R,
                             const ps_kernel_params *h_params,
                             const float *d_omega_in, float *d_kernel,
                             float *d_omega_out, ps_kernel_info *h_info,
                             void *d_ws, size_t ws_bytes, void *stream);

/*
 * Algorithm 2 (Sec. III-B): the HRMS image given the kernel, all bands in
 * one batch. Per band i:
 *   Z0_i solves (B^T D^T D B + lambda L^T M L) Z0_i = B^T D^T X_i
 *        (Eq. Z_ini_matting) by conjugate gradients, M the matting matrix of
 *        L Y (Eq. matting_matrix, denominator sigma^2 + eps), applied without
 *        forming it; FP32 vectors, FP64 inner products;
 *   A_i, C_i by the guided filter of Eq. ac_h_compute, giving L-hat;
 *   Z_i solves (B^T D^T D B + lambda' L^T L) Z_i = B^T D^T X_i + lambda' L L-hat
 *        (Eq. Z_solution) exactly, by FFT and a per-alias-group rank-one
 *        solve (lambda' = lambda, or lambda (2r+1)^2 with exact_weight).
 * d_z_init: N x H x W warm start for the CG, or NULL for zeros.
 * Out: d_hrms (N x H x W); d_z0 (N x H x W, may be NULL) receives Z0.
 * h_info: N entries or NULL.
 * Sizes: H and W must factor as 2^a 3^b (FFT), W a multiple of 4, and
 * H, W <= 16384.
 */
ps_status ps_solve_hrms(const float *d_lrms, const float *d_pan,
                        const float *d_kernel, int N, int H, int W, int ratio,
                        int R, const ps_hrms_params *h_params,
                        const float *d_z_init, float *d_hrms, float *d_z0,
                        ps_band_info *h_info, void *d_ws, size_t ws_bytes,
                        void *stream);

/*
 * The two-stage scheme of Sec. III-C: ps_estimate_kernel, then
 * ps_solve_hrms with the estimated kernel, no outer loop.
 * d_kernel_out (n x n, may be NULL) receives the estimated kernel.
 * The result is the same as the two calls in sequence. The solve's steps
 * that do not read the kernel (PAN statistics, warm start) run while the
 * kernel is estimated: the estimate goes on the library's own
 * high-priority streams, forked from and joined back to `stream` with
 * events, so the call stays ordered on `stream` like any other.
 */
ps_status ps_pansharpen(const float *d_lrms, const float *d_pan, int N, int H,
                        int W, int ratio, int R,
                        const ps_kernel_params *h_kparams,
                        const ps_hrms_params *h_hparams, float *d_hrms,
                        float *d_kernel_out, ps_kernel_info *h_kinfo,
                        ps_band_info *h_binfo, void *d_ws, size_t ws_bytes,
                        void *stream);

/* One scene of a batched call: device pointers and sizes as for
 * ps_pansharpen / ps_solve_hrms. */
typedef struct ps_scene {
    const float *lrms;   /* N x h x w                                      */
    const float *pan;    /* H x W                                          */
    float *hrms;         /* out: N x H x W                                 */
    float *kernel;       /* n x n, n = 2R + 1: written when the call
                            estimates the kernel, read otherwise           */
    int N, H, W, ratio, R;
    unsigned long long band_mask; /* X' of this scene (bit b: band b);
                            0 takes h_kparams->band_mask                   */
    /* Optional host copies in page-locked host memory (e.g. cudaHostAlloc;
     * NULL: none). The scene's branch of the batch graph first copies h_lrms
     * into lrms and h_pan into pan, and after its Z step copies hrms into
     * h_hrms. The copies are nodes of the batch's graph, so they overlap the
     * other scenes' work. A host pointer that is not page-locked is
     * PS_ERR_INVALID_ARG. */
    const float *h_lrms; /* N x h x w                                      */
    const float *h_pan;  /* H x W                                          */
    float *h_hrms;       /* N x H x W                                      */
} ps_scene;

/* Workspace bytes of ps_pansharpen_batched for these scenes: a header of
 * (count + 1) timer stamps, then one ps_workspace_size slice per scene.
 * 0 when a scene's sizes are invalid. */
size_t ps_batch_workspace_size(const ps_scene *h_scenes, int count,
                               const ps_hrms_params *h_hparams);

/*
 * Many scenes of uneven sizes (and band counts, and kernel supports) in one
 * launch: Algorithm 1 for every scene when h_kparams is non-NULL (else each
 * scene's kernel is given), then Algorithm 2 for all their bands, as
 * ps_pansharpen / ps_solve_hrms would compute them one by one. The whole
 * batch is one CUDA graph launched once: every scene is an independent
 * branch whose CG loop is a device-side conditional node of its own, so
 * small scenes run beside large ones and the GPU never waits on the host.
 * The executable graph is built on the first call and reused while the
 * scenes, parameters, workspace and tuning stay the same. host_loop must be
 * 0. h_kinfo: count entries or NULL; h_binfo: sum of the scenes' N entries,
 * in scene order, or NULL (either makes the call blocking). Scenes must not
 * overlap in their outputs.
 */
ps_status ps_pansharpen_batched(const ps_scene *h_scenes, int count,
                                const ps_kernel_params *h_kparams,
                                const ps_hrms_params *h_hparams,
                                ps_kernel_info *h_kinfo, ps_band_info *h_binfo,
                                void *d_ws, size_t ws_bytes, void *stream);

/* Finish time of every scene of the last batched call on this workspace,
 * in milliseconds after the batch started on the device (the device's
 * global timer). Synchronises the stream. h_ms: count entries. */
ps_status ps_batch_scene_ms(const void *d_ws, int count, void *stream,
                            double *h_ms);

#ifdef __cplusplus
}
#endif

#endif /* PS_H */
