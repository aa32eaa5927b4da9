// C-ABI of the F-BMP library: argument checks, workspace layout, stage
// orchestration and the CUDA graph that runs the CG loop on the device.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "ps.h"
#include "ps_ops.h"
#include "ps_cnn.h"

using namespace ps;

// Sizes every image entry point accepts (declared in kernels.cuh; the
// allocation-free entry point applies the same limits).
ps_status ps::check_dims(int N, int H, int W, int c, int R) {
    if (N < 1 || N > kMaxBands) return PS_ERR_INVALID_ARG;
    if (c < 2 || c > kMaxRatio) return PS_ERR_INVALID_ARG;
    if (R < 0 || R > kMaxR) return PS_ERR_INVALID_ARG;
    if (H < 1 || W < 1 || H % c || W % c) return PS_ERR_SHAPE;
    if (H > kMaxFFT || W > kMaxFFT) return PS_ERR_UNSUPPORTED;
    if (2 * R + 1 > H || 2 * R + 1 > W) return PS_ERR_SHAPE;
    if (W % 4) return PS_ERR_UNSUPPORTED;
    return PS_OK;
}

namespace {

// First non-OK status a device-side check of this library recorded in the
// current CUDA context since the last ps_sync_status (0: none): a band's CG
// status (not converged, non-finite, breakdown) or the kernel estimate's.
__device__ int g_sticky_status;

// Run at the end of every solve (bands) and kernel estimate (kinfo).
__global__ void collect_status_kernel(const CgBand *bands, int N, const int *kinfo) {
    if (threadIdx.x != 0) return;
    int s = 0;
    for (int b = 0; b < N && !s; ++b) s = bands[b].status;
    if (!s && kinfo) s = kinfo[1];
    if (s) atomicCAS(&g_sticky_status, 0, s);
}

void launch_collect_status(const CgBand *bands, int N, const int *kinfo, cudaStream_t st) {
    collect_status_kernel<<<1, 32, 0, st>>>(bands, N, kinfo);
}

}  // namespace

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// ---------------------------------------------------------------------------
// Workspace layout (offsets from the 256-byte aligned base).
// ---------------------------------------------------------------------------
struct Layout {
    size_t st4;                         // HW float4: packed PAN statistics (I, mu, s)
    size_t xbuf;                        // N HW f32 (Z0 when the caller gives none)
    size_t r, pA, pB, ap;               // N HW f32 each; [r,pA] and [pB,ap] double as
                                        // the complex FFT buffers
    size_t v;                           // N hw f32
    size_t z;                           // N HW f32: preconditioned residual
    size_t spec;                        // ceil(N/2) HW float2: preconditioner spectrum
    size_t bhat;                        // HW double2 (kernel spectrum)
    size_t bh32;                        // HW float2 (the same, rounded)
    size_t twW32, twH32, twW64, twH64;  // twiddles
    size_t bands, glob;                 // CG scalars; kMaxSplit loop-control records
    size_t bvec, f, G, omega, lags, ete, etf, zf, Q, kern, kinfo;
    size_t cnn;
    size_t total;
};

bool make_layout(int N, int H, int W, int c, int R, Layout *L) {
    if (N < 1 || H < 1 || W < 1 || c < 1 || R < 0) return false;
    const size_t HW = (size_t)H * W, hw = HW / ((size_t)c * c);
    const size_t nt = (size_t)(2 * R + 1) * (2 * R + 1);
    const size_t nl = (size_t)(4 * R + 1);
    size_t o = 0;
    auto take = [&o](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    L->st4 = take(HW * 16);
    L->xbuf = take((size_t)N * HW * 4);
    // r and pA contiguous, pB and ap contiguous: each pair doubles as one
    // complex FFT buffer of ceil(N/2) FP64 images
    const size_t pair = std::max((size_t)N * HW * 8, (size_t)((N + 1) / 2) * HW * 16);
    L->r = take(pair);
    L->pA = L->r + (size_t)N * HW * 4;
    L->pB = take(pair);
    L->ap = L->pB + (size_t)N * HW * 4;
    L->v = take((size_t)N * hw * 4);
    L->z = take((size_t)N * HW * 4);
    L->spec = take((size_t)((N + 1) / 2) * HW * 8);
    L->bhat = take(HW * 16);
    L->bh32 = take(HW * 8);
    L->twW32 = take((size_t)W * 8);
    L->twH32 = take((size_t)H * 8);
    L->twW64 = take((size_t)W * 16);
    L->twH64 = take((size_t)H * 16);
    L->bands = take((size_t)N * sizeof(CgBand));
    L->glob = take(kMaxSplit * sizeof(CgGlobal));  // one per branch loop
    L->bvec = take(hw * 4);
    L->f = take(hw * 4);
    L->G = take(((size_t)N * N + N) * 8);
    L->omega = take((size_t)N * 4);
    L->lags = take((size_t)c * c * nl * nl * 8);
    L->ete = take(nt * nt * 8);
    L->etf = take(nt * 8);
    L->zf = take(nt * 8);
    L->Q = take(nt * nt * 4);
    L->kern = take(nt * 4);
    L->kinfo = take(64);
    L->cnn = o;  // the warm-start network's workspace, when it is used
    L->total = o + kAlign;  // slack for aligning the caller's pointer
    return true;
}

struct Ws {
    char *base;
    Layout L;
    template <class T>
    T *at(size_t off) const { return reinterpret_cast<T *>(base + off); }
};

ps_status bind_ws(void *d_ws, size_t ws_bytes, int N, int H, int W, int c, int R, Ws *ws) {
    if (!d_ws) return PS_ERR_WORKSPACE;
    if (((uintptr_t)d_ws) % kAlign) return PS_ERR_WORKSPACE;
    if (!make_layout(N, H, W, c, R, &ws->L)) return PS_ERR_SHAPE;
    if (ws_bytes < ws->L.total - kAlign) return PS_ERR_WORKSPACE;
    ws->base = static_cast<char *>(d_ws);
    return PS_OK;
}

bool is_pow23(int L) {
    if (L < 1) return false;
    while (L % 2 == 0) L /= 2;
    while (L % 3 == 0) L /= 3;
    return L == 1;
}

ps_status check_fft_dims(int H, int W) {
    if (!is_pow23(H) || !is_pow23(W)) return PS_ERR_UNSUPPORTED;
    if (H < 4 || W < 4) return PS_ERR_UNSUPPORTED;
    return PS_OK;
}

ps_status check_hrms(const ps_hrms_params *p) {
    if (!p) return PS_ERR_INVALID_ARG;
    if (p->r < 1 || p->r > kMaxWinR) return PS_ERR_INVALID_ARG;
    if (!(p->lambda > 0.f) || !(p->eps > 0.f) || !(p->tol > 0.f) || p->max_iter < 1)
        return PS_ERR_INVALID_ARG;
    if (!isfinite(p->lambda) || !isfinite(p->eps) || !isfinite(p->tol))
        return PS_ERR_INVALID_ARG;
    if (p->precond < 0 || p->precond > 3) return PS_ERR_INVALID_ARG;
    if (p->precond == 1 && (!(p->precond_gamma > 0.f) || !isfinite(p->precond_gamma)))
        return PS_ERR_INVALID_ARG;
    if (p->precond == 2 && !p->precond_diag && !p->diag_params) return PS_ERR_INVALID_ARG;
    if (p->warm < 0 || p->warm > 2) return PS_ERR_INVALID_ARG;
    if (p->stop_rule != 0 && p->stop_rule != 1) return PS_ERR_INVALID_ARG;
    if (p->zstep_fp32 != 0 && p->zstep_fp32 != 1) return PS_ERR_INVALID_ARG;
    if (p->prior < PS_PRIOR_LLP || p->prior > PS_PRIOR_LGC) return PS_ERR_INVALID_ARG;
    if (p->prior != PS_PRIOR_LLP && p->precond) return PS_ERR_INVALID_ARG;
    if (p->warm == 2 && !p->cnn_params) return PS_ERR_INVALID_ARG;
    return PS_OK;
}

ps_status check_kernel_params(const ps_kernel_params *p) {
    if (!p) return PS_ERR_INVALID_ARG;
    if (p->l < 0 || p->l > 16) return PS_ERR_INVALID_ARG;
    if (!(p->lambda_omega >= 0.f) || !(p->alpha1 >= 0.f) || !(p->alpha2 >= 0.f))
        return PS_ERR_INVALID_ARG;
    if (!(p->mu1 > 0.f) || !(p->mu2 > 0.f) || !(p->mu3 > 0.f)) return PS_ERR_INVALID_ARG;
    if (!(p->rho > 0.f) || p->t_max < 1 || !(p->th >= 0.f)) return PS_ERR_INVALID_ARG;
    return PS_OK;
}

// The X' mask of Eq. objective1 selects bands that exist (0: all).
ps_status check_band_mask(unsigned long long mask, int N) {
    if (N < 64 && (mask >> N) != 0ull) return PS_ERR_INVALID_ARG;
    return PS_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p % 16) == 0; }

ps_status cuda_status(cudaError_t e) { return e == cudaSuccess ? PS_OK : PS_ERR_CUDA; }

ps_status last_launch() { return cuda_status(cudaGetLastError()); }

// One-time (per device) kernel attributes and the private capture stream.
struct DevState {
    int attrs_done = 0;
    int num_sms = 0;
    cudaStream_t capture = nullptr;
    // two branch streams and their fork / join events: the CG iteration runs
    // the two halves of the bands as parallel branches
    cudaStream_t branch[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[4] = {nullptr, nullptr, nullptr, nullptr};
    // ps_pansharpen's high-priority side stream (the kernel estimate)
    cudaStream_t early = nullptr;
    cudaEvent_t early_fork = nullptr, early_join = nullptr, early_lags = nullptr;
    // the kernel estimate's second branch (omega, E^T f, the z_f solve)
    cudaStream_t kside = nullptr;
    cudaEvent_t k_fork = nullptr, k_chol = nullptr, k_zf = nullptr;
};
std::mutex g_mu;
std::vector<DevState> g_dev;
// SMs that the warm-start network leaves free while it overlaps the kernel
// estimate (whose ADMM takes one whole SM, its Cholesky panels a few)
constexpr int kEarlyReserveSms = 2;

ps_status ensure_device(cudaStream_t *capture, int *num_sms = nullptr) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_dev.size() <= dev) g_dev.resize(dev + 1);
    DevState &d = g_dev[dev];
    if (!d.attrs_done) {
        if (operators_set_attrs() != cudaSuccess) return PS_ERR_CUDA;
        if (fft_set_attrs() != cudaSuccess) return PS_ERR_CUDA;
        if (kest_set_attrs() != cudaSuccess) return PS_ERR_CUDA;
        if (precond_set_attrs() != cudaSuccess) return PS_ERR_CUDA;
        if (cnn_set_attrs() != cudaSuccess) return PS_ERR_CUDA;
        if (cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) !=
            cudaSuccess)
            return PS_ERR_CUDA;
        d.attrs_done = 1;
    }
    if (num_sms) *num_sms = d.num_sms;
    if (capture) {
        if (!d.capture &&
            cudaStreamCreateWithFlags(&d.capture, cudaStreamNonBlocking) != cudaSuccess)
            return PS_ERR_CUDA;
        *capture = d.capture;
        for (int k = 0; k < 4; ++k) {
            if (!d.branch[k] &&
                cudaStreamCreateWithFlags(&d.branch[k], cudaStreamNonBlocking) != cudaSuccess)
                return PS_ERR_CUDA;
            if (!d.join[k] && cudaEventCreateWithFlags(&d.join[k], cudaEventDisableTiming) !=
                                  cudaSuccess)
                return PS_ERR_CUDA;
        }
        if (!d.fork && cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming) != cudaSuccess)
            return PS_ERR_CUDA;
        if (!d.early || !d.kside) {
            int lo = 0, hi = 0;
            if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) return PS_ERR_CUDA;
            if (!d.early &&
                cudaStreamCreateWithPriority(&d.early, cudaStreamNonBlocking, hi) != cudaSuccess)
                return PS_ERR_CUDA;
            if (!d.kside &&
                cudaStreamCreateWithPriority(&d.kside, cudaStreamNonBlocking, hi) != cudaSuccess)
                return PS_ERR_CUDA;
        }
        for (cudaEvent_t *ev : {&d.k_fork, &d.k_chol, &d.k_zf})
            if (!*ev && cudaEventCreateWithFlags(ev, cudaEventDisableTiming) != cudaSuccess)
                return PS_ERR_CUDA;
        if (!d.early_fork &&
            cudaEventCreateWithFlags(&d.early_fork, cudaEventDisableTiming) != cudaSuccess)
            return PS_ERR_CUDA;
        if (!d.early_join &&
            cudaEventCreateWithFlags(&d.early_join, cudaEventDisableTiming) != cudaSuccess)
            return PS_ERR_CUDA;
        if (!d.early_lags &&
            cudaEventCreateWithFlags(&d.early_lags, cudaEventDisableTiming) != cudaSuccess)
            return PS_ERR_CUDA;
    }
    return PS_OK;
}

// The high-priority side stream and events of ps_pansharpen (after
// ensure_device with a capture stream).
struct Early {
    cudaStream_t s;
    cudaEvent_t fork, join, lags;
};
Early device_early() {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_mu);
    const DevState &d = g_dev[dev];
    return Early{d.early, d.early_fork, d.early_join, d.early_lags};
}

// The kernel estimate's second branch: its stream and events (after
// ensure_device with a capture stream).
struct KSide {
    cudaStream_t s;
    cudaEvent_t fork, chol, zf;
};
KSide device_kside() {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_mu);
    const DevState &d = g_dev[dev];
    return KSide{d.kside, d.k_fork, d.k_chol, d.k_zf};
}

// Branch streams and events of the current device (after ensure_device with
// a capture stream).
struct Branches {
    cudaStream_t s[4];
    cudaEvent_t fork, join[4];
};
Branches device_branches() {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_mu);
    const DevState &d = g_dev[dev];
    Branches b;
    for (int k = 0; k < 4; ++k) {
        b.s[k] = d.branch[k];
        b.join[k] = d.join[k];
    }
    b.fork = d.fork;
    return b;
}

// Branch split of N bands into `split` parts on band-pair boundaries:
// first band of part k (k <= split).
int split_begin(int N, int split, int k) {
    const int pairs = (N + 1) / 2;
    const int pb = (pairs * k) / split;
    return std::min(N, 2 * pb);
}

// ---------------------------------------------------------------------------
// CG loop as a CUDA graph: conditional WHILE nodes whose bodies hold a few
// iterations each (the direction p alternates between two buffers).
// Executable graphs are cached per argument set.
// ---------------------------------------------------------------------------
// The alternative priors' operator pieces: filters F_d (radius fR), the
// statistics of their guides F_d Y, four N x H x W scratch images, the FP64
// symbol sum_d |F_d^|^2 of the Z step.
struct PriorOps {
    int prior, nf, fR, r;
    int N, H, W, pad_;
    const float *filt[2];
    const float4 *gst4[2];
    float *t[4];
    double *tsym;
};

struct CgLoopArgs {
    int dev;
    int N, H, W, c, R, r;
    float lam;
    const float *u;
    const float4 *st4;
    float *x, *rv, *pA, *pB, *ap, *v;
    CgBand *bands;
    CgGlobal *g;
    int precond;  // 0 none, 1 the FFT preconditioner, 2 diagonal
    PrecArgs pa;  // z = P^{-1} r (pa.z and pa.r valid when precond)
    const float *sd;  // the diagonal s of P^{-1} (precond == 2)
    int split;    // 1, 2 or 4: parts of the bands run as parallel branches
    Tuning tune;  // launch choices (part of the graph cache key)
    int pad_;
    PriorOps po;  // po.prior != PS_PRIOR_LLP: the generic-filter loop
    bool operator==(const CgLoopArgs &o) const { return memcmp(this, &o, sizeof(*this)) == 0; }
};

// sum_d F_d^T W_d(F_d z) with W_d the matting matrix of guide d (gf = 0) or
// its guided filter (gf = 1): into t[3] (d = 0) and t[1] (d = 1).
void prior_terms(const PriorOps &o, const float *z, int gf, const CgBand *bands,
                 const CgGlobal *g, cudaStream_t st) {
    for (int d = 0; d < o.nf; ++d) {
        launch_db(z, nullptr, nullptr, nullptr, nullptr, 0, o.N, o.H, o.W, 1, o.filt[d], o.fR,
                  o.t[0], st);
        launch_prior_window(o.t[0], o.gst4[d], o.N, o.H, o.W, o.r, gf, o.t[1], o.t[2], o.t[0],
                            bands, g, st);
        launch_adj(o.t[0], o.N, o.H, o.W, 1, o.filt[d], o.fR, d == 0 ? o.t[3] : o.t[1], st);
    }
}

// One CG iteration under an alternative prior (all bands, one branch):
// p = r + beta p and v = D B p; q = lam sum_d F_d^T M_d F_d p with p^T q and
// alpha; x, r, beta and the stop test.
void enqueue_prior_iteration(const CgLoopArgs &a, const float *p_old, float *p_new,
                             cudaStream_t st) {
    const size_t HW = (size_t)a.H * a.W;
    launch_db(p_old, a.rv, p_new, a.bands, a.g, 1, a.N, a.H, a.W, a.c, a.u, a.R, a.v, st);
    prior_terms(a.po, p_new, 0, a.bands, a.g, st);
    launch_prior_combine(a.po.t[3], a.po.nf == 2 ? a.po.t[1] : nullptr, p_new, a.ap, a.N, HW,
                         a.lam, a.bands, a.g, st);
    launch_cg_update(a.x, a.rv, p_new, a.ap, a.v, a.u, a.R, a.c, a.N, a.H, a.W, a.bands, a.g,
                     st);
}

struct CgGraph {
    CgLoopArgs key;
    cudaGraphExec_t exec;
};
std::vector<CgGraph> g_graphs;

// One iteration's kernels for the bands [b0, b0 + n) (b0 even).
void enqueue_bands(const CgLoopArgs &a, int b0, int n, const float *p_old, float *p_new,
                   cudaStream_t st) {
    const size_t HW = (size_t)a.H * a.W, hw = HW / ((size_t)a.c * a.c);
    const size_t o = (size_t)b0 * HW;
    CgBand *bands = a.bands + b0;
    float *v = a.v + (size_t)b0 * hw;
    // p_new = (z or r) + beta p_old, formed inside the blur-decimate load
    launch_db(p_old + o, (a.precond ? a.pa.z : a.rv) + o, p_new + o, bands, a.g, 1, n, a.H, a.W,
              a.c, a.u, a.R, v, st, a.tune.db_impl);
    LlpArgs la = {};
    la.in = p_new + o;
    la.lr = v;
    la.st4 = a.st4;
    la.u = a.u;
    la.R = a.R;
    la.c = a.c;
    la.H = a.H;
    la.W = a.W;
    la.N = n;
    la.lam = a.lam;
    la.out = a.ap + o;
    la.bands = bands;
    la.g = a.g;
    la.cg = 1;
    la.ty = a.tune.llp_rows;
    la.pf = a.tune.llp_pf;
    la.nbd = a.tune.llp_bands;
    la.form = a.tune.llp_form;
    launch_llp_cgq2(la, a.r, n, st);
    launch_cg_update(a.x + o, a.rv + o, p_new + o, a.ap + o, v, a.u, a.R, a.c, n, a.H, a.W, bands,
                     a.g, st);
    if (a.precond == 2) {
        launch_diag_precond(a.rv + o, a.sd + o, a.pa.z + o, n, HW, bands, st);
    } else if (a.precond) {
        PrecArgs pa = a.pa;
        pa.r = a.rv + o;
        pa.z = a.pa.z + o;
        pa.spec = a.pa.spec + (size_t)(b0 / 2) * HW;
        pa.N = n;
        pa.bands = bands;
        pa.rows = a.tune.prec_rows;
        pa.impl = a.tune.prec_impl;
        launch_precond(pa, st);
    }
}

void enqueue_iteration(const CgLoopArgs &a, const float *p_old, float *p_new, int use_cond,
                       cudaGraphConditionalHandle h, cudaStream_t st) {
    if (a.po.prior != PS_PRIOR_LLP) {
        enqueue_prior_iteration(a, p_old, p_new, st);
    } else if (a.split > 1) {
        // parts of the bands as parallel branches, joined before the loop
        // control
        const Branches br = device_branches();
        cudaEventRecord(br.fork, st);
        for (int k = 0; k < a.split; ++k) {
            const int b0 = split_begin(a.N, a.split, k), b1 = split_begin(a.N, a.split, k + 1);
            cudaStreamWaitEvent(br.s[k], br.fork, 0);
            if (b1 > b0) enqueue_bands(a, b0, b1 - b0, p_old, p_new, br.s[k]);
            cudaEventRecord(br.join[k], br.s[k]);
        }
        for (int k = 0; k < a.split; ++k) cudaStreamWaitEvent(st, br.join[k], 0);
    } else {
        enqueue_bands(a, 0, a.N, p_old, p_new, st);
    }
    launch_cg_control(a.bands, a.g, a.N, use_cond, h, st);
}

// Iterations per body of a CG loop (even: the direction alternates between
// two buffers). Iterations after the stop inside a body launch and return at
// once.
constexpr int kBranchBodyIters = 4;

// One conditional WHILE node (its handle starts at 1; cg_control clears it
// once every band of [b0, b0 + n) has stopped) whose body, captured on
// `capture`, holds kBranchBodyIters iterations of those bands' kernels, with
// `g` as the loop's control record.
ps_status add_branch_loop(cudaGraph_t graph, const cudaGraphNode_t *deps, size_t ndeps,
                          const CgLoopArgs &a, int b0, int n, CgGlobal *g, cudaStream_t capture,
                          cudaGraphNode_t *node) {
    cudaGraphConditionalHandle handle;
    if (cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault) !=
        cudaSuccess)
        return PS_ERR_CUDA;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(node, graph, deps, nullptr, ndeps, &cp) != cudaSuccess)
        return PS_ERR_CUDA;
    if (cudaStreamBeginCaptureToGraph(capture, cp.conditional.phGraph_out[0], nullptr, nullptr,
                                      0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return PS_ERR_CUDA;
    CgLoopArgs ak = a;
    ak.g = g;
    ak.pa.g = g;
    for (int i = 0; i < kBranchBodyIters; i += 2) {
        enqueue_bands(ak, b0, n, a.pA, a.pB, capture);
        launch_cg_control(a.bands + b0, g, n, 1, handle, capture);
        enqueue_bands(ak, b0, n, a.pB, a.pA, capture);
        launch_cg_control(a.bands + b0, g, n, 1, handle, capture);
    }
    cudaGraph_t captured = nullptr;
    if (cudaStreamEndCapture(capture, &captured) != cudaSuccess) {
        cudaGetLastError();
        return PS_ERR_CUDA;
    }
    return PS_OK;
}

// Adds to `graph`, after `deps`, the CG loop of `a`. With the bands split
// into branches, each branch is a loop of its own (its own WHILE node and
// control record a.g + k, all copies of a.g made by the prelude), so that
// no branch waits for the others between iterations and a branch whose
// bands have stopped launches nothing more; an empty node joins them.
// Otherwise one WHILE node whose body, captured on `capture`, holds
// kBranchBodyIters iterations (its handle starts at 1, and cg_control clears
// it once every band has stopped).
ps_status add_cg_loop_node(cudaGraph_t graph, const cudaGraphNode_t *deps, size_t ndeps,
                           const CgLoopArgs &a, cudaStream_t capture, cudaGraphNode_t *node) {
    if (a.po.prior == PS_PRIOR_LLP && a.split > 1) {
        cudaGraphNode_t loops[kMaxSplit];
        int nl = 0;
        for (int k = 0; k < a.split; ++k) {
            const int b0 = split_begin(a.N, a.split, k), b1 = split_begin(a.N, a.split, k + 1);
            if (b1 <= b0) continue;
            const ps_status s =
                add_branch_loop(graph, deps, ndeps, a, b0, b1 - b0, a.g + k, capture, &loops[nl]);
            if (s != PS_OK) return s;
            ++nl;
        }
        if (cudaGraphAddEmptyNode(node, graph, loops, nl) != cudaSuccess) return PS_ERR_CUDA;
        return PS_OK;
    }
    cudaGraphConditionalHandle handle;
    if (cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault) !=
        cudaSuccess)
        return PS_ERR_CUDA;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(node, graph, deps, nullptr, ndeps, &cp) != cudaSuccess)
        return PS_ERR_CUDA;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(capture, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return PS_ERR_CUDA;
    for (int i = 0; i < kBranchBodyIters; i += 2) {
        enqueue_iteration(a, a.pA, a.pB, 1, handle, capture);
        enqueue_iteration(a, a.pB, a.pA, 1, handle, capture);
    }
    cudaGraph_t captured = nullptr;
    if (cudaStreamEndCapture(capture, &captured) != cudaSuccess) {
        cudaGetLastError();
        return PS_ERR_CUDA;
    }
    return PS_OK;
}

ps_status get_cg_graph(const CgLoopArgs &a, cudaStream_t capture, cudaGraphExec_t *out) {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (auto &e : g_graphs)
            if (e.key == a) {
                *out = e.exec;
                return PS_OK;
            }
    }
    cudaGraph_t graph = nullptr;
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) return PS_ERR_CUDA;
    cudaGraphNode_t node;
    ps_status s = add_cg_loop_node(graph, nullptr, 0, a, capture, &node);
    if (s != PS_OK) {
        cudaGraphDestroy(graph);
        return s;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return PS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_graphs.size() >= 16) {
        cudaGraphExecDestroy(g_graphs.front().exec);
        g_graphs.erase(g_graphs.begin());
    }
    g_graphs.push_back({a, exec});
    *out = exec;
    return PS_OK;
}

// ---------------------------------------------------------------------------
// Z step (Eq. Z_solution) on the FFT path, given Z0 in `z0`.
// ---------------------------------------------------------------------------
// Twiddles and the kernel spectrum B^ (FP64, transposed layout [kx][ky], and
// its FP32 rounding for the preconditioner), once per solve.
ps_status prepare_spectrum(const Ws &ws, const float *u, int H, int W, int R, cudaStream_t st) {
    double2 *bhat = ws.at<double2>(ws.L.bhat);
    float2 *twW32 = ws.at<float2>(ws.L.twW32), *twH32 = ws.at<float2>(ws.L.twH32);
    double2 *twW64 = ws.at<double2>(ws.L.twW64), *twH64 = ws.at<double2>(ws.L.twH64);
    launch_fft_twiddles(W, twW32, twW64, st);
    launch_fft_twiddles(H, twH32, twH64, st);
    launch_kernel_spectrum(u, R, H, W, twW64, twH64, bhat, st);
    launch_spectrum_to_f32(bhat, ws.at<float2>(ws.L.bh32), (size_t)H * W, st);
    return last_launch();
}

PrecArgs make_prec_args(const Ws &ws, const float *r, float *z, int N, int H, int W, int c,
                        float lam, CgBand *bands, const CgGlobal *g) {
    PrecArgs pa;
    memset(&pa, 0, sizeof(pa));
    pa.r = r;
    pa.z = z;
    pa.spec = ws.at<float2>(ws.L.spec);
    pa.bh = ws.at<float2>(ws.L.bh32);
    pa.twW = ws.at<float2>(ws.L.twW32);
    pa.twH = ws.at<float2>(ws.L.twH32);
    fft_make_plan(W, &pa.pw);
    fft_make_plan(H, &pa.ph);
    pa.N = N;
    pa.H = H;
    pa.W = W;
    pa.c = c;
    pa.lam = lam;
    pa.bands = bands;
    pa.g = g;
    return pa;
}

// ---------------------------------------------------------------------------
// Z step (Eq. Z_solution) on the FFT path, given Z0 in `z0` and the spectrum
// from prepare_spectrum.
// ---------------------------------------------------------------------------
ps_status run_zstep(const Ws &ws, const float *lrms, const float *z0, const float *u, int N,
                    int H, int W, int c, int R, int r, float lam_z, float *out,
                    cudaStream_t st, const PriorOps *po = nullptr, int fp32 = 0) {
    FftPlan pw, ph;
    if (!fft_make_plan(W, &pw) || !fft_make_plan(H, &ph)) return PS_ERR_UNSUPPORTED;
    const size_t HW = (size_t)H * W;
    if (fp32 && !(po && po->prior != PS_PRIOR_LLP) && precond_supported(H, W, c) &&
        aligned16(out)) {
        // all FP32: the right-hand side as real bands, then the
        // preconditioner's solve, whose operator B^T D^T D B + lam L^T L is
        // the Z step's at lam = lam'
        float *rhs = ws.at<float>(ws.L.z);
        LlpArgs la = {};
        la.in = z0;
        la.lr = lrms;
        la.st4 = ws.at<float4>(ws.L.st4);
        la.u = u;
        la.R = R;
        la.c = c;
        la.H = H;
        la.W = W;
        la.N = N;
        la.lam = lam_z;
        la.out = rhs;
        launch_llp(la, LLP_ZRHS, r, N, st);
        PrecArgs pa = make_prec_args(ws, rhs, out, N, H, W, c, lam_z, nullptr, nullptr);
        launch_precond(pa, st);
        return last_launch();
    }
    const int nimg = (N + 1) / 2;
    double2 *cbuf64 = ws.at<double2>(ws.L.r);
    double2 *ctmp64 = ws.at<double2>(ws.L.pB);
    float2 *sol32 = ws.at<float2>(ws.L.r);     // reuses cbuf64 once it is consumed
    float2 *ctmp32 = ws.at<float2>(ws.L.pB);   // reuses ctmp64 once it is consumed
    double2 *bhat = ws.at<double2>(ws.L.bhat);
    float2 *twW32 = ws.at<float2>(ws.L.twW32), *twH32 = ws.at<float2>(ws.L.twH32);
    double2 *twW64 = ws.at<double2>(ws.L.twW64), *twH64 = ws.at<double2>(ws.L.twH64);
    const double *tsym = nullptr;
    if (po && po->prior != PS_PRIOR_LLP) {
        // B^T D^T X + lam' sum_d F_d^T L-hat_d, L-hat_d the guided filter of
        // F_d Z0 with guide F_d Y; the symbol sum_d |F_d^|^2 replaces S^2
        prior_terms(*po, z0, 1, nullptr, nullptr, st);
        if (po->nf == 2)
            launch_prior_combine(po->t[3], po->t[1], nullptr, po->t[3], N, HW, 1.0f, nullptr,
                                 nullptr, st);
        launch_adj(lrms, N, H, W, c, u, R, po->t[0], st);
        launch_prior_pack(po->t[0], po->t[3], lam_z, N, HW, cbuf64, st);
        tsym = po->tsym;
    } else {
        // right-hand side B^T D^T X + lam' L L-hat, packed two bands per image
        LlpArgs la = {};
        la.in = z0;
        la.lr = lrms;
        la.st4 = ws.at<float4>(ws.L.st4);
        la.u = u;
        la.R = R;
        la.c = c;
        la.H = H;
        la.W = W;
        la.N = N;
        la.lam = lam_z;
        la.cout = cbuf64;
        launch_llp(la, LLP_ZRHS, r, N, st);
    }
    // forward 2-D FFT (FP64), group solve, inverse 2-D FFT (FP32)
    launch_fft_rows64(cbuf64, pw, nimg * H, twW64, st);
    launch_transpose64(cbuf64, ctmp64, H, W, nimg, st);
    launch_fft_rows64(ctmp64, ph, nimg * W, twH64, st);
    launch_alias_solve(ctmp64, bhat, sol32, nimg, H, W, c, lam_z, st, tsym);
    launch_fft_rows32(sol32, ph, nimg * W, twH32, 1, nullptr, N, HW, st);
    launch_transpose32(sol32, ctmp32, W, H, nimg, st);
    launch_fft_rows32(ctmp32, pw, nimg * H, twW32, 1, out, N, HW, st);
    return last_launch();
}

// ---------------------------------------------------------------------------
// Stages of ps_solve_hrms, shared with the batched entry point: everything
// before the CG loop (PAN statistics, spectra, right-hand side, start point,
// CG state), and the Z step after it. Neither synchronises, so both can be
// captured into a graph.
// ---------------------------------------------------------------------------
struct SolveCall {
    Ws ws;
    size_t ws_bytes;
    size_t prior_off;  // start of the alternative prior's scratch (prior != LLP)
    const float *lrms, *pan, *u, *z_init;
    float *hrms, *z0;
    int N, H, W, c, R;
    ps_hrms_params p;
    int early;  // 1: solve_early has run (PAN statistics, warm start)
};

// The network's forward pass with `reserve` SMs left out of its persistent
// convolution grids (so that latency-bound work on another stream finds
// whole SMs free); defined with the network's other entry points.
ps_status cnn_forward_reserve(const float *d_params, const float *d_up, const float *d_pan,
                              size_t pan_stride, int B, int H, int W, float *d_z, void *d_ws,
                              size_t ws_bytes, int reserve, void *stream);

ps_status estimate_kernel_impl(const float *d_lrms, const float *d_pan, int N, int H, int W,
                               int ratio, int R, const ps_kernel_params *p,
                               const float *d_omega_in, float *d_kernel, float *d_omega_out,
                               ps_kernel_info *h_info, void *d_ws, size_t ws_bytes,
                               cudaStream_t st, cudaEvent_t lags_done);

// Scratch of an alternative prior, after the base layout (and after the
// network's workspace when that is used): four N x H x W images, the
// statistics of two guides, one FP64 spectrum, the FP64 symbol, two filters.
size_t prior_bytes(int N, int H, int W) {
    const size_t HW = (size_t)H * W;
    return 4 * align_up((size_t)N * HW * 4) + 3 * align_up(HW * 16) + align_up(HW * 8) +
           2 * align_up((size_t)kMaxTaps * 4);
}

// Whether a solve with parameters p may run a network (the warm start or the
// diagonal), which then takes its workspace at Layout::cnn.
bool runs_network(const ps_hrms_params *p) {
    return p && (p->warm == 2 || (p->precond == 2 && !p->precond_diag));
}

size_t prior_offset(const Layout &L, int N, int H, int W, const ps_hrms_params *p) {
    return align_up(L.cnn + (runs_network(p) ? ps_cnn_workspace_size(N, H, W, 0) : 0));
}

// The prior's operator pieces over the scratch at `off` (pointers only).
PriorOps prior_ops(const Ws &ws, size_t off, int prior, int N, int H, int W, int R, int r) {
    PriorOps o;
    memset(&o, 0, sizeof(o));
    o.prior = prior;
    o.nf = prior_filter_count(prior);
    o.fR = prior_filter_radius(prior, R);
    o.r = r;
    o.N = N;
    o.H = H;
    o.W = W;
    const size_t HW = (size_t)H * W;
    size_t at = off;
    for (int k = 0; k < 4; ++k) {
        o.t[k] = ws.at<float>(at);
        at += align_up((size_t)N * HW * 4);
    }
    float4 *g0 = ws.at<float4>(at);
    at += align_up(HW * 16);
    float4 *g1 = ws.at<float4>(at);
    at += align_up(HW * 16);
    o.gst4[0] = g0;
    o.gst4[1] = g1;
    at += align_up(HW * 16);  // FP64 filter spectrum (prior_fhat)
    o.tsym = ws.at<double>(at);
    at += align_up(HW * 8);
    o.filt[0] = ws.at<float>(at);
    at += align_up((size_t)kMaxTaps * 4);
    o.filt[1] = ws.at<float>(at);
    return o;
}

double2 *prior_fhat(const Ws &ws, size_t off, int N, int H, int W) {
    const size_t HW = (size_t)H * W;
    return ws.at<double2>(off + 4 * align_up((size_t)N * HW * 4) + 2 * align_up(HW * 16));
}

ps_status make_solve_call(const float *d_lrms, const float *d_pan, const float *d_kernel, int N,
                          int H, int W, int ratio, int R, const ps_hrms_params *p,
                          const float *d_z_init, float *d_hrms, float *d_z0, void *d_ws,
                          size_t ws_bytes, SolveCall *sc) {
    ps_status s;
    if ((s = check_dims(N, H, W, ratio, R)) != PS_OK) return s;
    if ((s = check_fft_dims(H, W)) != PS_OK) return s;
    if ((s = check_hrms(p)) != PS_OK) return s;
    if (p->precond == 1 && !precond_supported(H, W, ratio)) return PS_ERR_UNSUPPORTED;
    if (!d_lrms || !d_pan || !d_kernel || !d_hrms) return PS_ERR_INVALID_ARG;
    if ((d_z0 && !aligned16(d_z0)) || (d_z_init && !aligned16(d_z_init)))
        return PS_ERR_INVALID_ARG;
    if (p->precond == 2 && p->precond_diag && !aligned16(p->precond_diag))
        return PS_ERR_INVALID_ARG;
    if ((s = bind_ws(d_ws, ws_bytes, N, H, W, ratio, R, &sc->ws)) != PS_OK) return s;
    const bool net = (p->warm == 2 && !d_z_init) || (p->precond == 2 && !p->precond_diag);
    if (net && ws_bytes < sc->ws.L.cnn + ps_cnn_workspace_size(N, H, W, 0))
        return PS_ERR_WORKSPACE;
    sc->prior_off = 0;
    if (p->prior != PS_PRIOR_LLP) {
        sc->prior_off = prior_offset(sc->ws.L, N, H, W, p);
        if (ws_bytes < sc->prior_off + prior_bytes(N, H, W)) return PS_ERR_WORKSPACE;
    }
    sc->ws_bytes = ws_bytes;
    sc->early = 0;
    sc->lrms = d_lrms;
    sc->pan = d_pan;
    sc->u = d_kernel;
    sc->z_init = d_z_init;
    sc->hrms = d_hrms;
    sc->z0 = d_z0;
    sc->N = N;
    sc->H = H;
    sc->W = W;
    sc->c = ratio;
    sc->R = R;
    sc->p = *p;
    return PS_OK;
}

// The steps of the solve that do not read the blur kernel: the PAN window
// statistics of the LLP prior and the warm start (bicubic, and the network on
// it). ps_pansharpen runs them while the kernel is estimated on another
// stream, leaving `reserve` SMs out of the network's persistent grids; the
// network waits for `before_net` (when given), the statistics and bicubic
// do not.
ps_status solve_early(const SolveCall &sc, cudaStream_t st, int reserve,
                      cudaEvent_t before_net = nullptr) {
    const Ws &ws = sc.ws;
    const ps_hrms_params *p = &sc.p;
    const int N = sc.N, H = sc.H, W = sc.W, c = sc.c;
    float *x = sc.z0 ? sc.z0 : ws.at<float>(ws.L.xbuf);
    if (p->prior == PS_PRIOR_LLP)
        launch_pan_stats(sc.pan, H, W, p->r, p->eps, nullptr, nullptr, nullptr,
                         ws.at<float4>(ws.L.st4), st);
    if (!sc.z_init && p->warm >= 1) {
        launch_bicubic_up(sc.lrms, N, H / c, W / c, c, x, st);
        if (p->warm == 2) {
            if (before_net && cudaStreamWaitEvent(st, before_net, 0) != cudaSuccess)
                return PS_ERR_CUDA;
            ps_status s = cnn_forward_reserve(p->cnn_params, x, sc.pan, 0, N, H, W, x,
                                              ws.base + ws.L.cnn, sc.ws_bytes - ws.L.cnn,
                                              reserve, st);
            if (s != PS_OK) return s;
        }
    }
    return last_launch();
}

ps_status solve_prelude(const SolveCall &sc, cudaStream_t st, CgLoopArgs *a) {
    ps_status s;
    const Ws &ws = sc.ws;
    const ps_hrms_params *p = &sc.p;
    const int N = sc.N, H = sc.H, W = sc.W, c = sc.c, R = sc.R;
    const float *d_kernel = sc.u, *d_lrms = sc.lrms, *d_z_init = sc.z_init;
    const size_t HW = (size_t)H * W;
    float4 *st4 = ws.at<float4>(ws.L.st4);
    float *x = sc.z0 ? sc.z0 : ws.at<float>(ws.L.xbuf);
    float *rv = ws.at<float>(ws.L.r), *ap = ws.at<float>(ws.L.ap), *v = ws.at<float>(ws.L.v);
    CgBand *bands = ws.at<CgBand>(ws.L.bands);
    CgGlobal *g = ws.at<CgGlobal>(ws.L.glob);

    PriorOps po;
    memset(&po, 0, sizeof(po));
    if (p->prior == PS_PRIOR_LLP) {
        if (!sc.early) launch_pan_stats(sc.pan, H, W, p->r, p->eps, nullptr, nullptr, nullptr,
                                        st4, st);
    } else {
        po = prior_ops(ws, sc.prior_off, p->prior, N, H, W, R, p->r);
        launch_prior_filters(d_kernel, R, p->prior, const_cast<float *>(po.filt[0]),
                             const_cast<float *>(po.filt[1]), st);
        // the guides F_d Y and their window statistics
        for (int d = 0; d < po.nf; ++d) {
            launch_db(sc.pan, nullptr, nullptr, nullptr, nullptr, 0, 1, H, W, 1, po.filt[d],
                      po.fR, po.t[0], st);
            launch_guide_stats(po.t[0], H, W, p->r, p->eps, const_cast<float4 *>(po.gst4[d]),
                               st);
        }
    }
    // With the LLP prior, the kernel spectrum and b = B^T D^T X (disjoint
    // buffers) go on a side stream while A z_init is formed here; cg_init
    // waits for both.
    const bool side = p->prior == PS_PRIOR_LLP;
    const KSide k2 = device_kside();
    if (side) {
        if (cudaEventRecord(k2.fork, st) != cudaSuccess ||
            cudaStreamWaitEvent(k2.s, k2.fork, 0) != cudaSuccess)
            return PS_ERR_CUDA;
        if ((s = prepare_spectrum(ws, d_kernel, H, W, R, k2.s)) != PS_OK) return s;
        launch_adj(d_lrms, N, H, W, c, d_kernel, R, rv, k2.s);  // b = B^T D^T X
        if (cudaEventRecord(k2.zf, k2.s) != cudaSuccess) return PS_ERR_CUDA;
    } else if ((s = prepare_spectrum(ws, d_kernel, H, W, R, st)) != PS_OK) {
        return s;
    }
    if (p->prior != PS_PRIOR_LLP) {
        // the Z step's symbol sum_d |F_d^|^2
        double2 *fh = prior_fhat(ws, sc.prior_off, N, H, W);
        for (int d = 0; d < po.nf; ++d) {
            launch_kernel_spectrum(po.filt[d], po.fR, H, W, ws.at<double2>(ws.L.twW64),
                                   ws.at<double2>(ws.L.twH64), fh, st);
            launch_symbol_add(fh, po.tsym, HW, d == 0, st);
        }
    }
    const float *sd = nullptr;
    if (p->precond == 2 && p->precond_diag) {
        sd = p->precond_diag;
    } else if (p->precond == 2) {
        // the diagonal network on (bicubic, PAN): its output in z (free
        // until the first preconditioner application), the bicubic and then
        // s = max((net - bicubic) / 255, 1/64) in the unused spectrum buffer
        float *s_buf = ws.at<float>(ws.L.spec);
        float *net_out = ws.at<float>(ws.L.z);
        launch_bicubic_up(d_lrms, N, H / c, W / c, c, s_buf, st);
        if ((s = ps_cnn_forward(p->diag_params, s_buf, sc.pan, 0, N, H, W, net_out,
                                ws.base + ws.L.cnn, sc.ws_bytes - ws.L.cnn, st)) != PS_OK)
            return s;
        launch_diag_head(net_out, s_buf, (size_t)N * HW, 1.0f / 64.0f, st);
        sd = s_buf;
    } else if (p->precond == 3) {
        // Jacobi: s = 1 / diag(A), one copy per band, in the unused spectrum
        // buffer; the loop then runs the diagonal preconditioner
        float *s_buf = ws.at<float>(ws.L.spec);
        launch_jacobi_diag(st4, d_kernel, R, c, H, W, p->r, p->lambda, N, 1, s_buf, st);
        sd = s_buf;
    }
    if (!side) launch_adj(d_lrms, N, H, W, c, d_kernel, R, rv, st);  // b = B^T D^T X
    if (!d_z_init && p->warm >= 1 && !sc.early) {
        // bicubic start point, written where the iterate lives
        launch_bicubic_up(d_lrms, N, H / c, W / c, c, x, st);
        if (p->warm == 2) {
            // the network on (bicubic, PAN), in place: its last layer reads
            // the bicubic value of a pixel and writes the result there
            if ((s = ps_cnn_forward(p->cnn_params, x, sc.pan, 0, N, H, W, x,
                                    ws.base + ws.L.cnn, sc.ws_bytes - ws.L.cnn, st)) != PS_OK)
                return s;
        }
    }
    if (!d_z_init && p->warm >= 1) {
        d_z_init = x;
    }
    if (d_z_init && p->prior != PS_PRIOR_LLP) {
        // A z_init = B^T D^T D B z_init + lam sum_d F_d^T M_d F_d z_init
        launch_db(d_z_init, nullptr, nullptr, nullptr, nullptr, 0, N, H, W, c, d_kernel, R, v,
                  st);
        prior_terms(po, d_z_init, 0, nullptr, nullptr, st);
        launch_prior_combine(po.t[3], po.nf == 2 ? po.t[1] : nullptr, nullptr, ap, N, HW,
                             p->lambda, nullptr, nullptr, st);
        launch_adj(v, N, H, W, c, d_kernel, R, po.t[0], st);
        launch_prior_combine(ap, po.t[0], nullptr, ap, N, HW, 1.0f, nullptr, nullptr, st);
    } else if (d_z_init) {
        launch_db(d_z_init, nullptr, nullptr, nullptr, nullptr, 0, N, H, W, c, d_kernel, R, v,
                  st);
        LlpArgs la = {};
        la.in = d_z_init;
        la.lr = v;
        la.st4 = st4;
        la.u = d_kernel;
        la.R = R;
        la.c = c;
        la.H = H;
        la.W = W;
        la.N = N;
        la.lam = p->lambda;
        la.out = ap;
        launch_llp(la, LLP_APPLY, p->r, N, st);
    }
    if (side && cudaStreamWaitEvent(st, k2.zf, 0) != cudaSuccess) return PS_ERR_CUDA;
    launch_cg_reset(bands, g, N, (double)p->tol, p->max_iter, p->precond, p->stop_rule, st);
    launch_cg_init(rv, d_z_init ? ap : nullptr, d_z_init, x, rv, N, HW, bands, g, st);
    PrecArgs pa;
    memset(&pa, 0, sizeof(pa));
    if (p->precond == 2 || p->precond == 3) {
        // z0 = s r0, rho = r0^T z0
        pa.r = rv;
        pa.z = ws.at<float>(ws.L.z);
        launch_diag_precond(rv, sd, pa.z, N, HW, bands, st);
    } else if (p->precond) {
        // z0 = P^{-1} r0, rho = r0^T z0 (the first direction is p = z0)
        pa = make_prec_args(ws, rv, ws.at<float>(ws.L.z), N, H, W, c,
                            p->lambda * p->precond_gamma, bands, g);
        launch_precond(pa, st);
    }
    if ((s = last_launch()) != PS_OK) return s;

    memset(a, 0, sizeof(*a));
    cudaGetDevice(&a->dev);
    a->N = N; a->H = H; a->W = W; a->c = c; a->R = R; a->r = p->r; a->lam = p->lambda;
    a->u = d_kernel; a->st4 = st4;
    a->x = x; a->rv = rv; a->pA = ws.at<float>(ws.L.pA); a->pB = ws.at<float>(ws.L.pB);
    a->ap = ap; a->v = v;
    a->bands = bands; a->g = g;
    a->precond = p->precond == 3 ? 2 : p->precond;  // Jacobi runs the diagonal loop
    a->pa = pa;
    a->sd = sd;
    a->tune = tuning_get(a->dev, N, H, W, c, p->r);
    a->split = a->tune.split ? a->tune.split : ((N >= 4) ? 2 : 1);
    a->po = po;
    return PS_OK;
}

ps_status solve_epilogue(const SolveCall &sc, const CgLoopArgs &a, cudaStream_t st) {
    const ps_hrms_params *p = &sc.p;
    const float lam_z =
        p->lambda * (p->exact_weight ? (float)((2 * p->r + 1) * (2 * p->r + 1)) : 1.0f);
    const ps_status s = run_zstep(sc.ws, sc.lrms, a.x, sc.u, sc.N, sc.H, sc.W, sc.c, sc.R,
                                  p->r, lam_z, sc.hrms, st, &a.po, p->zstep_fp32);
    if (s == PS_OK) launch_collect_status(a.bands, sc.N, nullptr, st);
    return s;
}

// Per-band CG results (after the work that wrote them has finished).
ps_status read_band_info(const CgBand *d_bands, int N, ps_band_info *h_info) {
    std::vector<CgBand> hb(N);
    if (cudaMemcpy(hb.data(), d_bands, N * sizeof(CgBand), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return PS_ERR_CUDA;
    for (int b = 0; b < N; ++b) {
        h_info[b].status = hb[b].status;
        h_info[b].iters = hb[b].iters;
        h_info[b].rel_residual = hb[b].bb > 0.0 ? sqrt(hb[b].rr / hb[b].bb) : 0.0;
        h_info[b].ms = hb[b].t_done > hb[b].t_start
                           ? (float)((double)(hb[b].t_done - hb[b].t_start) * 1e-6)
                           : 0.0f;
    }
    return PS_OK;
}

// ---------------------------------------------------------------------------
// Batched scenes: one executable graph holds every scene of the batch. Each
// scene is an independent branch: its prelude (kernel estimate when asked,
// then the stages before the CG loop), its CG loop as a conditional WHILE
// node of its own, and its Z step. The branches are added largest scene
// first. A timer stamp opens the graph and closes every scene.
// ---------------------------------------------------------------------------
constexpr int kMaxBatch = 4096;

size_t batch_header_bytes(int count) { return align_up((size_t)(count + 1) * 8); }

size_t scene_ws_bytes(const ps_scene &q, const ps_hrms_params *hp) {
    return align_up(ps_workspace_size(q.N, q.H, q.W, q.ratio, q.R, hp));
}

struct BatchGraph {
    std::vector<char> key;
    cudaGraphExec_t exec;
};
std::vector<BatchGraph> g_batch;

template <class T>
void key_put(std::vector<char> &k, const T &v) {
    const char *b = reinterpret_cast<const char *>(&v);
    k.insert(k.end(), b, b + sizeof(T));
}

// Captures what `enqueue` launches on `capture` and adds it to `graph` as a
// child-graph node after `deps`.
template <class F>
ps_status capture_child(cudaGraph_t graph, const cudaGraphNode_t *deps, size_t ndeps,
                        cudaStream_t capture, F &&enqueue, cudaGraphNode_t *node) {
    if (cudaStreamBeginCapture(capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return PS_ERR_CUDA;
    ps_status s = enqueue(capture);
    cudaGraph_t child = nullptr;
    const cudaError_t e = cudaStreamEndCapture(capture, &child);
    if (s == PS_OK && e != cudaSuccess) s = PS_ERR_CUDA;
    if (s == PS_OK && cudaGraphAddChildGraphNode(node, graph, deps, ndeps, child) != cudaSuccess)
        s = PS_ERR_CUDA;
    if (child) cudaGraphDestroy(child);
    if (s != PS_OK) cudaGetLastError();
    return s;
}

ps_status build_batch_graph(const ps_scene *scenes, int count, const ps_kernel_params *kp,
                            const std::vector<SolveCall> &calls, unsigned long long *stamps,
                            cudaStream_t capture, cudaGraphExec_t *out) {
    cudaGraph_t graph = nullptr;
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) return PS_ERR_CUDA;
    ps_status s;
    cudaGraphNode_t root;
    s = capture_child(graph, nullptr, 0, capture,
                      [&](cudaStream_t st) {
                          launch_stamp(stamps, st);
                          return last_launch();
                      },
                      &root);
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const ps_scene &a = scenes[x], &b = scenes[y];
        return (double)a.N * a.H * a.W > (double)b.N * b.H * b.W;
    });
    for (int k = 0; k < count && s == PS_OK; ++k) {
        const int i = order[k];
        const ps_scene &q = scenes[i];
        const SolveCall &sc = calls[i];
        CgLoopArgs a;
        cudaGraphNode_t pre, loop, post;
        s = capture_child(graph, &root, 1, capture,
                          [&](cudaStream_t st) {
                              ps_status e = PS_OK;
                              // the scene's inputs from page-locked host memory
                              const size_t nl = (size_t)q.N * (q.H / q.ratio) * (q.W / q.ratio);
                              if (q.h_lrms &&
                                  cudaMemcpyAsync(const_cast<float *>(q.lrms), q.h_lrms,
                                                  nl * sizeof(float), cudaMemcpyHostToDevice,
                                                  st) != cudaSuccess)
                                  e = PS_ERR_CUDA;
                              if (e == PS_OK && q.h_pan &&
                                  cudaMemcpyAsync(const_cast<float *>(q.pan), q.h_pan,
                                                  (size_t)q.H * q.W * sizeof(float),
                                                  cudaMemcpyHostToDevice, st) != cudaSuccess)
                                  e = PS_ERR_CUDA;
                              if (e == PS_OK && kp) {
                                  // this scene's X' (Eq. objective1)
                                  ps_kernel_params kq = *kp;
                                  if (q.band_mask) kq.band_mask = q.band_mask;
                                  e = ps_estimate_kernel(q.lrms, q.pan, q.N, q.H, q.W, q.ratio,
                                                         q.R, &kq, nullptr, q.kernel, nullptr,
                                                         nullptr, sc.ws.base, sc.ws_bytes, st);
                              }
                              if (e == PS_OK) e = solve_prelude(sc, st, &a);
                              return e;
                          },
                          &pre);
        if (s == PS_OK) {
            // concurrency comes from the scenes: one branch per iteration
            a.split = 1;
            s = add_cg_loop_node(graph, &pre, 1, a, capture, &loop);
        }
        if (s == PS_OK)
            s = capture_child(graph, &loop, 1, capture,
                              [&](cudaStream_t st) {
                                  ps_status e = solve_epilogue(sc, a, st);
                                  launch_stamp(stamps + 1 + i, st);
                                  if (e == PS_OK) e = last_launch();
                                  // the HRMS back to page-locked host memory
                                  if (e == PS_OK && q.h_hrms &&
                                      cudaMemcpyAsync(q.h_hrms, q.hrms,
                                                      (size_t)q.N * q.H * q.W * sizeof(float),
                                                      cudaMemcpyDeviceToHost,
                                                      st) != cudaSuccess)
                                      e = PS_ERR_CUDA;
                                  return e;
                              },
                              &post);
    }
    if (s == PS_OK && cudaGraphInstantiate(out, graph, 0) != cudaSuccess) s = PS_ERR_CUDA;
    cudaGraphDestroy(graph);
    return s;
}

// Algorithm 2 on a prepared call: prelude, the CG loop (graph or host
// launched), the guided filter and Z step; per-band results into h_info.
ps_status run_solve(const SolveCall &sc, cudaStream_t st, ps_band_info *h_info) {
    ps_status s;
    const ps_hrms_params *p = &sc.p;
    cudaStream_t capture = nullptr;
    if ((s = ensure_device(&capture)) != PS_OK) return s;
    CgLoopArgs a;
    if ((s = solve_prelude(sc, st, &a)) != PS_OK) return s;
    if (p->host_loop) {
        // same kernels, launched by the host; the stop flag is read every 8
        // iterations, and the loop is bounded by max_iter whatever it says
        int stop = 0;
        for (int it = 0; it < p->max_iter + 2 && !stop; it += 2) {
            enqueue_iteration(a, a.pA, a.pB, 0, 0, st);
            enqueue_iteration(a, a.pB, a.pA, 0, 0, st);
            if ((it & 7) == 6 || it + 2 >= p->max_iter + 2) {
                if (cudaMemcpyAsync(&stop, &a.g->stop, sizeof(int), cudaMemcpyDeviceToHost,
                                    st) != cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess)
                    return PS_ERR_CUDA;
            }
        }
        if ((s = last_launch()) != PS_OK) return s;
    } else {
        cudaGraphExec_t exec;
        if ((s = get_cg_graph(a, capture, &exec)) != PS_OK) return s;
        if (cudaGraphLaunch(exec, st) != cudaSuccess) return PS_ERR_CUDA;
    }
    if ((s = solve_epilogue(sc, a, st)) != PS_OK) return s;
    if (h_info) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return PS_ERR_CUDA;
        if ((s = read_band_info(a.bands, sc.N, h_info)) != PS_OK) return s;
    }
    return PS_OK;
}

}  // namespace

// ===========================================================================
// Public entry points
// ===========================================================================
extern "C" {

void ps_default_kernel_params(ps_kernel_params *p) {
    if (!p) return;
    p->lambda_omega = 10.0f;
    p->l = 2;
    p->alpha1 = 1.0f;
    p->alpha2 = 0.006f;
    p->mu1 = p->mu2 = p->mu3 = 100.0f;
    p->rho = 0.5f;
    p->t_max = 10000;
    p->th = 1e-5f;
    p->band_mask = 0ull;
}

void ps_default_hrms_params(ps_hrms_params *p) {
    if (!p) return;
    p->lambda = 2e-4f;
    p->r = 1;
    p->eps = 1.0f;
    p->tol = 1e-6f;
    p->max_iter = 5000;
    p->exact_weight = 0;
    p->host_loop = 0;
    p->precond = 1;
    p->precond_gamma = 4.0f;
    p->warm = 0;
    p->cnn_params = nullptr;
    p->stop_rule = 0;
    p->zstep_fp32 = 0;
    p->prior = PS_PRIOR_LLP;
    p->precond_diag = nullptr;
    p->diag_params = nullptr;
}

const char *ps_status_string(int s) {
    switch (s) {
        case PS_OK: return "ok";
        case PS_ERR_INVALID_ARG: return "invalid argument";
        case PS_ERR_SHAPE: return "inconsistent shapes";
        case PS_ERR_CUDA: return "CUDA runtime error";
        case PS_ERR_WORKSPACE: return "workspace too small or misaligned";
        case PS_ERR_NOT_CONVERGED: return "iteration cap reached";
        case PS_ERR_NONFINITE: return "non-finite value in a reduction";
        case PS_ERR_BREAKDOWN: return "CG breakdown (p^T A p <= 0)";
        case PS_ERR_UNSUPPORTED: return "size not supported";
        case PS_ERR_TIMEOUT: return "a bounded device-side wait gave up";
        default: return "unknown status";
    }
}

ps_status ps_sync_status(void *stream) {
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return PS_ERR_CUDA;
    int h = 0;
    const int zero = 0;
    if (cudaMemcpyFromSymbol(&h, g_sticky_status, sizeof(int)) != cudaSuccess ||
        cudaMemcpyToSymbol(g_sticky_status, &zero, sizeof(int)) != cudaSuccess)
        return PS_ERR_CUDA;
    return (ps_status)h;
}

size_t ps_workspace_size(int N, int H, int W, int ratio, int R, const ps_hrms_params *hp) {
    if (check_dims(N, H, W, ratio, R) != PS_OK) return 0;
    Layout L;
    if (!make_layout(N, H, W, ratio, R, &L)) return 0;
    if (hp && hp->prior != PS_PRIOR_LLP)
        return prior_offset(L, N, H, W, hp) + prior_bytes(N, H, W) + kAlign;
    if (runs_network(hp)) return L.total + ps_cnn_workspace_size(N, H, W, 0);
    return L.total;
}

size_t ps_op_workspace_size(int N, int H, int W, int ratio, int R) {
    return ps_workspace_size(N, H, W, ratio, R, nullptr);
}

ps_status ps_estimate_kernel(const float *d_lrms, const float *d_pan, int N, int H, int W,
                             int ratio, int R, const ps_kernel_params *p,
                             const float *d_omega_in, float *d_kernel, float *d_omega_out,
                             ps_kernel_info *h_info, void *d_ws, size_t ws_bytes,
                             void *stream) {
    return estimate_kernel_impl(d_lrms, d_pan, N, H, W, ratio, R, p, d_omega_in, d_kernel,
                                d_omega_out, h_info, d_ws, ws_bytes, (cudaStream_t)stream,
                                nullptr);
}

}  // extern "C"

namespace {

// The ADMM's iteration count, status and last relative change, after the
// work queued on `st` (synchronises it).
ps_status read_kernel_info(const Ws &ws, cudaStream_t st, ps_kernel_info *h_info) {
    const int *ki = ws.at<int>(ws.L.kinfo);
    int hi[2];
    double ch = 0.0;
    if (cudaMemcpyAsync(hi, ki, sizeof(hi), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&ch, ki + 2, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PS_ERR_CUDA;
    h_info->iters = hi[0];
    h_info->status = hi[1];
    h_info->last_change = ch;
    return PS_OK;
}

// Algorithm 1. `lags_done`, when given, is recorded on `st` once the lag
// correlations behind E^T E (the estimate's one kernel that fills the GPU)
// are queued.
ps_status estimate_kernel_impl(const float *d_lrms, const float *d_pan, int N, int H, int W,
                               int ratio, int R, const ps_kernel_params *p,
                               const float *d_omega_in, float *d_kernel, float *d_omega_out,
                               ps_kernel_info *h_info, void *d_ws, size_t ws_bytes,
                               cudaStream_t st, cudaEvent_t lags_done) {
    ps_status s;
    if ((s = check_dims(N, H, W, ratio, R)) != PS_OK) return s;
    if ((s = check_kernel_params(p)) != PS_OK) return s;
    if ((s = check_band_mask(p->band_mask, N)) != PS_OK) return s;
    if (!d_lrms || !d_pan || !d_kernel) return PS_ERR_INVALID_ARG;
    Ws ws;
    if ((s = bind_ws(d_ws, ws_bytes, N, H, W, ratio, R, &ws)) != PS_OK) return s;
    cudaStream_t capture = nullptr;
    if ((s = ensure_device(&capture)) != PS_OK) return s;
    const int c = ratio, h = H / c, w = W / c, hw = h * w;
    const int nt = (2 * R + 1) * (2 * R + 1);
    float *omega = d_omega_out ? d_omega_out : ws.at<float>(ws.L.omega);
    double *ete = ws.at<double>(ws.L.ete);
    // Two branches, on disjoint parts of the workspace: E^T E and its
    // factor, then Q = mu3 (E^T E + mu3 I)^-1, on `st`; omega, f and E^T f,
    // then z_f (once the factor exists), on the side stream. ADMM waits for
    // both.
    const KSide k2 = device_kside();
    if (cudaEventRecord(k2.fork, st) != cudaSuccess ||
        cudaStreamWaitEvent(k2.s, k2.fork, 0) != cudaSuccess)
        return PS_ERR_CUDA;
    // omega over the bands X' of Eq. objective1 (zeros for the others), so
    // that f = X omega below is X' omega
    if (d_omega_in) {
        launch_omega_mask(d_omega_in, p->band_mask, N, omega, k2.s);
    } else {
        const BandSel sel = band_sel(p->band_mask, N);
        float *Aw = ws.at<float>(ws.L.v);
        launch_box_lr(d_lrms, sel, h, w, p->l, Aw, k2.s);
        launch_box_hr_dec(d_pan, H, W, c, c * p->l, ws.at<float>(ws.L.bvec), k2.s);
        launch_omega_normal(Aw, ws.at<float>(ws.L.bvec), sel.n, hw, ws.at<double>(ws.L.G),
                            k2.s);
        launch_omega_solve(ws.at<double>(ws.L.G), sel, N, p->lambda_omega, omega, k2.s);
    }
    float *f = ws.at<float>(ws.L.f);
    launch_combine_f(d_lrms, omega, N, hw, f, k2.s);
    launch_etf(d_pan, H, W, c, R, f, ws.at<double>(ws.L.etf), k2.s);
    launch_ete_lags(d_pan, H, W, c, R, ws.at<double>(ws.L.lags), st);
    if (lags_done && cudaEventRecord(lags_done, st) != cudaSuccess) return PS_ERR_CUDA;
    launch_ete_assemble(ws.at<double>(ws.L.lags), c, R, ete, st);
    launch_cholesky(ete, nt, p->mu3, st);
    if (cudaEventRecord(k2.chol, st) != cudaSuccess ||
        cudaStreamWaitEvent(k2.s, k2.chol, 0) != cudaSuccess)
        return PS_ERR_CUDA;
    launch_chol_solve(ete, ws.at<double>(ws.L.etf), nt, ws.at<double>(ws.L.zf), k2.s);
    if (cudaEventRecord(k2.zf, k2.s) != cudaSuccess) return PS_ERR_CUDA;
    launch_chol_inverse(ete, nt, p->mu3, ws.at<float>(ws.L.Q), nullptr, st);
    if (cudaStreamWaitEvent(st, k2.zf, 0) != cudaSuccess) return PS_ERR_CUDA;
    int *ki = ws.at<int>(ws.L.kinfo);
    launch_admm(ws.at<float>(ws.L.Q), ws.at<double>(ws.L.zf), R, *p, d_kernel, ki, ki + 1,
                reinterpret_cast<double *>(ki + 2), st);
    launch_collect_status(nullptr, 0, ki, st);
    if ((s = last_launch()) != PS_OK) return s;
    if (h_info) return read_kernel_info(ws, st, h_info);
    return PS_OK;
}

}  // namespace

extern "C" {

ps_status ps_solve_hrms(const float *d_lrms, const float *d_pan, const float *d_kernel, int N,
                        int H, int W, int ratio, int R, const ps_hrms_params *p,
                        const float *d_z_init, float *d_hrms, float *d_z0,
                        ps_band_info *h_info, void *d_ws, size_t ws_bytes, void *stream) {
    ps_status s;
    SolveCall sc;
    if ((s = make_solve_call(d_lrms, d_pan, d_kernel, N, H, W, ratio, R, p, d_z_init, d_hrms,
                             d_z0, d_ws, ws_bytes, &sc)) != PS_OK)
        return s;
    return run_solve(sc, (cudaStream_t)stream, h_info);
}

ps_status ps_autotune(int N, int H, int W, int ratio, int R, int r, const float *d_lrms,
                      const float *d_pan, const float *d_kernel, void *d_ws, size_t ws_bytes,
                      void *stream, ps_tuning *h_out) {
    ps_status s;
    if ((s = check_dims(N, H, W, ratio, R)) != PS_OK) return s;
    if ((s = check_fft_dims(H, W)) != PS_OK) return s;
    if (r < 1 || r > kMaxWinR) return PS_ERR_INVALID_ARG;
    if (!precond_supported(H, W, ratio)) return PS_ERR_UNSUPPORTED;
    Ws ws;
    if ((s = bind_ws(d_ws, ws_bytes, N, H, W, ratio, R, &ws)) != PS_OK) return s;
    cudaStream_t capture = nullptr;
    if ((s = ensure_device(&capture)) != PS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t HW = (size_t)H * W;
    // zeroed inputs: the kernels' times do not depend on the values
    const size_t vec = (size_t)N * HW * sizeof(float);
    if (cudaMemsetAsync(ws.base + ws.L.st4, 0, HW * 16, st) != cudaSuccess ||
        cudaMemsetAsync(ws.base + ws.L.r, 0, vec, st) != cudaSuccess ||
        cudaMemsetAsync(ws.base + ws.L.pA, 0, vec, st) != cudaSuccess)
        return PS_ERR_CUDA;
    // a kernel spectrum of ones: a zero one would make the DC group singular,
    // and the NaN it spreads would end the timed CG iterations early
    launch_fill(ws.at<float>(ws.L.bh32), 2 * HW, 1.0f, st);
    launch_fft_twiddles(W, ws.at<float2>(ws.L.twW32), ws.at<double2>(ws.L.twW64), st);
    launch_fft_twiddles(H, ws.at<float2>(ws.L.twH32), ws.at<double2>(ws.L.twH64), st);
    CgBand *bands = ws.at<CgBand>(ws.L.bands);
    CgGlobal *g = ws.at<CgGlobal>(ws.L.glob);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return PS_ERR_CUDA;
    // best of three single launches, the CG scalars reset before each
    auto timed = [&](auto launch, bool reset = true) -> float {
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            if (reset) {
                cudaMemsetAsync(bands, 0, N * sizeof(CgBand), st);
                cudaMemsetAsync(g, 0, sizeof(CgGlobal), st);
                cudaEventRecord(e0, st);
            }
            launch();
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;  // the first launch warms up
        }
        return best * 1000.f;
    };
    ps_tuning out;
    memset(&out, 0, sizeof(out));
    PrecArgs pa = make_prec_args(ws, ws.at<float>(ws.L.r), ws.at<float>(ws.L.z), N, H, W, ratio,
                                 2e-4f, nullptr, nullptr);
    const int trs[4] = {1, 2, 4, 8};
    float bestp = 1e30f;
    pa.impl = 1;  // the shared-memory passes, whose row passes take this knob
    for (int k = 0; k < 4; ++k) {
        if (!precond_rows_ok(H, W, ratio, trs[k])) continue;
        pa.rows = trs[k];
        out.prec_us[k] = timed([&] { launch_precond(pa, st); });
        if (out.prec_us[k] < bestp) {
            bestp = out.prec_us[k];
            out.prec_rows = trs[k];
        }
    }
    // the blur-decimate variants of the CG loop (p_new = z + beta p_old fused)
    {
        const float *uu = ws.at<float>(ws.L.kern);
        out.db_impl = 1;
        float bestd = 1e30f;
        for (int k = 0; k < 2; ++k) {
            out.db_impl_us[k] = timed([&] {
                launch_db(ws.at<float>(ws.L.pA), ws.at<float>(ws.L.z), ws.at<float>(ws.L.pB),
                          bands, g, 1, N, H, W, ratio, uu, R, ws.at<float>(ws.L.v), st, k + 1);
            });
            if (out.db_impl_us[k] < bestd) {
                bestd = out.db_impl_us[k];
                out.db_impl = k + 1;
            }
        }
    }
    // the register-resident passes against the best of those
    out.prec_impl = 1;
    out.prec_impl_us[0] = bestp;
    if (precond_reg_supported(H, W, ratio)) {
        pa.impl = 2;
        pa.rows = 0;
        out.prec_impl_us[1] = timed([&] { launch_precond(pa, st); });
        if (out.prec_impl_us[1] < bestp) out.prec_impl = 2;
    }
    LlpArgs la = {};
    la.in = ws.at<float>(ws.L.pA);
    la.st4 = ws.at<float4>(ws.L.st4);
    la.H = H;
    la.W = W;
    la.N = N;
    la.c = ratio;
    la.lam = 2e-4f;
    la.out = ws.at<float>(ws.L.ap);
    la.bands = bands;
    la.g = g;
    la.cg = 1;
    float bestl = 1e30f;
    const int pfs[3] = {2, 3, 4};
    for (int k = 0; k < 2; ++k) {
        for (int q = 0; q < 3; ++q) {
            la.ty = llp_cgq2_rows(r, k);
            la.pf = pfs[q];
            const float us = timed([&] { launch_llp_cgq2(la, r, N, st); });
            out.llp_us[k * 3 + q] = us;
            if (us < bestl) {
                bestl = us;
                out.llp_rows = la.ty;
                out.llp_pf = la.pf;
            }
        }
    }
    // the shared-memory ring of asynchronous copies, long and short walks
    for (int k = 0; k < 2; ++k) {
        la.ty = llp_cgq2_rows(r, k);
        la.pf = 8;
        const float us = timed([&] { launch_llp_cgq2(la, r, N, st); });
        out.llp_ring_us[k] = us;
        if (us < bestl) {
            bestl = us;
            out.llp_rows = la.ty;
            out.llp_pf = 8;
        }
    }
    // the lean walks (r = 1): two and four columns a lane, long and short
    // walks, 2 and 4 rows ahead
    out.llp_form = 1;
    const int forms[2] = {2, 4};
    for (int f = 0; f < 2; ++f) {
        if (!llp_lean_supported(forms[f], r, W)) continue;
        const int pf4[2] = {2, 4};
        la.form = forms[f];
        for (int k = 0; k < 2; ++k) {
            for (int q = 0; q < 2; ++q) {
                la.ty = llp_lean_rows(k);
                la.pf = pf4[q];
                const float us = timed([&] { launch_llp_cgq2(la, r, N, st); });
                out.llp_lean_us[f * 4 + k * 2 + q] = us;
                if (us < bestl) {
                    bestl = us;
                    out.llp_rows = la.ty;
                    out.llp_pf = la.pf;
                    out.llp_form = forms[f];
                }
            }
        }
        la.form = 0;
    }
    // two bands per CTA (shared statistics), long and short walks
    out.llp_bands = 1;
    for (int k = 0; k < 2 && N >= 2; ++k) {
        la.ty = llp_cgq2_rows(r, k);
        la.pf = 2;
        la.nbd = 2;
        const float us = timed([&] { launch_llp_cgq2(la, r, N, st); });
        out.llp2_us[k] = us;
        if (us < bestl) {
            bestl = us;
            out.llp_rows = la.ty;
            out.llp_pf = la.pf;
            out.llp_bands = 2;
            out.llp_form = 1;
        }
    }
    // branches of the CG iteration, when the scene is given: whole solves of
    // 20 iterations (tolerance out of reach) per candidate, on the caller's
    // data; the solves' results go to scratch (the preconditioner's z buffer)
    if (d_lrms && d_pan && d_kernel) {
        ps_hrms_params hp;
        ps_default_hrms_params(&hp);
        hp.r = r;
        hp.tol = 1e-30f;
        hp.max_iter = 20;
        const int splits[3] = {1, 2, 4};
        float bests = 1e30f;
        for (int k = 0; k < 3; ++k) {
            if (splits[k] > 1 && N < 2 * splits[k]) continue;
            tuning_set(dev, N, H, W, ratio, r,
                       Tuning{out.prec_rows, out.llp_rows, splits[k], out.llp_pf,
                              out.llp_bands, out.prec_impl, out.db_impl, out.llp_form});
            float best = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, st);
                s = ps_solve_hrms(d_lrms, d_pan, d_kernel, N, H, W, ratio, R, &hp, nullptr,
                                  ws.at<float>(ws.L.z), nullptr, nullptr, d_ws, ws_bytes, stream);
                if (s != PS_OK) return s;
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && ms < best) best = ms;  // the first run captures the graph
            }
            out.split_us[k] = best * 1000.f;
            if (out.split_us[k] < bests) {
                bests = out.split_us[k];
                out.split = splits[k];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if ((s = last_launch()) != PS_OK) return s;
    tuning_set(dev, N, H, W, ratio, r,
               Tuning{out.prec_rows, out.llp_rows, out.split, out.llp_pf, out.llp_bands,
                      out.prec_impl, out.db_impl, out.llp_form});
    if (h_out) *h_out = out;
    return PS_OK;
}

ps_status ps_get_tuning(int N, int H, int W, int ratio, int r, ps_tuning *h_out) {
    if (!h_out) return PS_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PS_ERR_CUDA;
    const Tuning t = tuning_get(dev, N, H, W, ratio, r);
    memset(h_out, 0, sizeof(*h_out));
    h_out->prec_rows = t.prec_rows;
    h_out->llp_rows = t.llp_rows;
    h_out->llp_pf = t.llp_pf;
    h_out->split = t.split;
    h_out->llp_bands = t.llp_bands;
    h_out->prec_impl = t.prec_impl;
    h_out->db_impl = t.db_impl;
    h_out->llp_form = t.llp_form;
    return PS_OK;
}

ps_status ps_set_tuning(int N, int H, int W, int ratio, int r, const ps_tuning *h_in) {
    ps_status s;
    if (!h_in) return PS_ERR_INVALID_ARG;
    if ((s = check_dims(N, H, W, ratio, 0)) != PS_OK) return s;
    if (r < 1 || r > kMaxWinR) return PS_ERR_INVALID_ARG;
    const ps_tuning &t = *h_in;
    if (t.prec_rows && !precond_rows_ok(H, W, ratio, t.prec_rows)) return PS_ERR_INVALID_ARG;
    if (t.llp_form < 0 || t.llp_form == 3 || t.llp_form > 4) return PS_ERR_INVALID_ARG;
    const bool lean = t.llp_form >= 2;
    if (lean && (!llp_lean_supported(t.llp_form, r, W) || t.llp_bands == 2 || t.llp_pf == 3 ||
                 t.llp_pf == 8))
        return PS_ERR_INVALID_ARG;
    if (lean ? (t.llp_rows && t.llp_rows != llp_lean_rows(0) && t.llp_rows != llp_lean_rows(1))
             : (t.llp_rows && t.llp_rows != llp_cgq2_rows(r, 0) &&
                t.llp_rows != llp_cgq2_rows(r, 1)))
        return PS_ERR_INVALID_ARG;
    if (t.llp_pf && t.llp_pf != 2 && t.llp_pf != 3 && t.llp_pf != 4 && t.llp_pf != 8)
        return PS_ERR_INVALID_ARG;
    if (t.split && t.split != 1 && t.split != 2 && t.split != 4) return PS_ERR_INVALID_ARG;
    if (t.llp_bands && t.llp_bands != 1 && t.llp_bands != 2) return PS_ERR_INVALID_ARG;
    if (t.prec_impl < 0 || t.prec_impl > 3 ||
        (t.prec_impl == 2 && !precond_reg_supported(H, W, ratio)) ||
        (t.prec_impl == 3 && !precond_cluster_supported(H, W, ratio)))
        return PS_ERR_INVALID_ARG;
    if (t.db_impl < 0 || t.db_impl > 2) return PS_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PS_ERR_CUDA;
    tuning_set(dev, N, H, W, ratio, r, Tuning{t.prec_rows, t.llp_rows, t.split, t.llp_pf,
                                              t.llp_bands, t.prec_impl, t.db_impl,
                                              t.llp_form});
    return PS_OK;
}

ps_status ps_pansharpen(const float *d_lrms, const float *d_pan, int N, int H, int W, int ratio,
                        int R, const ps_kernel_params *kp, const ps_hrms_params *hp,
                        float *d_hrms, float *d_kernel_out, ps_kernel_info *h_kinfo,
                        ps_band_info *h_binfo, void *d_ws, size_t ws_bytes, void *stream) {
    ps_status s;
    if ((s = check_dims(N, H, W, ratio, R)) != PS_OK) return s;
    if ((s = check_fft_dims(H, W)) != PS_OK) return s;
    if ((s = check_hrms(hp)) != PS_OK) return s;
    if ((s = check_kernel_params(kp)) != PS_OK) return s;
    if ((s = check_band_mask(kp->band_mask, N)) != PS_OK) return s;
    Ws ws;
    if ((s = bind_ws(d_ws, ws_bytes, N, H, W, ratio, R, &ws)) != PS_OK) return s;
    float *kern = d_kernel_out ? d_kernel_out : ws.at<float>(ws.L.kern);
    SolveCall sc;
    if ((s = make_solve_call(d_lrms, d_pan, kern, N, H, W, ratio, R, hp, nullptr, d_hrms, nullptr,
                             d_ws, ws_bytes, &sc)) != PS_OK)
        return s;
    cudaStream_t capture = nullptr;
    if ((s = ensure_device(&capture)) != PS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // The kernel estimate, mostly latency-bound kernels on a few SMs, runs
    // on a high-priority side stream while the solve's kernel-independent
    // steps (PAN statistics, warm start) run on the caller's stream. They
    // touch disjoint parts of the workspace; the solve proper waits for both.
    // The network starts once the estimate's lag correlations (its one
    // kernel that fills the GPU) are done, so that its persistent grids meet
    // only the estimate's latency-bound kernels; the PAN statistics and the
    // bicubic, memory-bound, run beside the lag correlations. Everything is
    // queued before h_kinfo is read back.
    const Early e = device_early();
    if (cudaEventRecord(e.fork, st) != cudaSuccess ||
        cudaStreamWaitEvent(e.s, e.fork, 0) != cudaSuccess)
        return PS_ERR_CUDA;
    s = estimate_kernel_impl(d_lrms, d_pan, N, H, W, ratio, R, kp, nullptr, kern, nullptr,
                             nullptr, d_ws, ws_bytes, e.s, e.lags);
    if (s != PS_OK) return s;
    if ((s = solve_early(sc, st, kEarlyReserveSms, e.lags)) != PS_OK) return s;
    if (cudaEventRecord(e.join, e.s) != cudaSuccess ||
        cudaStreamWaitEvent(st, e.join, 0) != cudaSuccess)
        return PS_ERR_CUDA;
    if (h_kinfo && (s = read_kernel_info(ws, e.s, h_kinfo)) != PS_OK) return s;
    sc.early = 1;
    return run_solve(sc, st, h_binfo);
}

size_t ps_batch_workspace_size(const ps_scene *scenes, int count, const ps_hrms_params *hp) {
    if (!scenes || count < 1 || count > kMaxBatch) return 0;
    size_t total = batch_header_bytes(count);
    for (int i = 0; i < count; ++i) {
        const size_t b = scene_ws_bytes(scenes[i], hp);
        if (b == 0) return 0;
        total += b;
    }
    return total;
}

ps_status ps_pansharpen_batched(const ps_scene *scenes, int count, const ps_kernel_params *kp,
                                const ps_hrms_params *hp, ps_kernel_info *h_kinfo,
                                ps_band_info *h_binfo, void *d_ws, size_t ws_bytes,
                                void *stream) {
    ps_status s;
    if (!scenes || count < 1 || count > kMaxBatch) return PS_ERR_INVALID_ARG;
    if ((s = check_hrms(hp)) != PS_OK) return s;
    if (hp->host_loop || hp->precond_diag) return PS_ERR_INVALID_ARG;
    if (kp && (s = check_kernel_params(kp)) != PS_OK) return s;
    if (!d_ws || ((uintptr_t)d_ws) % kAlign) return PS_ERR_WORKSPACE;
    for (int i = 0; i < count; ++i) {
        const ps_scene &q = scenes[i];
        if ((s = check_dims(q.N, q.H, q.W, q.ratio, q.R)) != PS_OK) return s;
        if (!q.kernel) return PS_ERR_INVALID_ARG;
        if (kp && (s = check_band_mask(q.band_mask ? q.band_mask : kp->band_mask, q.N)) !=
                      PS_OK)
            return s;
        const void *hp3[3] = {q.h_lrms, q.h_pan, q.h_hrms};
        for (const void *h : hp3) {
            if (!h) continue;
            cudaPointerAttributes at;
            if (cudaPointerGetAttributes(&at, h) != cudaSuccess || at.type != cudaMemoryTypeHost) {
                cudaGetLastError();
                return PS_ERR_INVALID_ARG;
            }
        }
    }
    if (ws_bytes < ps_batch_workspace_size(scenes, count, hp)) return PS_ERR_WORKSPACE;
    char *base = static_cast<char *>(d_ws);
    std::vector<SolveCall> calls(count);
    size_t off = batch_header_bytes(count);
    for (int i = 0; i < count; ++i) {
        const ps_scene &q = scenes[i];
        const size_t b = scene_ws_bytes(q, hp);
        if ((s = make_solve_call(q.lrms, q.pan, q.kernel, q.N, q.H, q.W, q.ratio, q.R, hp,
                                 nullptr, q.hrms, nullptr, base + off, b, &calls[i])) != PS_OK)
            return s;
        off += b;
    }
    cudaStream_t capture = nullptr;
    if ((s = ensure_device(&capture)) != PS_OK) return s;
    std::vector<char> key;
    int dev = 0;
    cudaGetDevice(&dev);
    key_put(key, dev);
    key_put(key, count);
    key_put(key, d_ws);
    // field by field: the callers' structs may carry uninitialised padding
    key_put(key, hp->lambda);
    key_put(key, hp->r);
    key_put(key, hp->eps);
    key_put(key, hp->tol);
    key_put(key, hp->max_iter);
    key_put(key, hp->exact_weight);
    key_put(key, hp->precond);
    key_put(key, hp->precond_gamma);
    key_put(key, hp->warm);
    key_put(key, hp->cnn_params);
    key_put(key, hp->stop_rule);
    key_put(key, hp->prior);
    key_put(key, hp->zstep_fp32);
    key_put(key, hp->diag_params);
    key_put(key, kp != nullptr);
    if (kp) {
        key_put(key, kp->lambda_omega);
        key_put(key, kp->l);
        key_put(key, kp->alpha1);
        key_put(key, kp->alpha2);
        key_put(key, kp->mu1);
        key_put(key, kp->mu2);
        key_put(key, kp->mu3);
        key_put(key, kp->rho);
        key_put(key, kp->t_max);
        key_put(key, kp->th);
        key_put(key, kp->band_mask);
    }
    for (int i = 0; i < count; ++i) {
        const ps_scene &q = scenes[i];
        key_put(key, q.lrms);
        key_put(key, q.pan);
        key_put(key, q.hrms);
        key_put(key, q.kernel);
        const int dims[5] = {q.N, q.H, q.W, q.ratio, q.R};
        key_put(key, dims);
        key_put(key, q.band_mask);
        key_put(key, q.h_lrms);
        key_put(key, q.h_pan);
        key_put(key, q.h_hrms);
        const Tuning t = tuning_get(dev, q.N, q.H, q.W, q.ratio, hp->r);
        const int tk[8] = {t.prec_rows, t.llp_rows, t.split, t.llp_pf, t.llp_bands,
                           t.prec_impl, t.db_impl, t.llp_form};
        key_put(key, tk);
    }
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (auto &e : g_batch)
            if (e.key == key) exec = e.exec;
    }
    if (!exec) {
        unsigned long long *stamps = reinterpret_cast<unsigned long long *>(base);
        if ((s = build_batch_graph(scenes, count, kp, calls, stamps, capture, &exec)) != PS_OK)
            return s;
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_batch.size() >= 4) {
            cudaGraphExecDestroy(g_batch.front().exec);
            g_batch.erase(g_batch.begin());
        }
        g_batch.push_back({key, exec});
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaGraphLaunch(exec, st) != cudaSuccess) return PS_ERR_CUDA;
    if (h_kinfo || h_binfo) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return PS_ERR_CUDA;
        int nb = 0;
        for (int i = 0; i < count; ++i) {
            const Ws &ws = calls[i].ws;
            if (h_binfo) {
                if ((s = read_band_info(ws.at<CgBand>(ws.L.bands), scenes[i].N, h_binfo + nb)) !=
                    PS_OK)
                    return s;
                nb += scenes[i].N;
            }
            if (h_kinfo) {
                int hi[2] = {0, 0};
                double ch = 0.0;
                if (kp) {
                    const int *ki = ws.at<int>(ws.L.kinfo);
                    if (cudaMemcpy(hi, ki, sizeof(hi), cudaMemcpyDeviceToHost) != cudaSuccess ||
                        cudaMemcpy(&ch, ki + 2, sizeof(double), cudaMemcpyDeviceToHost) !=
                            cudaSuccess)
                        return PS_ERR_CUDA;
                }
                h_kinfo[i].iters = hi[0];
                h_kinfo[i].status = hi[1];
                h_kinfo[i].last_change = ch;
            }
        }
    }
    return PS_OK;
}

ps_status ps_batch_scene_ms(const void *d_ws, int count, void *stream, double *h_ms) {
    if (!d_ws || !h_ms || count < 1 || count > kMaxBatch) return PS_ERR_INVALID_ARG;
    std::vector<unsigned long long> t(count + 1);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(t.data(), d_ws, t.size() * 8, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PS_ERR_CUDA;
    for (int i = 0; i < count; ++i) h_ms[i] = (double)(long long)(t[1 + i] - t[0]) * 1e-6;
    return PS_OK;
}

// ---------------------------------------------------------------------------
// Operator-level entry points (ps_ops.h)
// ---------------------------------------------------------------------------
ps_status ps_op_blur_decimate(const float *d_z, int N, int H, int W, int ratio,
                              const float *d_kernel, int R, float *d_v, void *stream) {
    ps_status s;
    if ((s = check_dims(N, H, W, ratio, R)) != PS_OK) return s;
    if (!d_z || !d_kernel || !d_v) return PS_ERR_INVALID_ARG;
    if ((s = ensure_device(nullptr)) != PS_OK) return s;
    launch_db(d_z, nullptr, nullptr, nullptr, nullptr, 0, N, H, W, ratio, d_kernel, R, d_v,
              (cudaStream_t)stream);
    return last_launch();
}

ps_status ps_op_blur_decimate_adj(const float *d_v, int N, int H, int W, int ratio,
                                  const float *d_kernel, int R, float *d_z, void *stream) {
    ps_status s;
    if ((s = check_dims(N, H, W, ratio, R)) != PS_OK) return s;
    if (!d_z || !d_kernel || !d_v) return PS_ERR_INVALID_ARG;
    if ((s = ensure_device(nullptr)) != PS_OK) return s;
    launch_adj(d_v, N, H, W, ratio, d_kernel, R, d_z, (cudaStream_t)stream);
    return last_launch();
}

ps_status ps_op_pan_stats(const float *d_pan, int H, int W, int r, float eps, float *d_I,
                          float *d_mu, float *d_s, void *stream) {
    if (H < 1 || W < 1 || r < 1 || r > kMaxWinR || !(eps > 0.f)) return PS_ERR_INVALID_ARG;
    if (!d_pan || !d_I || !d_mu || !d_s) return PS_ERR_INVALID_ARG;
    ps_status s;
    if ((s = ensure_device(nullptr)) != PS_OK) return s;
    launch_pan_stats(d_pan, H, W, r, eps, d_I, d_mu, d_s, nullptr, (cudaStream_t)stream);
    return last_launch();
}

ps_status ps_op_apply_z0(const float *d_z, int N, int H, int W, int ratio,
                         const float *d_kernel, int R, const float *d_I, const float *d_mu,
                         const float *d_s, int r, float lambda, float *d_out, void *d_ws,
                         size_t ws_bytes, void *stream) {
    ps_status s;
    if ((s = check_dims(N, H, W, ratio, R)) != PS_OK) return s;
    if (r < 1 || r > kMaxWinR || !isfinite(lambda)) return PS_ERR_INVALID_ARG;
    if (!d_z || !d_kernel || !d_I || !d_mu || !d_s || !d_out) return PS_ERR_INVALID_ARG;
    Ws ws;
    if ((s = bind_ws(d_ws, ws_bytes, N, H, W, ratio, R, &ws)) != PS_OK) return s;
    if ((s = ensure_device(nullptr)) != PS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    float *v = ws.at<float>(ws.L.v);
    float4 *st4 = ws.at<float4>(ws.L.st4);
    launch_pack_stats(d_I, d_mu, d_s, (size_t)H * W, st4, st);
    launch_db(d_z, nullptr, nullptr, nullptr, nullptr, 0, N, H, W, ratio, d_kernel, R, v, st);
    LlpArgs la = {};
    la.in = d_z;
    la.lr = v;
    la.st4 = st4;
    la.u = d_kernel;
    la.R = R;
    la.c = ratio;
    la.H = H;
    la.W = W;
    la.N = N;
    la.lam = lambda;
    la.out = d_out;
    launch_llp(la, LLP_APPLY, r, N, st);
    return last_launch();
}

ps_status ps_op_jacobi_diag(int H, int W, int ratio, const float *d_kernel, int R,
                            const float *d_I, const float *d_mu, const float *d_s, int r,
                            float lambda, float *d_diag, void *d_ws, size_t ws_bytes,
                            void *stream) {
    ps_status s;
    if ((s = check_dims(1, H, W, ratio, R)) != PS_OK) return s;
    if (r < 1 || r > kMaxWinR || !isfinite(lambda)) return PS_ERR_INVALID_ARG;
    if (!d_kernel || !d_I || !d_mu || !d_s || !d_diag) return PS_ERR_INVALID_ARG;
    Ws ws;
    if ((s = bind_ws(d_ws, ws_bytes, 1, H, W, ratio, R, &ws)) != PS_OK) return s;
    if ((s = ensure_device(nullptr)) != PS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    float4 *st4 = ws.at<float4>(ws.L.st4);
    launch_pack_stats(d_I, d_mu, d_s, (size_t)H * W, st4, st);
    launch_jacobi_diag(st4, d_kernel, R, ratio, H, W, r, lambda, 1, 0, d_diag, st);
    return last_launch();
}

ps_status ps_op_guided_filter(const float *d_q, int N, int H, int W, const float *d_I,
                              const float *d_mu, const float *d_s, int r, float *d_out,
                              void *d_ws, size_t ws_bytes, void *stream) {
    if (N < 1 || N > kMaxBands || H < 1 || W < 1 || r < 1 || r > kMaxWinR)
        return PS_ERR_INVALID_ARG;
    if (!d_q || !d_I || !d_mu || !d_s || !d_out) return PS_ERR_INVALID_ARG;
    ps_status s;
    if (!d_ws || ((uintptr_t)d_ws) % kAlign) return PS_ERR_WORKSPACE;
    if (ws_bytes < (size_t)H * W * 16) return PS_ERR_WORKSPACE;
    if ((s = ensure_device(nullptr)) != PS_OK) return s;
    float4 *st4 = static_cast<float4 *>(d_ws);
    launch_pack_stats(d_I, d_mu, d_s, (size_t)H * W, st4, (cudaStream_t)stream);
    LlpArgs la = {};
    la.in = d_q;
    la.st4 = st4;
    la.H = H;
    la.W = W;
    la.N = N;
    la.c = 1;
    la.out = d_out;
    launch_llp(la, LLP_GF, r, N, (cudaStream_t)stream);
    return last_launch();
}

ps_status ps_op_zstep(const float *d_lrms, const float *d_z0, int N, int H, int W, int ratio,
                      const float *d_kernel, int R, const float *d_I, const float *d_mu,
                      const float *d_s, int r, float lambda, int exact_weight, float *d_z,
                      void *d_ws, size_t ws_bytes, void *stream) {
    ps_status s;
    if ((s = check_dims(N, H, W, ratio, R)) != PS_OK) return s;
    if ((s = check_fft_dims(H, W)) != PS_OK) return s;
    if (r < 1 || r > kMaxWinR || !(lambda > 0.f)) return PS_ERR_INVALID_ARG;
    if (!d_lrms || !d_z0 || !d_kernel || !d_I || !d_mu || !d_s || !d_z)
        return PS_ERR_INVALID_ARG;
    Ws ws;
    if ((s = bind_ws(d_ws, ws_bytes, N, H, W, ratio, R, &ws)) != PS_OK) return s;
    if ((s = ensure_device(nullptr)) != PS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t HW = (size_t)H * W;
    // the Z step reads the statistics, packed, from the workspace
    launch_pack_stats(d_I, d_mu, d_s, HW, ws.at<float4>(ws.L.st4), st);
    const float lam_z = lambda * (exact_weight ? (float)((2 * r + 1) * (2 * r + 1)) : 1.0f);
    if ((s = prepare_spectrum(ws, d_kernel, H, W, R, st)) != PS_OK) return s;
    return run_zstep(ws, d_lrms, d_z0, d_kernel, N, H, W, ratio, R, r, lam_z, d_z, st);
}

ps_status ps_op_bicubic_up(const float *d_lrms, int N, int H, int W, int ratio, float *d_out,
                           void *stream) {
    ps_status s;
    if ((s = check_dims(N, H, W, ratio, 0)) != PS_OK) return s;
    if (!d_lrms || !d_out || !aligned16(d_out)) return PS_ERR_INVALID_ARG;
    if ((s = ensure_device(nullptr)) != PS_OK) return s;
    launch_bicubic_up(d_lrms, N, H / ratio, W / ratio, ratio, d_out, (cudaStream_t)stream);
    return last_launch();
}

// ---------------------------------------------------------------------------
// Warm-start network (include/ps_cnn.h)
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

constexpr size_t kWPack = 18432;

struct CnnLayout {
    size_t act[6];    // act[1..5]: hidden activations (training); act[1], act[2] ping-pong
    size_t D[2];      // gradients between hidden layers (training)
    size_t d5;        // gradient of the output (training)
    size_t wf, wb;    // packed B operands, 4 layers each (forward, adjoint)
    size_t err;
    size_t total;
};

bool cnn_make_layout(int B, int H, int W, int training, CnnLayout *L) {
    if (B < 1 || H < 1 || W < 1) return false;
    const size_t P = (size_t)B * H * W;
    size_t o = 0;
    auto take = [&o](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    memset(L, 0, sizeof(*L));
    const int nact = training ? 5 : 2;
    for (int l = 1; l <= nact; ++l) L->act[l] = take(P * 64);
    if (training) {
        L->D[0] = take(P * 64);
        L->D[1] = take(P * 64);
        L->d5 = take(P * 4);
    }
    L->wf = take(4 * kWPack);
    L->wb = take(4 * kWPack);
    L->err = take(256);
    L->total = o + kAlign;
    return true;
}

struct CnnCall {
    char *base;
    CnnLayout L;
    int w_off[7], b_off[6];
    int sms;
    template <class T>
    T *at(size_t off) const { return reinterpret_cast<T *>(base + off); }
};

ps_status cnn_bind(void *d_ws, size_t ws_bytes, int B, int H, int W, int training, CnnCall *c) {
    if (!d_ws || ((uintptr_t)d_ws) % kAlign) return PS_ERR_WORKSPACE;
    if (!cnn_make_layout(B, H, W, training, &c->L)) return PS_ERR_INVALID_ARG;
    if (ws_bytes < c->L.total - kAlign) return PS_ERR_WORKSPACE;
    c->base = static_cast<char *>(d_ws);
    cnn_layout(c->w_off, c->b_off);
    ps_status s = ensure_device(nullptr, &c->sms);
    return s;
}

void cnn_conv(const CnnCall &c, const __nv_bfloat16 *in, __nv_bfloat16 *out, int layer,
              int adjoint, const __nv_bfloat16 *mask, const float *params, int B, int H, int W,
              cudaStream_t st, int mode = CONV_PLAIN, const float *up = nullptr,
              float *z = nullptr) {
    Conv32Args a;
    memset(&a, 0, sizeof(a));
    a.mode = mode;
    a.up = up;
    a.w5 = params + c.w_off[5];
    a.z = z;
    a.in = in;
    a.out = out;
    a.wpack = c.base + (adjoint ? c.L.wb : c.L.wf) + (size_t)(layer - 1) * kWPack;
    a.bias = adjoint ? nullptr : params + c.b_off[layer];
    a.mask = mask;
    a.N = B;
    a.H = H;
    a.W = W;
    a.relu = adjoint ? 0 : 1;
    a.rpi = 32;
    a.err = c.at<int>(c.L.err);
    launch_conv32(a, c.sms, st);
}

ps_status cnn_check_inputs(const float *params, const float *up, const float *pan, int B, int H,
                           int W) {
    if (!params || !up || !pan || B < 1 || H < 3 || W < 3) return PS_ERR_INVALID_ARG;
    if (W % 4) return PS_ERR_UNSUPPORTED;
    return PS_OK;
}

}  // namespace

extern "C" {

int ps_cnn_param_count(void) {
    int w[7], b[6];
    cnn_layout(w, b);
    return w[6];
}

size_t ps_cnn_workspace_size(int B, int H, int W, int training) {
    CnnLayout L;
    if (!cnn_make_layout(B, H, W, training, &L)) return 0;
    return L.total;
}

ps_status ps_cnn_forward(const float *d_params, const float *d_up, const float *d_pan,
                         size_t pan_stride, int B, int H, int W, float *d_z, void *d_ws,
                         size_t ws_bytes, void *stream) {
    return cnn_forward_reserve(d_params, d_up, d_pan, pan_stride, B, H, W, d_z, d_ws, ws_bytes,
                               0, stream);
}

}  // extern "C"

namespace {

ps_status cnn_forward_reserve(const float *d_params, const float *d_up, const float *d_pan,
                              size_t pan_stride, int B, int H, int W, float *d_z, void *d_ws,
                              size_t ws_bytes, int reserve, void *stream) {
    ps_status s;
    if ((s = cnn_check_inputs(d_params, d_up, d_pan, B, H, W)) != PS_OK) return s;
    if (!d_z) return PS_ERR_INVALID_ARG;
    CnnCall c;
    if ((s = cnn_bind(d_ws, ws_bytes, B, H, W, 0, &c)) != PS_OK) return s;
    if (reserve > 0 && c.sms > 2 * reserve) c.sms -= reserve;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(c.at<int>(c.L.err), 0, sizeof(int), st) != cudaSuccess) return PS_ERR_CUDA;
    for (int l = 1; l <= 4; ++l)
        launch_pack_w32(d_params + c.w_off[l], c.base + c.L.wf + (l - 1) * kWPack, 0, st);
    __nv_bfloat16 *A = c.at<__nv_bfloat16>(c.L.act[1]), *Bf = c.at<__nv_bfloat16>(c.L.act[2]);
    // the first layer on the CUDA cores; layer 4 applies the last layer in
    // its epilogue, so a5 never reaches memory
    launch_cnn_first(d_up, d_pan, pan_stride, d_params + c.w_off[0], B, H, W, A, st);
    cnn_conv(c, A, Bf, 1, 0, nullptr, d_params, B, H, W, st);
    cnn_conv(c, Bf, A, 2, 0, nullptr, d_params, B, H, W, st);
    cnn_conv(c, A, Bf, 3, 0, nullptr, d_params, B, H, W, st);
    cnn_conv(c, Bf, nullptr, 4, 0, nullptr, d_params, B, H, W, st, CONV_LAST, d_up, d_z);
    return last_launch();
}

}  // namespace

extern "C" {

ps_status ps_cnn_loss_grad(const float *d_params, const float *d_up, const float *d_pan,
                           size_t pan_stride, const float *d_target, int B, int H, int W,
                           float *d_grad, double *d_loss, void *d_ws, size_t ws_bytes,
                           void *stream) {
    return ps_cnn_loss_grad_weighted(d_params, d_up, d_pan, pan_stride, d_target, nullptr, B, H,
                                     W, d_grad, d_loss, d_ws, ws_bytes, stream);
}

ps_status ps_cnn_loss_grad_weighted(const float *d_params, const float *d_up,
                                    const float *d_pan, size_t pan_stride, const float *d_target,
                                    const float *d_weight, int B, int H, int W, float *d_grad,
                                    double *d_loss, void *d_ws, size_t ws_bytes, void *stream) {
    ps_status s;
    if ((s = cnn_check_inputs(d_params, d_up, d_pan, B, H, W)) != PS_OK) return s;
    if (!d_target || !d_grad || !d_loss) return PS_ERR_INVALID_ARG;
    CnnCall c;
    if ((s = cnn_bind(d_ws, ws_bytes, B, H, W, 1, &c)) != PS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(c.at<int>(c.L.err), 0, sizeof(int), st) != cudaSuccess) return PS_ERR_CUDA;
    if (cudaMemsetAsync(d_grad, 0, (size_t)c.w_off[6] * sizeof(float), st) != cudaSuccess ||
        cudaMemsetAsync(d_loss, 0, sizeof(double), st) != cudaSuccess)
        return PS_ERR_CUDA;
    for (int l = 1; l <= 4; ++l) {
        launch_pack_w32(d_params + c.w_off[l], c.base + c.L.wf + (l - 1) * kWPack, 0, st);
        launch_pack_w32(d_params + c.w_off[l], c.base + c.L.wb + (l - 1) * kWPack, 1, st);
    }
    __nv_bfloat16 *act[6];
    for (int l = 1; l <= 5; ++l) act[l] = c.at<__nv_bfloat16>(c.L.act[l]);
    __nv_bfloat16 *D[2] = {c.at<__nv_bfloat16>(c.L.D[0]), c.at<__nv_bfloat16>(c.L.D[1])};
    float *d5 = c.at<float>(c.L.d5);
    // forward, keeping every activation
    launch_cnn_first(d_up, d_pan, pan_stride, d_params + c.w_off[0], B, H, W, act[1], st);
    for (int l = 1; l <= 4; ++l) cnn_conv(c, act[l], act[l + 1], l, 0, nullptr, d_params, B, H, W, st);
    launch_cnn_last(act[5], d_up, d_params + c.w_off[5], B, H, W, nullptr, d_target, d_weight, d5,
                    d_loss, st);
    // backward: D_l = dL / d(conv_l output before its ReLU)
    launch_cnn_last_bwd(act[5], d5, d_params + c.w_off[5], B, H, W, D[0], d_grad + c.w_off[5],
                        st);
    int cur = 0;
    for (int l = 4; l >= 1; --l) {
        launch_cnn_wgrad32(act[l], D[cur], B, H, W, d_grad + c.w_off[l], d_grad + c.b_off[l],
                           c.sms, st);
        cnn_conv(c, D[cur], D[cur ^ 1], l, 1, act[l], d_params, B, H, W, st);
        cur ^= 1;
    }
    launch_cnn_wgrad_first(d_up, d_pan, pan_stride, D[cur], B, H, W, d_grad + c.w_off[0], st);
    return last_launch();
}

ps_status ps_cnn_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int step,
                      float lr, float beta1, float beta2, float eps, void *stream) {
    if (!d_params || !d_grad || !d_m || !d_v || step < 1) return PS_ERR_INVALID_ARG;
    if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
        !(eps > 0.f))
        return PS_ERR_INVALID_ARG;
    launch_cnn_adam(d_params, d_grad, d_m, d_v, ps_cnn_param_count(), step, lr, beta1, beta2, eps,
                    (cudaStream_t)stream);
    return last_launch();
}

ps_status ps_cnn_sync_status(void *d_ws, int B, int H, int W, int training, void *stream) {
    CnnLayout L;
    if (!d_ws || !cnn_make_layout(B, H, W, training, &L)) return PS_ERR_INVALID_ARG;
    int *err = reinterpret_cast<int *>(static_cast<char *>(d_ws) + L.err);
    int h = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PS_ERR_CUDA;
    if (h && cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return PS_ERR_CUDA;
    return h ? PS_ERR_TIMEOUT : PS_OK;
}

ps_status ps_op_cnn_conv32(const void *d_in, int N, int H, int W, const float *d_weight,
                           const float *d_bias, const void *d_mask, int mode, void *d_out,
                           void *d_ws, size_t ws_bytes, void *stream) {
    if (N < 1 || H < 1 || W < 1 || mode < 0 || mode > 2) return PS_ERR_INVALID_ARG;
    if (!d_in || !d_weight || !d_out || d_in == d_out) return PS_ERR_INVALID_ARG;
    if (!aligned16(d_in) || !aligned16(d_out) || (d_mask && !aligned16(d_mask)))
        return PS_ERR_INVALID_ARG;
    if (!d_ws || ((uintptr_t)d_ws) % kAlign) return PS_ERR_WORKSPACE;
    if (ws_bytes < 18432 + 256) return PS_ERR_WORKSPACE;
    ps_status s;
    int sms = 0;
    if ((s = ensure_device(nullptr, &sms)) != PS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = static_cast<char *>(d_ws);
    int *err = reinterpret_cast<int *>(ws + 18432);
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return PS_ERR_CUDA;
    launch_pack_w32(d_weight, ws, mode == 2 ? 1 : 0, st);
    Conv32Args a;
    memset(&a, 0, sizeof(a));
    a.mode = CONV_PLAIN;
    a.in = static_cast<const __nv_bfloat16 *>(d_in);
    a.out = static_cast<__nv_bfloat16 *>(d_out);
    a.wpack = ws;
    a.bias = mode == 2 ? nullptr : d_bias;
    a.mask = mode == 2 ? static_cast<const __nv_bfloat16 *>(d_mask) : nullptr;
    a.N = N;
    a.H = H;
    a.W = W;
    a.relu = mode == 0 ? 1 : 0;
    a.rpi = 32;
    a.err = err;
    launch_conv32(a, sms, st);
    if ((s = last_launch()) != PS_OK) return s;
    int h_err = 0;
    if (cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PS_ERR_CUDA;
    return h_err ? PS_ERR_TIMEOUT : PS_OK;
}

ps_status ps_op_precond(const float *d_r, int N, int H, int W, int ratio, const float *d_kernel,
                        int R, float lambda_gamma, float *d_z, void *d_ws, size_t ws_bytes,
                        void *stream) {
    ps_status s;
    if ((s = check_dims(N, H, W, ratio, R)) != PS_OK) return s;
    if ((s = check_fft_dims(H, W)) != PS_OK) return s;
    if (!(lambda_gamma > 0.f) || !isfinite(lambda_gamma)) return PS_ERR_INVALID_ARG;
    if (!d_r || !d_kernel || !d_z) return PS_ERR_INVALID_ARG;
    if (!precond_supported(H, W, ratio)) return PS_ERR_UNSUPPORTED;
    Ws ws;
    if ((s = bind_ws(d_ws, ws_bytes, N, H, W, ratio, R, &ws)) != PS_OK) return s;
    if ((s = ensure_device(nullptr)) != PS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = prepare_spectrum(ws, d_kernel, H, W, R, st)) != PS_OK) return s;
    PrecArgs pa = make_prec_args(ws, d_r, d_z, N, H, W, ratio, lambda_gamma, nullptr, nullptr);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PS_ERR_CUDA;
    const Tuning t = tuning_get(dev, N, H, W, ratio, 1);  // the recorded implementation
    pa.impl = t.prec_impl;
    pa.rows = t.prec_rows;
    launch_precond(pa, st);
    return last_launch();
}

ps_status ps_op_omega(const float *d_lrms, const float *d_pan, int N, int H, int W, int ratio,
                      int l, float lambda_omega, float *d_omega, void *d_ws, size_t ws_bytes,
                      void *stream) {
    ps_status s;
    if ((s = check_dims(N, H, W, ratio, 0)) != PS_OK) return s;
    if (l < 0 || l > 16 || !(lambda_omega >= 0.f)) return PS_ERR_INVALID_ARG;
    if (!d_lrms || !d_pan || !d_omega) return PS_ERR_INVALID_ARG;
    Ws ws;
    if ((s = bind_ws(d_ws, ws_bytes, N, H, W, ratio, 0, &ws)) != PS_OK) return s;
    if ((s = ensure_device(nullptr)) != PS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int h = H / ratio, w = W / ratio;
    float *Aw = ws.at<float>(ws.L.v);
    const BandSel all = band_sel(0ull, N);
    launch_box_lr(d_lrms, all, h, w, l, Aw, st);
    launch_box_hr_dec(d_pan, H, W, ratio, ratio * l, ws.at<float>(ws.L.bvec), st);
    launch_omega_normal(Aw, ws.at<float>(ws.L.bvec), N, h * w, ws.at<double>(ws.L.G), st);
    launch_omega_solve(ws.at<double>(ws.L.G), all, N, lambda_omega, d_omega, st);
    return last_launch();
}

ps_status ps_op_kernel_normal_eq(const float *d_lrms, const float *d_pan, const float *d_omega,
                                 int N, int H, int W, int ratio, int R, double *d_EtE,
                                 double *d_Etf, void *d_ws, size_t ws_bytes, void *stream) {
    ps_status s;
    if ((s = check_dims(N, H, W, ratio, R)) != PS_OK) return s;
    if (!d_lrms || !d_pan || !d_omega || !d_EtE || !d_Etf) return PS_ERR_INVALID_ARG;
    Ws ws;
    if ((s = bind_ws(d_ws, ws_bytes, N, H, W, ratio, R, &ws)) != PS_OK) return s;
    if ((s = ensure_device(nullptr)) != PS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int hw = (H / ratio) * (W / ratio);
    float *f = ws.at<float>(ws.L.f);
    launch_combine_f(d_lrms, d_omega, N, hw, f, st);
    launch_ete_lags(d_pan, H, W, ratio, R, ws.at<double>(ws.L.lags), st);
    launch_ete_assemble(ws.at<double>(ws.L.lags), ratio, R, d_EtE, st);
    launch_etf(d_pan, H, W, ratio, R, f, d_Etf, st);
    return last_launch();
}

ps_status ps_op_admm(const double *d_EtE, const double *d_Etf, int R, const ps_kernel_params *p,
                     float *d_kernel, ps_kernel_info *h_info, void *d_ws, size_t ws_bytes,
                     void *stream) {
    ps_status s;
    if (R < 0 || R > kMaxR) return PS_ERR_INVALID_ARG;
    if ((s = check_kernel_params(p)) != PS_OK) return s;
    if (!d_EtE || !d_Etf || !d_kernel) return PS_ERR_INVALID_ARG;
    const int n = 2 * R + 1, nt = n * n;
    Ws ws;
    if ((s = bind_ws(d_ws, ws_bytes, 1, n, n, 1, R, &ws)) != PS_OK) return s;
    if ((s = ensure_device(nullptr)) != PS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    double *ete = ws.at<double>(ws.L.ete);
    if (cudaMemcpyAsync(ete, d_EtE, (size_t)nt * nt * 8, cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
        return PS_ERR_CUDA;
    launch_cholesky(ete, nt, p->mu3, st);
    launch_chol_solve(ete, d_Etf, nt, ws.at<double>(ws.L.zf), st);
    launch_chol_inverse(ete, nt, p->mu3, ws.at<float>(ws.L.Q), nullptr, st);
    int *ki = ws.at<int>(ws.L.kinfo);
    launch_admm(ws.at<float>(ws.L.Q), ws.at<double>(ws.L.zf), R, *p, d_kernel, ki, ki + 1,
                reinterpret_cast<double *>(ki + 2), st);
    launch_collect_status(nullptr, 0, ki, st);
    if ((s = last_launch()) != PS_OK) return s;
    if (h_info) return read_kernel_info(ws, st, h_info);
    return PS_OK;
}

}  // extern "C"
