// Allocation-free variant of the kernel normal equations operator.
//
// Some callers cannot allocate device memory on their call path: plugins whose
// host application owns all device memory and hands out only the inputs and
// outputs, or real-time code where a cudaMalloc (with its possible implicit
// synchronisation and its possible failure) is not acceptable. For them,
// ps_op_kernel_normal_eq_noalloc takes no workspace: its scratch lives in
// the fixed-size array below, defined by this library and held on every GPU
// that loads it until the process exits.
#include <cuda.h>  // CUcontext and CUresult only: the two driver calls below are
                   // fetched through the runtime, so nothing links libcuda

#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "ps_ops.h"

namespace {

// Scratch of the allocation-free entry point: the combined LRMS f (h w
// floats) followed, 256-byte aligned, by the lag correlations
// (c^2 (4R+1)^2 doubles). Every call shares it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PS_NOALLOC_SCRATCH_BYTES];

// A __device__ array has one address per CUDA context (the module is loaded
// into each context on its own), so the looked-up address is cached per
// context, keyed by the context's unique ID: a context the caller made
// current through the driver API, or a primary context created anew after
// cudaDeviceReset, gets its own lookup.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

struct CtxCalls {
    CtxGetCurrentFn get_current = nullptr;
    CtxGetIdFn get_id = nullptr;
};

const CtxCalls &ctx_calls() {
    static const CtxCalls calls = [] {
        CtxCalls c;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            c.get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            c.get_id = reinterpret_cast<CtxGetIdFn>(f);
        return c;
    }();
    return calls;
}

struct CachedAddr {
    unsigned long long ctx_id;
    void *addr;
};

std::mutex g_noalloc_mu;
std::vector<CachedAddr> g_noalloc_addr;

// Device address of the scratch array in the current context (in host code
// the array's name is a host-side stand-in, not a device address).
ps_status noalloc_scratch(void **out) {
    const CtxCalls &d = ctx_calls();
    if (!d.get_current || !d.get_id) return PS_ERR_CUDA;
    CUcontext ctx = nullptr;
    if (d.get_current(&ctx) != CUDA_SUCCESS) return PS_ERR_CUDA;
    if (!ctx) {
        // No context is current on this thread yet: the runtime's symbol
        // lookup makes the current device's primary context current.
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
            return PS_ERR_CUDA;
        if (d.get_current(&ctx) != CUDA_SUCCESS || !ctx) return PS_ERR_CUDA;
    }
    unsigned long long id = 0;
    if (d.get_id(ctx, &id) != CUDA_SUCCESS) return PS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    for (const CachedAddr &e : g_noalloc_addr)
        if (e.ctx_id == id) {
            *out = e.addr;
            return PS_OK;
        }
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PS_ERR_CUDA;
    g_noalloc_addr.push_back({id, p});
    *out = p;
    return PS_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bytes of the scratch array one call needs.
size_t scratch_need(int H, int W, int ratio, int R) {
    const size_t hw = (size_t)(H / ratio) * (W / ratio);
    const size_t nl = (size_t)(4 * R + 1);
    return align256(hw * sizeof(float)) + (size_t)ratio * ratio * nl * nl * sizeof(double);
}

}  // namespace

extern "C" ps_status ps_op_kernel_normal_eq_noalloc(const float *d_lrms, const float *d_pan,
                                                    const float *d_omega, int N, int H, int W,
                                                    int ratio, int R, double *d_EtE,
                                                    double *d_Etf, void *stream) {
    using namespace ps;
    // the limits of ps_op_kernel_normal_eq, then the array's own
    ps_status s = check_dims(N, H, W, ratio, R);
    if (s != PS_OK) return s;
    if (!d_lrms || !d_pan || !d_omega || !d_EtE || !d_Etf) return PS_ERR_INVALID_ARG;
    if (scratch_need(H, W, ratio, R) > (size_t)PS_NOALLOC_SCRATCH_BYTES)
        return PS_ERR_UNSUPPORTED;
    void *base = nullptr;
    if ((s = noalloc_scratch(&base)) != PS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int hw = (H / ratio) * (W / ratio);
    // f and the lag table are written in full by their kernels: nothing in
    // the shared array needs clearing between calls.
    float *f = static_cast<float *>(base);
    double *lags = reinterpret_cast<double *>(static_cast<unsigned char *>(base) +
                                              align256((size_t)hw * sizeof(float)));
    launch_combine_f(d_lrms, d_omega, N, hw, f, st);
    launch_ete_lags(d_pan, H, W, ratio, R, lags, st);
    launch_ete_assemble(lags, ratio, R, d_EtE, st);
    launch_etf(d_pan, H, W, ratio, R, f, d_Etf, st);
    return cudaGetLastError() == cudaSuccess ? PS_OK : PS_ERR_CUDA;
}
