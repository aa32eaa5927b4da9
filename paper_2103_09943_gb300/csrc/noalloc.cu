// Allocation-free variant of the kernel normal equations operator.
//
// Some callers cannot allocate device memory on their call path: plugins whose
// host application owns all device memory and hands out only the inputs and
// outputs, or real-time code where a cudaMalloc (with its possible implicit
// synchronisation and its possible failure) is not acceptable. For them,
// ps_op_kernel_normal_eq_noalloc takes no workspace: its scratch lives in
// the fixed-size array below, defined by this library and held on every GPU
// that loads it until the process exits.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "ps_ops.h"

namespace {

// Scratch of the allocation-free entry point: the combined LRMS f (h w
// floats) followed, 256-byte aligned, by the lag correlations
// (c^2 (4R+1)^2 doubles). Every call shares it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PS_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
void *g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (in host code the array's name is not a device address).
ps_status noalloc_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PS_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return PS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
            return PS_ERR_CUDA;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
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
    if (N < 1 || N > kMaxBands || ratio < 2 || ratio > kMaxRatio || R < 0 || R > kMaxR)
        return PS_ERR_INVALID_ARG;
    if (H < 1 || W < 1 || H % ratio || W % ratio || 2 * R + 1 > H || 2 * R + 1 > W)
        return PS_ERR_SHAPE;
    if (!d_lrms || !d_pan || !d_omega || !d_EtE || !d_Etf) return PS_ERR_INVALID_ARG;
    if (scratch_need(H, W, ratio, R) > (size_t)PS_NOALLOC_SCRATCH_BYTES)
        return PS_ERR_UNSUPPORTED;
    void *base = nullptr;
    ps_status s = noalloc_scratch(&base);
    if (s != PS_OK) return s;
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
