// Diagonal preconditioner of the Z0 CG (an extension of Eq. Z_ini_matting's
// solve: the paper runs plain CG): z = s * r with a per-pixel s > 0, and the
// head that turns the diagonal network's output into s.
//
// HBM per px.band: the preconditioner reads r and s and writes z (12 B);
// the head reads the network output and the bicubic input and writes s
// (12 B, once per solve).
#include "kernels.cuh"

namespace ps {
namespace {

// z = s r over the bands of the launch (grid.y = band) and the per-band
// r^T z. The last CTA of a band sets beta = r^T z / rho (0 before the first
// iteration) and rho = r^T z, or stops the band on a non-finite or
// non-positive r^T z, as the FFT preconditioner's last pass does.
__global__ void __launch_bounds__(256) diag_precond_kernel(const float4 *__restrict__ r,
                                                           const float4 *__restrict__ s,
                                                           float4 *__restrict__ z, size_t n4,
                                                           CgBand *bands) {
    __shared__ double red[8];
    const size_t off = (size_t)blockIdx.y * n4;
    float acc = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x) {
        const float4 rv = __ldg(r + off + i), sv = __ldg(s + off + i);
        const float4 zv = make_float4(sv.x * rv.x, sv.y * rv.y, sv.z * rv.z, sv.w * rv.w);
        z[off + i] = zv;
        acc = fmaf(rv.x, zv.x, fmaf(rv.y, zv.y, fmaf(rv.z, zv.z, fmaf(rv.w, zv.w, acc))));
    }
    const double t = block_sum_d((double)acc, red);
    if (threadIdx.x != 0 || !bands) return;
    CgBand *bd = bands + blockIdx.y;
    atomicAdd(&bd->rz_new, t);
    __threadfence();
    if (atomicAdd(&bd->cnt_prec, 1u) != gridDim.x - 1) return;
    __threadfence();
    bd->cnt_prec = 0u;
    const double rz = atomicAdd(&bd->rz_new, 0.0);
    bd->rz_new = 0.0;
    if (bd->done) return;
    if (!isfinite(rz)) {
        bd->status = PS_ERR_NONFINITE;
        bd->done = 1;
    } else if (!(rz > 0.0)) {
        bd->status = PS_ERR_BREAKDOWN;
        bd->done = 1;
    } else {
        bd->beta = bd->iters > 0 ? rz / bd->rho : 0.0;
        bd->rho = rz;
    }
}

// s = max((zd - up) / 255, floor), in place over up; fmaxf returns the floor
// for a NaN.
__global__ void __launch_bounds__(256) diag_head_kernel(const float4 *__restrict__ zd,
                                                        float4 *__restrict__ s, size_t n4,
                                                        float floor_) {
    constexpr float kInv = 1.0f / 255.0f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x) {
        const float4 a = __ldg(zd + i), b = s[i];
        s[i] = make_float4(fmaxf((a.x - b.x) * kInv, floor_), fmaxf((a.y - b.y) * kInv, floor_),
                           fmaxf((a.z - b.z) * kInv, floor_), fmaxf((a.w - b.w) * kInv, floor_));
    }
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n < 1) n = 1;
    }
    return n;
}

}  // namespace

void launch_diag_precond(const float *r, const float *s, float *z, int N, size_t HW,
                         CgBand *bands, cudaStream_t st) {
    const size_t n4 = HW / 4;
    // about eight 256-thread CTAs per SM over the launch's bands
    long long per = (long long)sm_count() * 8 / N;
    const long long need = (long long)((n4 + 255) / 256);
    if (per > need) per = need;
    if (per < 1) per = 1;
    diag_precond_kernel<<<dim3((unsigned)per, N), 256, 0, st>>>(
        reinterpret_cast<const float4 *>(r), reinterpret_cast<const float4 *>(s),
        reinterpret_cast<float4 *>(z), n4, bands);
}

void launch_diag_head(const float *zd, float *s, size_t n, float floor_, cudaStream_t st) {
    const size_t n4 = n / 4;
    long long grid = (long long)((n4 + 255) / 256);
    if (grid > (long long)sm_count() * 8) grid = (long long)sm_count() * 8;
    if (grid < 1) grid = 1;
    diag_head_kernel<<<(unsigned)grid, 256, 0, st>>>(reinterpret_cast<const float4 *>(zd),
                                                    reinterpret_cast<float4 *>(s), n4, floor_);
}

}  // namespace ps
