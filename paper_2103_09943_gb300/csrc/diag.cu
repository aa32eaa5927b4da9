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

// diag(A) of the Z0 operator A = B^T D^T D B + lam L^T M L (Eq.
// Z_ini_matting), one thread per pixel m = (y, x). Data part: the sum of
// u(i, j)^2 over the taps with i = -y, j = -x (mod c), one of c^2 phase sums
// formed first in shared memory. Prior part: sum over a, b in the 5-point
// stencil of m of L_ma L_mb M_ab, M_ab summed over the windows w_k (centres
// within RW + 1 of m) holding a and b: delta_ab - (1 + (I_a - mu_k)(I_b -
// mu_k) s_k) / |w| (Eq. matting_matrix). Written N times (once per band),
// inverted when `invert` (the Jacobi preconditioner s = 1 / diag(A)).
template <int RW>
__global__ void __launch_bounds__(256) jacobi_diag_kernel(const float4 *__restrict__ st4,
                                                          const float *__restrict__ u, int R,
                                                          int c, int H, int W, float lam,
                                                          int N, int invert,
                                                          float *__restrict__ out) {
    __shared__ float ph[kMaxRatio * kMaxRatio];
    const int n = 2 * R + 1;
    for (int q = threadIdx.y * blockDim.x + threadIdx.x; q < c * c; q += blockDim.x * blockDim.y) {
        const int a = q / c, b = q - (q / c) * c;
        float acc = 0.f;
        for (int i = -R; i <= R; ++i) {
            if ((((i % c) + c) % c) != a) continue;
            for (int j = -R; j <= R; ++j)
                if ((((j % c) + c) % c) == b) {
                    const float t = u[(i + R) * n + (j + R)];
                    acc = fmaf(t, t, acc);
                }
        }
        ph[q] = acc;
    }
    __syncthreads();
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    const float data = ph[((c - y % c) % c) * c + ((c - x % c) % c)];
    constexpr int sy[5] = {0, -1, 1, 0, 0}, sx[5] = {0, 0, 0, -1, 1};
    constexpr float lw[5] = {4.f, -1.f, -1.f, -1.f, -1.f};
    constexpr float inw = 1.0f / (float)((2 * RW + 1) * (2 * RW + 1));
    float Ia[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) Ia[a] = __ldg(&st4[(size_t)wrapi(y + sy[a], H) * W + wrapi(x + sx[a], W)]).x;
    float prior = 0.f;
#pragma unroll
    for (int ky = -RW - 1; ky <= RW + 1; ++ky)
#pragma unroll
        for (int kx = -RW - 1; kx <= RW + 1; ++kx) {
            bool in[5], any = false;
#pragma unroll
            for (int a = 0; a < 5; ++a) {
                const int dy = ky - sy[a], dx = kx - sx[a];
                in[a] = dy >= -RW && dy <= RW && dx >= -RW && dx <= RW;
                any = any || in[a];
            }
            if (!any) continue;
            const float4 q = __ldg(&st4[(size_t)wrapi(y + ky, H) * W + wrapi(x + kx, W)]);
            const float mu = q.y, sk = q.z;
#pragma unroll
            for (int a = 0; a < 5; ++a) {
                if (!in[a]) continue;
                const float da = (Ia[a] - mu) * sk;
#pragma unroll
                for (int b = 0; b < 5; ++b) {
                    if (!in[b]) continue;
                    const float term = (a == b ? 1.f : 0.f) - inw * fmaf(da, Ia[b] - mu, 1.f);
                    prior = fmaf(lw[a] * lw[b], term, prior);
                }
            }
        }
    const float d = fmaf(lam, prior, data);
    const float v = invert ? 1.0f / d : d;
    const size_t HW = (size_t)H * W, m = (size_t)y * W + x;
    for (int b = 0; b < N; ++b) out[b * HW + m] = v;
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

void launch_jacobi_diag(const float4 *st4, const float *u, int R, int c, int H, int W, int r,
                        float lam, int N, int invert, float *out, cudaStream_t st) {
    const dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8);
    switch (r) {
        case 1: jacobi_diag_kernel<1><<<grd, blk, 0, st>>>(st4, u, R, c, H, W, lam, N, invert, out); break;
        case 2: jacobi_diag_kernel<2><<<grd, blk, 0, st>>>(st4, u, R, c, H, W, lam, N, invert, out); break;
        case 3: jacobi_diag_kernel<3><<<grd, blk, 0, st>>>(st4, u, R, c, H, W, lam, N, invert, out); break;
        default: jacobi_diag_kernel<4><<<grd, blk, 0, st>>>(st4, u, R, c, H, W, lam, N, invert, out); break;
    }
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
