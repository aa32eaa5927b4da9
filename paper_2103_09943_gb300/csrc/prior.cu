// Alternative cross-channel priors (Sec. IV-D, Table III), sm_103a.
//
// The LLP regularises the local affine relation between L Z_i and L Y. The
// alternatives replace the Laplacian L by other filters F_d, each with its
// own affine model against the guide F_d Y:
//   LPF  F = u (the blur kernel, low-pass)     HPF  F = delta - u
//   LPP  F = delta (the pixels)                 LGC  F_h, F_v = first differences
// so the Z0 operator becomes B^T D^T D B + lam sum_d F_d^T M_d F_d (M_d the
// matting matrix of F_d Y) and the Z step (B^T D^T D B + lam' sum_d F_d^T F_d)
// Z = B^T D^T X + lam' sum_d F_d^T L-hat_d. The filters are applied with the
// blur kernels at ratio 1 (circular convolution and its adjoint); the kernels
// here are the window parts: guide statistics, the matting matrix and the
// guided filter as two window-sum passes, the combination with p^T q and
// alpha for the CG, the filters themselves, and the Fourier symbol
// sum_d |F_d^|^2 of the Z step.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace ps {

namespace {

constexpr int TX = 32, TY = 8;

__device__ __forceinline__ int wrapq(int i, int n) {
    int m = i % n;
    return m < 0 ? m + n : m;
}

__device__ __forceinline__ bool band_idle(const CgBand *bands, const CgGlobal *g, int b) {
    return bands && (g->stop || bands[b].done);
}

// Window sums over (2r+1)^2 torus windows of up to two images, tile TX x TY,
// via shared memory. `fa(y, x)` / `fb(y, x)` give the values at global
// (wrapped) coordinates; the sums at the thread's pixel are returned.
template <int RW, class FA, class FB>
__device__ __forceinline__ void window_sums2(float (*sa)[TX + 2 * RW], float (*sb)[TX + 2 * RW],
                                             int y0, int x0, FA fa, FB fb, float &ra, float &rb) {
    const int tid = threadIdx.y * TX + threadIdx.x;
    constexpr int GY = TY + 2 * RW, GX = TX + 2 * RW;
    for (int k = tid; k < GY * GX; k += TX * TY) {
        const int yy = k / GX, xx = k - (k / GX) * GX;
        sa[yy][xx] = fa(y0 - RW + yy, x0 - RW + xx);
        sb[yy][xx] = fb(y0 - RW + yy, x0 - RW + xx);
    }
    __syncthreads();
    float s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int dy = 0; dy <= 2 * RW; ++dy)
#pragma unroll
        for (int dx = 0; dx <= 2 * RW; ++dx) {
            s1 += sa[threadIdx.y + dy][threadIdx.x + dx];
            s2 += sb[threadIdx.y + dy][threadIdx.x + dx];
        }
    ra = s1;
    rb = s2;
}

// Pass 1: per window j the affine coefficients of alpha against the guide,
// a_j = (mean_j(I alpha) - mu_j mean_j(alpha)) s_j, b_j = mean_j(alpha) - a_j mu_j.
template <int RW>
__global__ void __launch_bounds__(TX * TY) prior_ab_kernel(const float *__restrict__ alpha,
                                                           const float4 *__restrict__ st4, int H,
                                                           int W, float *__restrict__ aout,
                                                           float *__restrict__ bout,
                                                           const CgBand *bands, const CgGlobal *g) {
    __shared__ float sa[TY + 2 * RW][TX + 2 * RW], sb[TY + 2 * RW][TX + 2 * RW];
    const int b = blockIdx.z;
    if (band_idle(bands, g, b)) return;
    const size_t HW = (size_t)H * W;
    const float *al = alpha + (size_t)b * HW;
    const int y0 = blockIdx.y * TY, x0 = blockIdx.x * TX;
    float s1, s2;
    window_sums2<RW>(
        sa, sb, y0, x0,
        [&](int y, int x) { return al[(size_t)wrapq(y, H) * W + wrapq(x, W)]; },
        [&](int y, int x) {
            const size_t o = (size_t)wrapq(y, H) * W + wrapq(x, W);
            return al[o] * st4[o].x;
        },
        s1, s2);
    const int y = y0 + threadIdx.y, x = x0 + threadIdx.x;
    if (y >= H || x >= W) return;
    constexpr float inw = 1.0f / (float)((2 * RW + 1) * (2 * RW + 1));
    const size_t o = (size_t)y * W + x;
    const float4 s = st4[o];
    const float ma = s1 * inw, mia = s2 * inw;
    const float av = (mia - s.y * ma) * s.z;
    aout[(size_t)b * HW + o] = av;
    bout[(size_t)b * HW + o] = ma - av * s.y;
}

// Pass 2: window sums Sa, Sb of the coefficients, then the matting matrix
// M alpha = |w| alpha - Sa I - Sb (gf = 0) or the guided filter
// (Sa I + Sb) / |w| (gf = 1), in place over alpha allowed.
template <int RW>
__global__ void __launch_bounds__(TX * TY) prior_m_kernel(const float *__restrict__ ain,
                                                          const float *__restrict__ bin,
                                                          const float *alpha,
                                                          const float4 *__restrict__ st4, int H,
                                                          int W, int gf, float *out,
                                                          const CgBand *bands, const CgGlobal *g) {
    __shared__ float sa[TY + 2 * RW][TX + 2 * RW], sb[TY + 2 * RW][TX + 2 * RW];
    const int b = blockIdx.z;
    if (band_idle(bands, g, b)) return;
    const size_t HW = (size_t)H * W;
    const float *A = ain + (size_t)b * HW, *B = bin + (size_t)b * HW;
    const int y0 = blockIdx.y * TY, x0 = blockIdx.x * TX;
    float s1, s2;
    window_sums2<RW>(
        sa, sb, y0, x0, [&](int y, int x) { return A[(size_t)wrapq(y, H) * W + wrapq(x, W)]; },
        [&](int y, int x) { return B[(size_t)wrapq(y, H) * W + wrapq(x, W)]; }, s1, s2);
    const int y = y0 + threadIdx.y, x = x0 + threadIdx.x;
    if (y >= H || x >= W) return;
    constexpr float nw = (float)((2 * RW + 1) * (2 * RW + 1));
    const size_t o = (size_t)y * W + x;
    const float I = st4[o].x;
    const size_t ob = (size_t)b * HW + o;
    out[ob] = gf ? (s1 * I + s2) / nw : nw * alpha[ob] - s1 * I - s2;
}

// Guide statistics of a given guide image G: (G, mean, 1/(var + eps), 0) per
// pixel over (2r+1)^2 torus windows, the window sums in FP64 (the E[G^2] -
// mean^2 difference cancels).
template <int RW>
__global__ void __launch_bounds__(TX * TY) guide_stats_kernel(const float *__restrict__ G, int H,
                                                              int W, float eps,
                                                              float4 *__restrict__ st4) {
    __shared__ double sg[TY + 2 * RW][TX + 2 * RW];
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int y0 = blockIdx.y * TY, x0 = blockIdx.x * TX;
    constexpr int GY = TY + 2 * RW, GX = TX + 2 * RW;
    for (int k = tid; k < GY * GX; k += TX * TY) {
        const int yy = k / GX, xx = k - (k / GX) * GX;
        sg[yy][xx] = (double)G[(size_t)wrapq(y0 - RW + yy, H) * W + wrapq(x0 - RW + xx, W)];
    }
    __syncthreads();
    const int y = y0 + threadIdx.y, x = x0 + threadIdx.x;
    if (y >= H || x >= W) return;
    double s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int dy = 0; dy <= 2 * RW; ++dy)
#pragma unroll
        for (int dx = 0; dx <= 2 * RW; ++dx) {
            const double v = sg[threadIdx.y + dy][threadIdx.x + dx];
            s1 += v;
            s2 += v * v;
        }
    constexpr double nw = (double)((2 * RW + 1) * (2 * RW + 1));
    const double m = s1 / nw, var = s2 / nw - m * m;
    st4[(size_t)y * W + x] =
        make_float4((float)sg[threadIdx.y + RW][threadIdx.x + RW], (float)m,
                    (float)(1.0 / (var + (double)eps)), 0.0f);
}

// q = lam (t0 + t1) and p^T q per band; the band's last CTA sets
// alpha = rho / (p^T q + ||D B p||^2), as the LLP kernel does in the CG loop.
__global__ void __launch_bounds__(256) prior_combine_kernel(const float4 *__restrict__ t0,
                                                            const float4 *__restrict__ t1,
                                                            const float4 *__restrict__ p,
                                                            float4 *__restrict__ q, size_t n4,
                                                            float lam, CgBand *bands,
                                                            const CgGlobal *g) {
    __shared__ double red[8];
    const int b = blockIdx.y;
    if (band_idle(bands, g, b)) return;
    const size_t off = (size_t)b * n4;
    double part = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x) {
        float4 v = t0[off + i];
        if (t1) {
            const float4 w = t1[off + i];
            v.x += w.x;
            v.y += w.y;
            v.z += w.z;
            v.w += w.w;
        }
        v.x *= lam;
        v.y *= lam;
        v.z *= lam;
        v.w *= lam;
        q[off + i] = v;
        if (bands) {
            const float4 pv = p[off + i];
            part += (double)(pv.x * v.x + pv.y * v.y + pv.z * v.z + pv.w * v.w);
        }
    }
    if (!bands) return;
    const double tot = block_sum_d(part, red);
    if (threadIdx.x != 0) return;
    CgBand *bd = bands + b;
    atomicAdd(&bd->pAp, tot);
    __threadfence();
    const unsigned int t = atomicAdd(&bd->cnt_apply, 1u);
    if (t != gridDim.x - 1) return;
    __threadfence();
    const double pAp = atomicAdd(&bd->pAp, 0.0) + bd->vv;
    bd->cnt_apply = 0u;
    if (!isfinite(pAp)) {
        bd->status = PS_ERR_NONFINITE;
        bd->done = 1;
        bd->alpha = 0.0;
    } else if (!(pAp > 0.0)) {
        bd->status = PS_ERR_BREAKDOWN;
        bd->done = 1;
        bd->alpha = 0.0;
    } else {
        bd->alpha = bd->rho / pAp;
    }
}

// The filters of a prior on (2 Rf + 1)^2 grids, tap (i, j) at
// (i + Rf) n + (j + Rf), from the blur kernel u ((2R+1)^2).
__global__ void prior_filters_kernel(const float *__restrict__ u, int R, int prior,
                                     float *__restrict__ f0, float *__restrict__ f1) {
    const int n = 2 * R + 1, nt = n * n;
    for (int k = threadIdx.x; k < nt; k += blockDim.x) {
        if (prior == PS_PRIOR_LPF) f0[k] = u[k];
        if (prior == PS_PRIOR_HPF) f0[k] = (k == R * n + R ? 1.0f : 0.0f) - u[k];
    }
    if (threadIdx.x == 0) {
        if (prior == PS_PRIOR_LPP) f0[0] = 1.0f;
        if (prior == PS_PRIOR_LGC) {
            // z(y, x) - z(y, x - 1) and z(y, x) - z(y - 1, x), 3 x 3
            for (int k = 0; k < 9; ++k) f0[k] = f1[k] = 0.0f;
            f0[4] = 1.0f;
            f0[5] = -1.0f;
            f1[4] = 1.0f;
            f1[7] = -1.0f;
        }
    }
}

// T += |F^|^2 (T FP64, [kx][ky] as the spectra).
__global__ void symbol_add_kernel(const double2 *__restrict__ fh, double *__restrict__ T,
                                  size_t n, int first) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const double2 v = fh[i];
        const double m = v.x * v.x + v.y * v.y;
        T[i] = first ? m : T[i] + m;
    }
}

// rhs = b + lam acc, packed two bands per FP64 complex image.
__global__ void prior_pack_kernel(const float *__restrict__ b, const float *__restrict__ acc,
                                  float lam, int N, size_t HW, double2 *__restrict__ out) {
    const int nimg = (N + 1) / 2;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)nimg * HW;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t k = i / HW, o = i - k * HW;
        const size_t o0 = (2 * k) * HW + o;
        const double re = (double)b[o0] + (double)lam * (double)acc[o0];
        double im = 0.0;
        if (2 * k + 1 < (size_t)N) {
            const size_t o1 = o0 + HW;
            im = (double)b[o1] + (double)lam * (double)acc[o1];
        }
        out[i] = make_double2(re, im);
    }
}

int grid_for(size_t n, int per) {
    size_t bl = (n + (size_t)per - 1) / (size_t)per;
    if (bl < 1) bl = 1;
    if (bl > 4096) bl = 4096;
    return (int)bl;
}

}  // namespace

int prior_filter_radius(int prior, int R) {
    switch (prior) {
        case PS_PRIOR_LPF:
        case PS_PRIOR_HPF: return R;
        case PS_PRIOR_LPP: return 0;
        case PS_PRIOR_LGC: return 1;
        default: return 1;
    }
}

int prior_filter_count(int prior) { return prior == PS_PRIOR_LGC ? 2 : 1; }

void launch_prior_filters(const float *u, int R, int prior, float *f0, float *f1,
                          cudaStream_t st) {
    prior_filters_kernel<<<1, 256, 0, st>>>(u, R, prior, f0, f1);
}

void launch_guide_stats(const float *G, int H, int W, int r, float eps, float4 *st4,
                        cudaStream_t st) {
    dim3 blk(TX, TY), grd((W + TX - 1) / TX, (H + TY - 1) / TY);
    switch (r) {
        case 1: guide_stats_kernel<1><<<grd, blk, 0, st>>>(G, H, W, eps, st4); break;
        case 2: guide_stats_kernel<2><<<grd, blk, 0, st>>>(G, H, W, eps, st4); break;
        case 3: guide_stats_kernel<3><<<grd, blk, 0, st>>>(G, H, W, eps, st4); break;
        default: guide_stats_kernel<4><<<grd, blk, 0, st>>>(G, H, W, eps, st4); break;
    }
}

void launch_prior_window(const float *alpha, const float4 *st4, int N, int H, int W, int r,
                         int gf, float *ta, float *tb, float *out, const CgBand *bands,
                         const CgGlobal *g, cudaStream_t st) {
    dim3 blk(TX, TY), grd((W + TX - 1) / TX, (H + TY - 1) / TY, N);
#define PS_WIN(RW)                                                                            \
    prior_ab_kernel<RW><<<grd, blk, 0, st>>>(alpha, st4, H, W, ta, tb, bands, g);            \
    prior_m_kernel<RW><<<grd, blk, 0, st>>>(ta, tb, alpha, st4, H, W, gf, out, bands, g);
    switch (r) {
        case 1: PS_WIN(1) break;
        case 2: PS_WIN(2) break;
        case 3: PS_WIN(3) break;
        default: PS_WIN(4) break;
    }
#undef PS_WIN
}

void launch_prior_combine(const float *t0, const float *t1, const float *p, float *q, int N,
                          size_t HW, float lam, CgBand *bands, const CgGlobal *g,
                          cudaStream_t st) {
    const size_t n4 = HW / 4;
    dim3 grd(grid_for(n4, 256 * 8), N);
    prior_combine_kernel<<<grd, 256, 0, st>>>(
        reinterpret_cast<const float4 *>(t0), reinterpret_cast<const float4 *>(t1),
        reinterpret_cast<const float4 *>(p), reinterpret_cast<float4 *>(q), n4, lam, bands, g);
}

void launch_symbol_add(const double2 *fh, double *T, size_t n, int first, cudaStream_t st) {
    symbol_add_kernel<<<grid_for(n, 256), 256, 0, st>>>(fh, T, n, first);
}

void launch_prior_pack(const float *b, const float *acc, float lam, int N, size_t HW,
                       double2 *out, cudaStream_t st) {
    prior_pack_kernel<<<grid_for((size_t)((N + 1) / 2) * HW, 256), 256, 0, st>>>(b, acc, lam, N,
                                                                                HW, out);
}

}  // namespace ps
