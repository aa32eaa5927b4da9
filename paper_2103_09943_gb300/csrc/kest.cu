// Blur kernel estimation (Algorithm 1), sm_103a.
//
//   omega      Eq. objective3: box filters, FP64 normal equations, tiny solve
//   E^T E      Eq. z_solution with E = D C(Y): E^T E[a, b] depends only on the
//              phase of a modulo c and on the lag a - b, so it is assembled
//              from c^2 (4R+1)^2 lag correlations of the PAN,
//              C[phi][d] = sum_k Y(c k + phi) Y(c k + phi + d),
//              accumulated in double-float (error-free products and sums in
//              FP32, the FP64 rate of this part being 1/64 of FP32)
//   Cholesky   of E^T E + mu3 I in FP64; z_f = (E^T E + mu3 I)^{-1} E^T f in
//              FP64 and Q = mu3 (E^T E + mu3 I)^{-1} (FP32, column-parallel),
//              so that the z step of Eq. z_solution is z_f + Q (u + Lambda3)
//   ADMM       the loop of Eq. subproblems in one CTA: shrink, z step with
//              simplex projection, {u, p} by n x n DFTs and Cramer's rule
//              (Eq. u_p_solution), multiplier updates, stop test
#include <math.h>


#include "common.cuh"
#include "kernels.cuh"

namespace ps {

__device__ __forceinline__ int wrapk(int i, int n) {
    int m = i % n;
    return m < 0 ? m + n : m;
}

// Error-free accumulation of a*b into (s, c): s + c carries ~48 bits.
__device__ __forceinline__ void df_acc(float a, float b, float &s, float &c) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float t = s + p;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (p - bp);
    s = t;
    c += err + e;
}

// ---------------------------------------------------------------------------
// omega (Eq. objective3)
// ---------------------------------------------------------------------------
BandSel band_sel(unsigned long long mask, int N) {
    BandSel s;
    s.n = 0;
    for (int b = 0; b < N && b < kMaxBands; ++b)
        if (!mask || ((mask >> b) & 1ull)) s.idx[s.n++] = (unsigned char)b;
    return s;
}

// B(u1) X'_z for the z-th selected band, into row z of `out`.
__global__ void box_lr_kernel(const float *__restrict__ X, BandSel sel, int h, int w, int l,
                              float *__restrict__ out) {
    const int z = blockIdx.z, b = sel.idx[z];
    const int y = blockIdx.y * 8 + threadIdx.y, x = blockIdx.x * 32 + threadIdx.x;
    if (y >= h || x >= w) return;
    const float *Xb = X + (size_t)b * h * w;
    float s = 0.f;
    for (int dy = -l; dy <= l; ++dy)
        for (int dx = -l; dx <= l; ++dx) s += Xb[(size_t)wrapk(y + dy, h) * w + wrapk(x + dx, w)];
    out[(size_t)z * h * w + (size_t)y * w + x] = s / (float)((2 * l + 1) * (2 * l + 1));
}

void launch_box_lr(const float *X, const BandSel &sel, int h, int w, int l, float *out,
                   cudaStream_t st) {
    dim3 blk(32, 8), grd((w + 31) / 32, (h + 7) / 8, sel.n);
    box_lr_kernel<<<grd, blk, 0, st>>>(X, sel, h, w, l, out);
}

// D B(u2) Y with u2 the (2 half + 1)^2 unit box: one thread per LR site.
__global__ void box_hr_dec_kernel(const float *__restrict__ Y, int H, int W, int c, int half,
                                  float *__restrict__ out) {
    const int h = H / c, w = W / c;
    const int k = blockIdx.y * 8 + threadIdx.y, l = blockIdx.x * 32 + threadIdx.x;
    if (k >= h || l >= w) return;
    float s = 0.f, cmp = 0.f;
    for (int dy = -half; dy <= half; ++dy) {
        const float *row = Y + (size_t)wrapk(c * k + dy, H) * W;
        for (int dx = -half; dx <= half; ++dx) df_acc(row[wrapk(c * l + dx, W)], 1.0f, s, cmp);
    }
    const double nb = (double)((2 * half + 1) * (2 * half + 1));
    out[(size_t)k * w + l] = (float)(((double)s + (double)cmp) / nb);
}

void launch_box_hr_dec(const float *Y, int H, int W, int c, int half, float *out,
                       cudaStream_t st) {
    const int h = H / c, w = W / c;
    dim3 blk(32, 8), grd((w + 31) / 32, (h + 7) / 8);
    box_hr_dec_kernel<<<grd, blk, 0, st>>>(Y, H, W, c, half, out);
}

// G[j][k] = sum_q A_j[q] A_k[q] (j <= k < N) and G[N][j] = sum_q A_j[q] bv[q];
// one CTA per entry, double-float accumulation.
__global__ void __launch_bounds__(256) omega_normal_kernel(const float *__restrict__ A,
                                                           const float *__restrict__ bv, int N,
                                                           int hw, double *G) {
    __shared__ double red[8];
    int e = blockIdx.x, j = 0, k = 0;
    bool rhs = false;
    const int npair = N * (N + 1) / 2;
    if (e < npair) {
        while (e >= N - j) { e -= N - j; ++j; }
        k = j + e;
    } else {
        rhs = true;
        j = e - npair;
    }
    const float *a = A + (size_t)j * hw;
    const float *bb = rhs ? bv : A + (size_t)k * hw;
    float s = 0.f, cmp = 0.f;
    for (int q = threadIdx.x; q < hw; q += 256) df_acc(a[q], bb[q], s, cmp);
    const double tot = block_sum_d((double)s + (double)cmp, red);
    if (threadIdx.x == 0) {
        if (rhs) {
            G[(size_t)N * N + j] = tot;
        } else {
            G[(size_t)j * N + k] = tot;
            G[(size_t)k * N + j] = tot;
        }
    }
}

void launch_omega_normal(const float *A, const float *bv, int N, int hw, double *G,
                         cudaStream_t st) {
    const int nblk = N * (N + 1) / 2 + N;
    omega_normal_kernel<<<nblk, 256, 0, st>>>(A, bv, N, hw, G);
}

// (A^T A + lambda_omega G^T G) omega = A^T b by Cholesky over the N'
// selected bands, one thread (N' <= 64); G holds the N' x N' normal matrix,
// G the first differences of consecutive selected weights. The weights go to
// their bands' slots of omega (N entries), zeros to the other bands.
__global__ void omega_solve_kernel(double *G, BandSel sel, int Nall, float lam, float *omega) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int N = sel.n;
    double *M = G;                 // N x N, overwritten
    double *rhs = G + (size_t)N * N;
    for (int i = 0; i < N; ++i) {
        // G^T G of first differences: diag 1, 2, ..., 2, 1; off-diagonal -1
        double d = (N == 1) ? 0.0 : ((i == 0 || i == N - 1) ? 1.0 : 2.0);
        M[(size_t)i * N + i] += lam * d;
        if (i + 1 < N) {
            M[(size_t)i * N + i + 1] -= lam;
            M[(size_t)(i + 1) * N + i] -= lam;
        }
    }
    for (int k = 0; k < N; ++k) {
        double dkk = M[(size_t)k * N + k];
        for (int t = 0; t < k; ++t) dkk -= M[(size_t)k * N + t] * M[(size_t)k * N + t];
        const double lkk = sqrt(dkk > 0.0 ? dkk : 1e-300);
        M[(size_t)k * N + k] = lkk;
        for (int i = k + 1; i < N; ++i) {
            double v = M[(size_t)i * N + k];
            for (int t = 0; t < k; ++t) v -= M[(size_t)i * N + t] * M[(size_t)k * N + t];
            M[(size_t)i * N + k] = v / lkk;
        }
    }
    for (int i = 0; i < N; ++i) {
        double v = rhs[i];
        for (int t = 0; t < i; ++t) v -= M[(size_t)i * N + t] * rhs[t];
        rhs[i] = v / M[(size_t)i * N + i];
    }
    for (int i = N - 1; i >= 0; --i) {
        double v = rhs[i];
        for (int t = i + 1; t < N; ++t) v -= M[(size_t)t * N + i] * rhs[t];
        rhs[i] = v / M[(size_t)i * N + i];
    }
    for (int b = 0; b < Nall; ++b) omega[b] = 0.f;
    for (int i = 0; i < N; ++i) omega[sel.idx[i]] = (float)rhs[i];
}

void launch_omega_solve(double *G, const BandSel &sel, int N, float lambda_omega, float *omega,
                        cudaStream_t st) {
    omega_solve_kernel<<<1, 32, 0, st>>>(G, sel, N, lambda_omega, omega);
}

// Given weights restricted to X': out[b] = in[b] for the bands of the mask
// (all when 0), 0 for the others (in and out may be the same array).
__global__ void omega_mask_kernel(const float *in, unsigned long long mask, int N, float *out) {
    const int b = threadIdx.x;
    if (b < N) out[b] = (!mask || ((mask >> b) & 1ull)) ? in[b] : 0.f;
}

void launch_omega_mask(const float *in, unsigned long long mask, int N, float *out,
                       cudaStream_t st) {
    omega_mask_kernel<<<1, 64, 0, st>>>(in, mask, N, out);
}

__global__ void combine_f_kernel(const float *__restrict__ X, const float *__restrict__ om,
                                 int N, int hw, float *__restrict__ f) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= hw) return;
    float s = 0.f;
    for (int b = 0; b < N; ++b) s = fmaf(om[b], X[(size_t)b * hw + q], s);
    f[q] = s;
}

void launch_combine_f(const float *X, const float *omega, int N, int hw, float *f,
                      cudaStream_t st) {
    combine_f_kernel<<<(hw + 255) / 256, 256, 0, st>>>(X, omega, N, hw, f);
}

// ---------------------------------------------------------------------------
// E^T E from lag correlations
// ---------------------------------------------------------------------------
constexpr int LAG_CHUNK = 17;

// grid: (2R+1 dy >= 0, c*c phases, ceil((4R+1)/LAG_CHUNK) dx chunks)
// lags[((py*c + px) * (4R+1) + (dy+2R)) * (4R+1) + (dx+2R)]; the rows dy < 0
// follow from C[phi][d] = C[(phi + d) mod c][-d] (E^T E is symmetric) and are
// read through that identity by ete_assemble_kernel.
__global__ void __launch_bounds__(256) ete_lag_kernel(const float *__restrict__ Y, int H, int W,
                                                      int c, int R, double *lags) {
    __shared__ double red[8];
    const int nl = 4 * R + 1;
    const int dy = (int)blockIdx.x;                      // 0 .. 2R
    const int py = blockIdx.y / c, px = blockIdx.y - (blockIdx.y / c) * c;
    const int dx0 = (int)blockIdx.z * LAG_CHUNK - 2 * R;
    const int ndx = min(LAG_CHUNK, 2 * R - dx0 + 1);
    const int h = H / c, w = W / c;
    float s[LAG_CHUNK], cm[LAG_CHUNK];
#pragma unroll
    for (int t = 0; t < LAG_CHUNK; ++t) { s[t] = 0.f; cm[t] = 0.f; }
    int ky = 0, kx = threadIdx.x;
    while (kx >= w) { kx -= w; ++ky; }
    for (; ky < h;) {
        const int yy = c * ky + py, xx = c * kx + px;
        const float a = Y[(size_t)yy * W + xx];
        const float *row = Y + (size_t)wrapk(yy + dy, H) * W;
        const int cx0 = xx + dx0;
        if (cx0 >= 0 && cx0 + LAG_CHUNK <= W) {
            const float *seg = row + cx0;
#pragma unroll
            for (int t = 0; t < LAG_CHUNK; ++t) df_acc(a, seg[t], s[t], cm[t]);
        } else {
            int cx = cx0 < 0 ? cx0 + W : (cx0 >= W ? cx0 - W : cx0);
#pragma unroll
            for (int t = 0; t < LAG_CHUNK; ++t) {
                df_acc(a, row[cx], s[t], cm[t]);
                cx = (cx + 1 == W) ? 0 : cx + 1;
            }
        }
        kx += 256;
        while (kx >= w) { kx -= w; ++ky; }
    }
#pragma unroll
    for (int t = 0; t < LAG_CHUNK; ++t) {
        if (t < ndx) {
            const double tot = block_sum_d((double)s[t] + (double)cm[t], red);
            if (threadIdx.x == 0)
                lags[((size_t)blockIdx.y * nl + (dy + 2 * R)) * nl + (dx0 + t + 2 * R)] = tot;
        }
    }
}

// The same sums for a compile-time ratio C, LAG_SITES horizontally adjacent LR
// sites per thread: their row segments overlap in all but C (LAG_SITES - 1)
// samples, so one register copy of the union (LAG_CHUNK + C (LAG_SITES - 1)
// values) feeds LAG_SITES x LAG_CHUNK products, about half the loads of the
// one-site walk.
constexpr int LAG_SITES = 4;

// The walk over the CTA's LR sites. OFF = (px + dx0) mod 4 is the same for
// every site group of a CTA (C kx0 is a multiple of 4), so with a 16-byte
// aligned PAN a group's row segment is NV aligned float4 loads shifted by
// OFF: a warp's load instruction touches the same 16 cache lines for four
// values as a scalar load does for one.
template <int C, int OFF>
__device__ __forceinline__ void lag_sites_walk(const float *__restrict__ Y, int H, int W, int py,
                                               int px, int dy, int dx0, int h, int w, int gw,
                                               bool vec, float (&s)[LAG_CHUNK],
                                               float (&cm)[LAG_CHUNK]) {
    constexpr int SEG = LAG_CHUNK + C * (LAG_SITES - 1);
    constexpr int NV = (SEG + OFF + 3) / 4;
    for (int gi = threadIdx.x; gi < h * gw; gi += 256) {
        const int ky = gi / gw, kx0 = (gi - ky * gw) * LAG_SITES;
        const int yy = C * ky + py;
        const float *arow = Y + (size_t)yy * W;
        const float *row = Y + (size_t)wrapk(yy + dy, H) * W;
        const int cx0 = C * kx0 + px + dx0;
        const int base = cx0 - OFF;
        float seg[SEG];
        if (vec && base >= 0 && base + 4 * NV <= W) {
            float v[4 * NV];
            const float4 *rv = reinterpret_cast<const float4 *>(row + base);
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const float4 q = __ldg(rv + k);
                v[4 * k] = q.x;
                v[4 * k + 1] = q.y;
                v[4 * k + 2] = q.z;
                v[4 * k + 3] = q.w;
            }
#pragma unroll
            for (int t = 0; t < SEG; ++t) seg[t] = v[t + OFF];
        } else if (cx0 >= 0 && cx0 + SEG <= W) {
#pragma unroll
            for (int t = 0; t < SEG; ++t) seg[t] = row[cx0 + t];
        } else {
            int cx = wrapk(cx0, W);
#pragma unroll
            for (int t = 0; t < SEG; ++t) {
                seg[t] = row[cx];
                cx = (cx + 1 == W) ? 0 : cx + 1;
            }
        }
#pragma unroll
        for (int q = 0; q < LAG_SITES; ++q) {
            if (kx0 + q >= w) break;
            const float a = arow[C * (kx0 + q) + px];
#pragma unroll
            for (int t = 0; t < LAG_CHUNK; ++t) df_acc(a, seg[C * q + t], s[t], cm[t]);
        }
    }
}

template <int C>
__global__ void __launch_bounds__(256) ete_lag_sites_kernel(const float *__restrict__ Y, int H,
                                                            int W, int R, int vec,
                                                            double *lags) {
    __shared__ double red[8];
    const int nl = 4 * R + 1;
    const int dy = (int)blockIdx.x;
    const int py = blockIdx.y / C, px = blockIdx.y - (blockIdx.y / C) * C;
    const int dx0 = (int)blockIdx.z * LAG_CHUNK - 2 * R;
    const int ndx = min(LAG_CHUNK, 2 * R - dx0 + 1);
    const int h = H / C, w = W / C;
    const int gw = (w + LAG_SITES - 1) / LAG_SITES;   // site groups per LR row
    float s[LAG_CHUNK], cm[LAG_CHUNK];
#pragma unroll
    for (int t = 0; t < LAG_CHUNK; ++t) { s[t] = 0.f; cm[t] = 0.f; }
    const bool v = vec != 0;
    switch (((px + dx0) % 4 + 4) % 4) {
        case 0: lag_sites_walk<C, 0>(Y, H, W, py, px, dy, dx0, h, w, gw, v, s, cm); break;
        case 1: lag_sites_walk<C, 1>(Y, H, W, py, px, dy, dx0, h, w, gw, v, s, cm); break;
        case 2: lag_sites_walk<C, 2>(Y, H, W, py, px, dy, dx0, h, w, gw, v, s, cm); break;
        default: lag_sites_walk<C, 3>(Y, H, W, py, px, dy, dx0, h, w, gw, v, s, cm); break;
    }
#pragma unroll
    for (int t = 0; t < LAG_CHUNK; ++t) {
        if (t < ndx) {
            const double tot = block_sum_d((double)s[t] + (double)cm[t], red);
            if (threadIdx.x == 0)
                lags[((size_t)blockIdx.y * nl + (dy + 2 * R)) * nl + (dx0 + t + 2 * R)] = tot;
        }
    }
}

void launch_ete_lags(const float *Y, int H, int W, int c, int R, double *lags,
                     cudaStream_t st) {
    const int nl = 4 * R + 1;
    dim3 grd(2 * R + 1, c * c, (nl + LAG_CHUNK - 1) / LAG_CHUNK);
    const int vec = ((uintptr_t)Y % 16) == 0 && W % 4 == 0;
    if (c == 4)
        ete_lag_sites_kernel<4><<<grd, 256, 0, st>>>(Y, H, W, R, vec, lags);
    else if (c == 2)
        ete_lag_sites_kernel<2><<<grd, 256, 0, st>>>(Y, H, W, R, vec, lags);
    else
        ete_lag_kernel<<<grd, 256, 0, st>>>(Y, H, W, c, R, lags);
}

// E^T E[a][b] = C[(-a) mod c][a - b], taps a = (ai, aj), b = (bi, bj).
__global__ void ete_assemble_kernel(const double *__restrict__ lags, int c, int R,
                                    double *EtE) {
    const int n = 2 * R + 1, nt = n * n, nl = 4 * R + 1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nt * nt) return;
    const int ia = idx / nt, ib = idx - (idx / nt) * nt;
    const int ai = ia / n - R, aj = ia % n - R, bi = ib / n - R, bj = ib % n - R;
    int py = wrapk(-ai, c), px = wrapk(-aj, c);
    int dy = ai - bi, dx = aj - bj;
    if (dy < 0) {  // C[phi][d] = C[(phi + d) mod c][-d]
        py = wrapk(py + dy, c);
        px = wrapk(px + dx, c);
        dy = -dy;
        dx = -dx;
    }
    EtE[idx] = lags[((size_t)(py * c + px) * nl + (dy + 2 * R)) * nl + (dx + 2 * R)];
}

void launch_ete_assemble(const double *lags, int c, int R, double *EtE, cudaStream_t st) {
    const int nt = (2 * R + 1) * (2 * R + 1);
    ete_assemble_kernel<<<(nt * nt + 255) / 256, 256, 0, st>>>(lags, c, R, EtE);
}

// E^T f[a] = sum_q Y(c q - a) f_q, one CTA per tap.
__global__ void __launch_bounds__(256) etf_kernel(const float *__restrict__ Y, int H, int W,
                                                  int c, int R, const float *__restrict__ f,
                                                  double *Etf) {
    __shared__ double red[8];
    const int n = 2 * R + 1;
    const int ai = (int)blockIdx.x / n - R, aj = (int)blockIdx.x % n - R;
    const int h = H / c, w = W / c;
    float s = 0.f, cm = 0.f;
    int ky = 0, kx = threadIdx.x;
    while (kx >= w) { kx -= w; ++ky; }
    for (; ky < h;) {
        df_acc(Y[(size_t)wrapk(c * ky - ai, H) * W + wrapk(c * kx - aj, W)],
               f[(size_t)ky * w + kx], s, cm);
        kx += 256;
        while (kx >= w) { kx -= w; ++ky; }
    }
    const double tot = block_sum_d((double)s + (double)cm, red);
    if (threadIdx.x == 0) Etf[blockIdx.x] = tot;
}

void launch_etf(const float *Y, int H, int W, int c, int R, const float *f, double *Etf,
                cudaStream_t st) {
    const int nt = (2 * R + 1) * (2 * R + 1);
    etf_kernel<<<nt, 256, 0, st>>>(Y, H, W, c, R, f, Etf);
}

// ---------------------------------------------------------------------------
// FP64 Cholesky of A + mu3 I (lower triangle, in place), blocked right-looking
// over 32-column panels: per panel one CTA factors the diagonal tile and
// solves the rows below it, then one CTA per trailing tile applies the
// rank-32 update. A is nt x nt row-major.
// ---------------------------------------------------------------------------
constexpr int CB = 32;

__global__ void add_diag_kernel(double *A, int n, float mu3) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) A[(size_t)i * n + i] += (double)mu3;
}

// Factor the 32 x 32 diagonal tile of panel k0 in place. Four warps, lane i
// of each holding row i; warp w holds the columns j = w (mod 4) in
// registers, so that the FP64 work of the rank-1 updates (the pipe is 1/64
// of the FP32 rate on this part) spreads over four schedulers. Right-looking:
// per column k the owning warp takes the pivot from lane k,
// l_kk = d_kk rsqrt(d_kk), scales the rows below by rsqrt(d_kk) and
// publishes the column in shared memory; then every warp updates its own
// columns j > k by -= l_ik l_jk.
constexpr int kDiagWarps = 4;

__global__ void __launch_bounds__(32 * kDiagWarps) chol_diag_kernel(double *A, int nt, int k0) {
    constexpr int CPW = CB / kDiagWarps;
    __shared__ double col[CB];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int kb = min(CB, nt - k0);
    double x[CPW];
    const double *row = A + (size_t)(k0 + lane) * nt + k0;
#pragma unroll
    for (int m = 0; m < CPW; ++m) {
        const int j = w + kDiagWarps * m;
        x[m] = (lane < kb && j < kb) ? ((j <= lane) ? row[j] : 0.0) : (lane == j ? 1.0 : 0.0);
    }
#pragma unroll
    for (int k = 0; k < CB; ++k) {
        const int mk = k / kDiagWarps;
        if (w == k % kDiagWarps) {
            const double dkk = __shfl_sync(0xffffffffu, x[mk], k);
            const double rs = rsqrt(dkk > 0.0 ? dkk : 1e-300);
            double v = x[mk];
            if (lane == k) v = dkk * rs;
            else if (lane > k) v *= rs;
            x[mk] = v;
            col[lane] = v;
        }
        __syncthreads();
        const double lik = col[lane];
#pragma unroll
        for (int m = 0; m < CPW; ++m) {
            const int j = w + kDiagWarps * m;
            if (j > k) {
                const double ljk = col[j];
                if (lane >= j) x[m] -= lik * ljk;
            }
        }
        __syncthreads();
    }
    if (lane < kb) {
        double *out = A + (size_t)(k0 + lane) * nt + k0;
#pragma unroll
        for (int m = 0; m < CPW; ++m) {
            const int j = w + kDiagWarps * m;
            if (j < kb && j <= lane) out[j] = x[m];
        }
    }
}

// Rows below the diagonal tile: L[i][k0 + k] = (A[i][k0+k] - sum_{m<k}
// L[i][k0+m] D[k][m]) / D[k][k]; one warp per 32 rows, one row per lane.
__global__ void __launch_bounds__(32) chol_panel_kernel(double *A, int nt, int k0) {
    __shared__ double D[CB][CB + 1];
    const int lane = threadIdx.x;
    const int k1 = min(k0 + CB, nt), kb = k1 - k0;
    for (int e = lane; e < CB * CB; e += 32) {
        const int i = e / CB, j = e - (e / CB) * CB;
        double v;
        if (i < kb && j < kb) v = (j <= i) ? A[(size_t)(k0 + i) * nt + k0 + j] : 0.0;
        else v = (i == j) ? 1.0 : 0.0;
        D[i][j] = v;
    }
    __shared__ double rdiag[CB];
    __syncwarp();
    rdiag[lane] = 1.0 / D[lane][lane];
    __syncwarp();
    const int i = k1 + blockIdx.x * 32 + lane;
    if (i >= nt) return;
    double x[CB];
    double *row = A + (size_t)i * nt + k0;
#pragma unroll
    for (int k = 0; k < CB; ++k) x[k] = (k < kb) ? row[k] : 0.0;
#pragma unroll
    for (int k = 0; k < CB; ++k) {
        double v = x[k];
#pragma unroll
        for (int m = 0; m < k; ++m) v -= x[m] * D[k][m];
        x[k] = v * rdiag[k];
    }
#pragma unroll
    for (int k = 0; k < CB; ++k)
        if (k < kb) row[k] = x[k];
}

// Trailing update A[I][J] -= L[I][K] L[J][K]^T over tiles I >= J of the
// trailing matrix (one CTA per tile pair).
__global__ void __launch_bounds__(256) chol_update_kernel(double *A, int nt, int k0) {
    __shared__ double Li[CB][CB + 1], Lj[CB][CB + 1];
    const int k1 = min(k0 + CB, nt), kb = k1 - k0;
    int e = blockIdx.x, ti = 0;
    while (e > ti) { e -= ti + 1; ++ti; }
    const int tj = e;
    const int i0 = k1 + ti * CB, j0 = k1 + tj * CB;
    const int tid = threadIdx.x;
    for (int q = tid; q < CB * CB; q += blockDim.x) {
        const int r = q / CB, k = q - (q / CB) * CB;
        Li[r][k] = (i0 + r < nt && k < kb) ? A[(size_t)(i0 + r) * nt + k0 + k] : 0.0;
        Lj[r][k] = (j0 + r < nt && k < kb) ? A[(size_t)(j0 + r) * nt + k0 + k] : 0.0;
    }
    __syncthreads();
    for (int q = tid; q < CB * CB; q += blockDim.x) {
        const int r = q / CB, cc = q - (q / CB) * CB;
        const int i = i0 + r, j = j0 + cc;
        if (i >= nt || j >= nt || j > i) continue;
        double acc = 0.0;
#pragma unroll 8
        for (int k = 0; k < CB; ++k) acc += Li[r][k] * Lj[cc][k];
        A[(size_t)i * nt + j] -= acc;
    }
}

void launch_cholesky(double *A, int n, float mu3, cudaStream_t st) {
    add_diag_kernel<<<(n + 255) / 256, 256, 0, st>>>(A, n, mu3);
    for (int k0 = 0; k0 < n; k0 += CB) {
        chol_diag_kernel<<<1, 32 * kDiagWarps, 0, st>>>(A, n, k0);
        const int rem = n - (k0 + CB);
        if (rem > 0) {
            chol_panel_kernel<<<(rem + 31) / 32, 32, 0, st>>>(A, n, k0);
            const int nbt = (rem + CB - 1) / CB;
            chol_update_kernel<<<nbt * (nbt + 1) / 2, 256, 0, st>>>(A, n, k0);
        }
    }
}

// Solve (L L^T) x = b for `ncol` right-hand sides, one CTA per column; the
// rhs of column j is b (ncol == 1) or e_j scaled (the inverse). Forward
// substitution by 32-row tiles: the rows of a tile take their dot products
// with the solved part in parallel (one warp per row, coalesced rows of L),
// then one warp finishes the tile's triangle. Backward substitution on L^T by
// tiles from the bottom: one warp solves the tile, then all threads update
// the unknowns above from the tile's rows of L (coalesced).
__device__ void chol_two_solves(const double *L, int nt, double *y, double *Dt) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    constexpr unsigned FULLM = 0xffffffffu;
    for (int t0 = 0; t0 < nt; t0 += CB) {
        const int kb = min(CB, nt - t0);
        for (int r = warp; r < kb; r += nwarp) {
            const double *row = L + (size_t)(t0 + r) * nt;
            double acc = 0.0;
            for (int k = lane; k < t0; k += 32) acc += row[k] * y[k];
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULLM, acc, o);
            if (lane == 0) y[t0 + r] -= acc;
        }
        for (int q = tid; q < kb * kb; q += blockDim.x) {
            const int r = q / kb, k = q - (q / kb) * kb;
            Dt[r * CB + k] = (k <= r) ? L[(size_t)(t0 + r) * nt + t0 + k] : 0.0;
        }
        __syncthreads();
        if (warp == 0) {
            // column-oriented: lane k holds y_k; x_r = y_r / L_rr, then every
            // later row subtracts its L[k][r] x_r
            const double rinv = lane < kb ? 1.0 / Dt[lane * CB + lane] : 0.0;
            double yk = lane < kb ? y[t0 + lane] : 0.0;
            for (int r = 0; r < kb; ++r) {
                const double xr = __shfl_sync(FULLM, yk * rinv, r);
                if (lane == r) yk = xr;
                else if (lane > r && lane < kb) yk = fma(-Dt[lane * CB + r], xr, yk);
            }
            if (lane < kb) y[t0 + lane] = yk;
        }
        __syncthreads();
    }
    const int ntile = (nt + CB - 1) / CB;
    for (int tt = ntile - 1; tt >= 0; --tt) {
        const int t0 = tt * CB, kb = min(CB, nt - t0);
        for (int q = tid; q < kb * kb; q += blockDim.x) {
            const int r = q / kb, k = q - (q / kb) * kb;
            Dt[r * CB + k] = (k <= r) ? L[(size_t)(t0 + r) * nt + t0 + k] : 0.0;
        }
        __syncthreads();
        if (warp == 0) {
            // L^T x = y on the tile, from its last row up: x_r = y_r / L_rr,
            // then rows k < r subtract L[r][k] x_r
            const double rinv = lane < kb ? 1.0 / Dt[lane * CB + lane] : 0.0;
            double yk = lane < kb ? y[t0 + lane] : 0.0;
            for (int r = kb - 1; r >= 0; --r) {
                const double xr = __shfl_sync(FULLM, yk * rinv, r);
                if (lane == r) yk = xr;
                else if (lane < r) yk = fma(-Dt[r * CB + lane], xr, yk);
            }
            if (lane < kb) y[t0 + lane] = yk;
        }
        __syncthreads();
        for (int i = tid; i < t0; i += blockDim.x) {
            double acc = 0.0;
            for (int k = 0; k < kb; ++k) acc += L[(size_t)(t0 + k) * nt + i] * y[t0 + k];
            y[i] -= acc;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) chol_solve_kernel(const double *L, const double *b,
                                                         int n, double *x) {
    extern __shared__ double ysm[];
    double *y = ysm, *Dt = ysm + ((n + 1) & ~1);
    for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = b[i];
    __syncthreads();
    chol_two_solves(L, n, y, Dt);
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = y[i];
}

void launch_chol_solve(const double *L, const double *b, int n, double *x, cudaStream_t st) {
    const size_t sm = (((n + 1) & ~1) + CB * CB) * sizeof(double);
    chol_solve_kernel<<<1, 256, sm, st>>>(L, b, n, x);
}

// Q[:, j] = scale (L L^T)^{-1} e_j, one CTA per column (Q is symmetric).
__global__ void __launch_bounds__(256) chol_inverse_kernel(const double *L, int n, float scale,
                                                           float *Q) {
    extern __shared__ double ysm[];
    double *y = ysm, *Dt = ysm + ((n + 1) & ~1);
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = (i == j) ? 1.0 : 0.0;
    __syncthreads();
    chol_two_solves(L, n, y, Dt);
    for (int i = threadIdx.x; i < n; i += blockDim.x) Q[(size_t)i * n + j] = (float)(scale * y[i]);
}

void launch_chol_inverse(const double *L, int n, float scale, float *Q, double *,
                         cudaStream_t st) {
    const size_t sm = (((n + 1) & ~1) + CB * CB) * sizeof(double);
    chol_inverse_kernel<<<n, 256, sm, st>>>(L, n, scale, Q);
}

// ---------------------------------------------------------------------------
// ADMM loop (Algorithm 1), one CTA of 1024 threads, state in shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 c_div(float2 a, float2 b) {
    const float d = b.x * b.x + b.y * b.y;
    return make_float2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ float2 det3c(float2 a11, float2 a12, float2 a13, float2 a21, float2 a22,
                                        float2 a23, float2 a31, float2 a32, float2 a33) {
    float2 r = c_mul(c_mul(a11, a22), a33);
    r = c_add(r, c_mul(c_mul(a12, a23), a31));
    r = c_add(r, c_mul(c_mul(a13, a21), a32));
    r = c_sub(r, c_mul(c_mul(a13, a22), a31));
    r = c_sub(r, c_mul(c_mul(a12, a21), a33));
    r = c_sub(r, c_mul(c_mul(a11, a32), a23));
    return r;
}

// Block sums (double) of two values; all threads receive the results.
// Block-wide sums of two floats by a pairwise tree (warp shuffles, then one
// warp over the warp sums): the result is valid in every thread.
__device__ __forceinline__ void block_sum2f(float a, float b, double *red, float &ra, float &rb) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    float *rf = reinterpret_cast<float *>(red);
    const int tid = threadIdx.x, nw = blockDim.x >> 5;
    __syncthreads();
    if ((tid & 31) == 0) {
        rf[tid >> 5] = a;
        rf[32 + (tid >> 5)] = b;
    }
    __syncthreads();
    if (tid < 32) {
        float sa = (tid < nw) ? rf[tid] : 0.f, sb = (tid < nw) ? rf[32 + tid] : 0.f;
        for (int o = 16; o > 0; o >>= 1) {
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            sb += __shfl_xor_sync(0xffffffffu, sb, o);
        }
        if (tid == 0) {
            rf[64] = sa;
            rf[65] = sb;
        }
    }
    __syncthreads();
    ra = rf[64];
    rb = rf[65];
}

__device__ __forceinline__ void block_sum2(double a, double b, double *red, double &ra,
                                           double &rb) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int tid = threadIdx.x, nw = blockDim.x >> 5;
    __syncthreads();
    if ((tid & 31) == 0) {
        red[tid >> 5] = a;
        red[32 + (tid >> 5)] = b;
    }
    __syncthreads();
    if (tid < 32) {
        double sa = (tid < nw) ? red[tid] : 0.0, sb = (tid < nw) ? red[32 + tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            sb += __shfl_xor_sync(0xffffffffu, sb, o);
        }
        if (tid == 0) {
            red[64] = sa;
            red[65] = sb;
        }
    }
    __syncthreads();
    ra = red[64];
    rb = red[65];
}

// 2-D DFT of three real n x n arrays (sg = -1) or inverse of three complex
// spectra to real arrays (sg = +1, scaled by 1/n^2).
// NC > 0: n = NC known at compile time (divisions by n become multiplies,
// the tap loops unroll); NC = 0: n = n_rt.
template <int NC>
__device__ __forceinline__ void dft3_forward(const float *a0, const float *a1, const float *a2,
                                             float2 *T0, float2 *T1, float2 *T2, float2 *F0,
                                             float2 *F1, float2 *F2, const float2 *tw,
                                             int n_rt) {
    const int n = NC ? NC : n_rt;
    const int nt = n * n;
    for (int k = threadIdx.x; k < 3 * nt; k += blockDim.x) {
        const int which = k / nt, e = k - which * nt;
        const int i = e / n, kx = e - (e / n) * n;
        const float *a = which == 0 ? a0 : (which == 1 ? a1 : a2);
        float2 acc = make_float2(0.f, 0.f);
        for (int j = 0, ix = 0; j < n; ++j) {
            const float2 wv = tw[ix];
            const float v = a[i * n + j];
            acc.x += v * wv.x;
            acc.y += v * wv.y;
            ix += kx;
            if (ix >= n) ix -= n;
        }
        (which == 0 ? T0 : (which == 1 ? T1 : T2))[e] = acc;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * nt; k += blockDim.x) {
        const int which = k / nt, e = k - which * nt;
        const int ky = e / n, kx = e - (e / n) * n;
        const float2 *T = which == 0 ? T0 : (which == 1 ? T1 : T2);
        float2 acc = make_float2(0.f, 0.f);
        for (int i = 0, ix = 0; i < n; ++i) {
            acc = c_add(acc, c_mul(T[i * n + kx], tw[ix]));
            ix += ky;
            if (ix >= n) ix -= n;
        }
        (which == 0 ? F0 : (which == 1 ? F1 : F2))[e] = acc;
    }
    __syncthreads();
}

template <int NC>
__device__ __forceinline__ void dft3_inverse(const float2 *F0, const float2 *F1,
                                             const float2 *F2, float2 *T0, float2 *T1,
                                             float2 *T2, float *o0, float *o1, float *o2,
                                             const float2 *tw, int n_rt) {
    const int n = NC ? NC : n_rt;
    const int nt = n * n;
    for (int k = threadIdx.x; k < 3 * nt; k += blockDim.x) {
        const int which = k / nt, e = k - which * nt;
        const int i = e / n, kx = e - (e / n) * n;
        const float2 *F = which == 0 ? F0 : (which == 1 ? F1 : F2);
        float2 acc = make_float2(0.f, 0.f);
        for (int ky = 0, ix = 0; ky < n; ++ky) {
            acc = c_add(acc, c_mul(F[ky * n + kx], c_conj(tw[ix])));
            ix += i;
            if (ix >= n) ix -= n;
        }
        (which == 0 ? T0 : (which == 1 ? T1 : T2))[e] = acc;
    }
    __syncthreads();
    const float inv = 1.0f / (float)nt;
    for (int k = threadIdx.x; k < 3 * nt; k += blockDim.x) {
        const int which = k / nt, e = k - which * nt;
        const int i = e / n, j = e - (e / n) * n;
        const float2 *T = which == 0 ? T0 : (which == 1 ? T1 : T2);
        float acc = 0.f;
        for (int kx = 0, ix = 0; kx < n; ++kx) {
            const float2 wv = c_conj(tw[ix]);
            const float2 tv = T[i * n + kx];
            acc += tv.x * wv.x - tv.y * wv.y;
            ix += j;
            if (ix >= n) ix -= n;
        }
        (which == 0 ? o0 : (which == 1 ? o1 : o2))[e] = acc * inv;
    }
    __syncthreads();
}

size_t admm_state_bytes(int R) {
    const int nt = (2 * R + 1) * (2 * R + 1);
    const size_t ntp = (nt + 3) & ~3;
    return 26 * ntp * sizeof(float) + (6 * ntp + 64) * sizeof(float2) + 80 * sizeof(double) +
           16;
}

constexpr size_t kAdmmMaxSmem = 227 * 1024;

// Q (nt x nt, FP32) after the state, when the whole fits in shared memory
// (n <= 13); larger kernels read it from global memory, where it stays in
// L1 and L2 across the iterations.
__host__ __device__ inline bool admm_q_fits(int R, size_t state) {
    const size_t nt = (size_t)(2 * R + 1) * (2 * R + 1);
    return state + nt * nt * sizeof(float) <= kAdmmMaxSmem;
}

size_t admm_smem_bytes(int R) {
    const size_t st = admm_state_bytes(R);
    const size_t nt = (size_t)(2 * R + 1) * (2 * R + 1);
    return admm_q_fits(R, st) ? st + nt * nt * sizeof(float) : st;
}

__device__ __forceinline__ bool admm_q_in_smem(int R) {
    const int nt = (2 * R + 1) * (2 * R + 1);
    const size_t ntp = (nt + 3) & ~3;
    const size_t state = 26 * ntp * sizeof(float) + (6 * ntp + 64) * sizeof(float2) +
                         80 * sizeof(double) + 16;
    return admm_q_fits(R, state);
}

// NC > 0: compiled for the kernel side n = 2R + 1 = NC (every index
// division by n or n^2 becomes a multiply); NC = 0: any R.
template <int NC>
__global__ void __launch_bounds__(1024) admm_kernel(const float *__restrict__ Q,
                                                    const double *__restrict__ zf, int R,
                                                    ps_kernel_params p, float *kernel_out,
                                                    int *info_iters, int *info_status,
                                                    double *info_change) {
    extern __shared__ __align__(16) unsigned char admm_sm[];
    const int n = NC ? NC : 2 * R + 1, nt = n * n;
    const int ntp = (nt + 3) & ~3;
    const int tid = threadIdx.x, nthr = blockDim.x;
    double *red = reinterpret_cast<double *>(admm_sm);
    float2 *cbase = reinterpret_cast<float2 *>(admm_sm + 80 * sizeof(double));
    float2 *F0 = cbase, *F1 = F0 + ntp, *F2 = F1 + ntp, *T0 = F2 + ntp, *T1 = T0 + ntp,
           *T2 = T1 + ntp, *tw = T2 + ntp;
    float *fb = reinterpret_cast<float *>(tw + 64);
    float *u = fb, *un = u + ntp, *p1 = un + ntp, *p2 = p1 + ntp, *x0 = p2 + ntp, *x1 = x0 + ntp,
          *y0 = x1 + ntp, *y1 = y0 + ntp, *y2 = y1 + ntp, *y3 = y2 + ntp, *l10 = y3 + ntp,
          *l11 = l10 + ntp, *l20 = l11 + ntp, *l21 = l20 + ntp, *l22 = l21 + ntp,
          *l23 = l22 + ntp, *l3 = l23 + ntp, *z = l3 + ntp, *zs = z + ntp, *wv = zs + ntp,
          *t0 = wv + ntp, *t1 = t0 + ntp, *t2 = t1 + ntp, *t3 = t2 + ntp, *t4 = t3 + ntp,
          *b3s = t4 + ntp;
    int *flag = reinterpret_cast<int *>(b3s + ntp);
    // split of the O(nt^2) phases: `parts` groups of threads per entry, their
    // partial results in the DFT scratch T0..T2 (free at that point: 6 ntp
    // floats), ranks after them
    const int parts = max(1, min(3, nthr / nt));
    const int chunk = (nt + parts - 1) / parts;
    float *pbuf = reinterpret_cast<float *>(T0);
    int *pcnt = reinterpret_cast<int *>(T0) + 3 * ntp;
    // Q (FP32) in shared memory when it fits, else read from global memory
    float *qs = admm_q_in_smem(R) ? reinterpret_cast<float *>(flag + 4) : nullptr;
    if (qs)
        for (int i = tid; i < nt * nt; i += nthr) qs[i] = Q[i];

    const float a1 = p.alpha1 * p.mu1, a2 = p.alpha2 * p.mu2;
    for (int k = tid; k < nt; k += nthr) {
        u[k] = 1.0f / (float)nt;
        z[k] = 1.0f / (float)nt;
        zs[k] = (float)zf[k];
        p1[k] = p2[k] = x0[k] = x1[k] = y0[k] = y1[k] = y2[k] = y3[k] = 0.f;
        l10[k] = l11[k] = l20[k] = l21[k] = l22[k] = l23[k] = l3[k] = 0.f;
    }
    for (int k = tid; k < n; k += nthr) {
        double sn, cs;
        sincospi(-2.0 * (double)k / (double)n, &sn, &cs);
        tw[k] = make_float2((float)cs, (float)sn);
    }
    __syncthreads();

    int it = 0, status = PS_ERR_NOT_CONVERGED;
    double change = 0.0;
    auto at = [n](const float *a, int i, int j) {
        i = i < 0 ? i + n : (i >= n ? i - n : i);
        j = j < 0 ? j + n : (j >= n ? j - n : j);
        return a[i * n + j];
    };
    for (int t = 0; t < p.t_max; ++t) {
        // 1-2. x and y by row-wise shrinkage (Eq. x_update, Eq. y_update)
        for (int k = tid; k < nt; k += nthr) {
            const int i = k / n, j = k - (k / n) * n;
            const float g0 = at(u, i, j + 1) - u[k] - p1[k] + l10[k];
            const float g1 = at(u, i + 1, j) - u[k] - p2[k] + l11[k];
            float nr = sqrtf(g0 * g0 + g1 * g1);
            float sc = nr > 1.0f / p.mu1 ? (nr - 1.0f / p.mu1) / nr : 0.0f;
            x0[k] = g0 * sc;
            x1[k] = g1 * sc;
            const float m = 0.5f * (at(p1, i + 1, j) - p1[k] + at(p2, i, j + 1) - p2[k]);
            const float e0 = at(p1, i, j + 1) - p1[k] + l20[k];
            const float e1 = m + l21[k];
            const float e2 = m + l22[k];
            const float e3 = at(p2, i + 1, j) - p2[k] + l23[k];
            nr = sqrtf(e0 * e0 + e1 * e1 + e2 * e2 + e3 * e3);
            sc = nr > 1.0f / p.mu2 ? (nr - 1.0f / p.mu2) / nr : 0.0f;
            y0[k] = e0 * sc;
            y1[k] = e1 * sc;
            y2[k] = e2 * sc;
            y3[k] = e3 * sc;
            wv[k] = u[k] + l3[k];
        }
        __syncthreads();
        // 3. z = P_S(z_f + Q (u + Lambda3)) (Eq. z_solution, then projection).
        // The matvec's inner index is split over `parts` thread groups (the
        // CTA has several threads per entry), partial sums in the DFT scratch.
        for (int job = tid; job < parts * nt; job += nthr) {
            const int part = job / nt, k = job - (job / nt) * nt;
            const int m0 = part * chunk, m1 = min(nt, m0 + chunk);
            float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
            int m = m0;
            if (qs) {
                for (; m + 3 < m1; m += 4) {
                    c0 = fmaf(qs[m * nt + k], wv[m], c0);
                    c1 = fmaf(qs[(m + 1) * nt + k], wv[m + 1], c1);
                    c2 = fmaf(qs[(m + 2) * nt + k], wv[m + 2], c2);
                    c3 = fmaf(qs[(m + 3) * nt + k], wv[m + 3], c3);
                }
                for (; m < m1; ++m) c0 = fmaf(qs[m * nt + k], wv[m], c0);
            } else {
                for (; m + 3 < m1; m += 4) {
                    c0 = fmaf(__ldg(Q + (size_t)m * nt + k), wv[m], c0);
                    c1 = fmaf(__ldg(Q + (size_t)(m + 1) * nt + k), wv[m + 1], c1);
                    c2 = fmaf(__ldg(Q + (size_t)(m + 2) * nt + k), wv[m + 2], c2);
                    c3 = fmaf(__ldg(Q + (size_t)(m + 3) * nt + k), wv[m + 3], c3);
                }
                for (; m < m1; ++m) c0 = fmaf(__ldg(Q + (size_t)m * nt + k), wv[m], c0);
            }
            pbuf[part * nt + k] = (c0 + c1) + (c2 + c3);
        }
        __syncthreads();
        for (int k = tid; k < nt; k += nthr) {
            float acc = zs[k];
            for (int q = 0; q < parts; ++q) acc += pbuf[q * nt + k];
            t0[k] = acc;
        }
        __syncthreads();
        // Euclidean projection onto the simplex (the sort-based method): the
        // position of each entry in descending order (ties by index) and the
        // sum of the entries up to it give the largest position rho with
        // v_rho + (1 - S_rho)/rho > 0 and tau = (1 - S_rho)/rho, without a sort.
        {
            // ranks and sums over the entries ahead, split like the matvec
            for (int job = tid; job < parts * nt; job += nthr) {
                const int part = job / nt, k = job - (job / nt) * nt;
                const int m0 = part * chunk, m1 = min(nt, m0 + chunk);
                const float wk = t0[k];
                int rk = 0;
                float sk = 0.f;
                for (int m = m0; m < m1; ++m) {
                    const float wm = t0[m];
                    if (wm > wk || (wm == wk && m < k)) {
                        ++rk;
                        sk += wm;
                    }
                }
                pbuf[part * nt + k] = sk;
                pcnt[part * nt + k] = rk;
            }
            __syncthreads();
            int best = 0;
            float btau = 0.f;
            for (int k = tid; k < nt; k += nthr) {
                const float wk = t0[k];
                int rk = 1;
                float sk = wk;
                for (int q = 0; q < parts; ++q) {
                    rk += pcnt[q * nt + k];
                    sk += pbuf[q * nt + k];
                }
                const float tk = (1.0f - sk) / (float)rk;
                if (wk + tk > 0.0f && rk > best) {
                    best = rk;
                    btau = tk;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const int ob = __shfl_xor_sync(0xffffffffu, best, o);
                const float ot = __shfl_xor_sync(0xffffffffu, btau, o);
                if (ob > best) {
                    best = ob;
                    btau = ot;
                }
            }
            if ((tid & 31) == 0) {
                red[tid >> 5] = (double)best;
                red[32 + (tid >> 5)] = (double)btau;
            }
            __syncthreads();
            if (tid == 0) {
                double bb = -1.0, bt = 0.0;
                for (int k = 0; k < (nthr >> 5); ++k)
                    if (red[k] > bb) {
                        bb = red[k];
                        bt = red[32 + k];
                    }
                red[0] = bt;
            }
            __syncthreads();
            const float tau = (float)red[0];
            for (int k = tid; k < nt; k += nthr) z[k] = fmaxf(t0[k] + tau, 0.f);
        }
        __syncthreads();
        // 4. {u, p} (Appendix A, with + mu3 (z - Lambda3) in B1 and + mu3 in d1)
        for (int k = tid; k < nt; k += nthr) {
            t0[k] = x0[k] - l10[k];
            t1[k] = x1[k] - l11[k];
            t2[k] = y0[k] - l20[k];
            t3[k] = 0.5f * ((y1[k] - l21[k]) + (y2[k] - l22[k]));
            t4[k] = y3[k] - l23[k];
        }
        __syncthreads();
        for (int k = tid; k < nt; k += nthr) {
            const int i = k / n, j = k - (k / n) * n;
            // DhT f (i,j) = f(i, j-1) - f(i,j);  DvT f (i,j) = f(i-1, j) - f(i,j)
            const float b1 = a1 * ((at(t0, i, j - 1) - t0[k]) + (at(t1, i - 1, j) - t1[k])) +
                             p.mu3 * (z[k] - l3[k]);
            const float b2 = -a1 * t0[k] + a2 * ((at(t2, i, j - 1) - t2[k]) + (at(t3, i - 1, j) - t3[k]));
            const float b3 = -a1 * t1[k] + a2 * ((at(t4, i - 1, j) - t4[k]) + (at(t3, i, j - 1) - t3[k]));
            un[k] = b1;
            wv[k] = b2;
            b3s[k] = b3;
        }
        __syncthreads();
        dft3_forward<NC>(un, wv, b3s, T0, T1, T2, F0, F1, F2, tw, n);
        for (int k = tid; k < nt; k += nthr) {
            const int ky = k / n, kx = k - (k / n) * n;
            const float2 dh = make_float2(tw[kx].x - 1.0f, -tw[kx].y);   // exp(+2 pi i kx/n) - 1
            const float2 dv = make_float2(tw[ky].x - 1.0f, -tw[ky].y);
            const float ah = dh.x * dh.x + dh.y * dh.y, av = dv.x * dv.x + dv.y * dv.y;
            const float2 d1 = make_float2(a1 * (ah + av) + p.mu3, 0.f);
            const float2 d2 = make_float2(a1 + a2 * ah + 0.5f * a2 * av, 0.f);
            const float2 d3 = make_float2(a1 + a2 * av + 0.5f * a2 * ah, 0.f);
            const float2 d4 = make_float2(-a1 * dh.x, -a1 * dh.y);
            const float2 d5 = make_float2(-a1 * dv.x, -a1 * dv.y);
            const float2 d6 = c_mul(make_float2(0.5f * a2 * dh.x, -0.5f * a2 * dh.y), dv);
            const float2 c4 = c_conj(d4), c5 = c_conj(d5), c6 = c_conj(d6);
            const float2 B1 = F0[k], B2 = F1[k], B3 = F2[k];
            const float2 den = det3c(d1, c4, c5, d4, d2, c6, d5, d6, d3);
            const float2 uu = c_div(det3c(B1, c4, c5, B2, d2, c6, B3, d6, d3), den);
            const float2 q1 = c_div(det3c(d1, B1, c5, d4, B2, c6, d5, B3, d3), den);
            const float2 q2 = c_div(det3c(d1, c4, B1, d4, d2, B2, d5, d6, B3), den);
            F0[k] = uu;
            F1[k] = q1;
            F2[k] = q2;
        }
        __syncthreads();
        dft3_inverse<NC>(F0, F1, F2, T0, T1, T2, un, p1, p2, tw, n);
        // 5-7. multiplier updates (Eq. subproblems), stop test
        float dn = 0.f, nn = 0.f;
        for (int k = tid; k < nt; k += nthr) {
            const int i = k / n, j = k - (k / n) * n;
            const float gu0 = at(un, i, j + 1) - un[k];
            const float gu1 = at(un, i + 1, j) - un[k];
            l10[k] += p.rho * (gu0 - p1[k] - x0[k]);
            l11[k] += p.rho * (gu1 - p2[k] - x1[k]);
            const float m = 0.5f * (at(p1, i + 1, j) - p1[k] + at(p2, i, j + 1) - p2[k]);
            l20[k] += p.rho * (at(p1, i, j + 1) - p1[k] - y0[k]);
            l21[k] += p.rho * (m - y1[k]);
            l22[k] += p.rho * (m - y2[k]);
            l23[k] += p.rho * (at(p2, i + 1, j) - p2[k] - y3[k]);
            l3[k] += p.rho * (un[k] - z[k]);
            // stop-test norms: each thread holds at most a few entries, the
            // rest is a pairwise tree, so FP32 sums are accurate to ~1e-6
            // relative, far inside the threshold th
            const float d = u[k] - un[k];
            dn = fmaf(d, d, dn);
            nn = fmaf(un[k], un[k], nn);
        }
        float DN, NN;
        block_sum2f(dn, nn, red, DN, NN);
        __syncthreads();
        for (int k = tid; k < nt; k += nthr) u[k] = un[k];
        __syncthreads();
        it = t + 1;
        change = (double)sqrtf(DN / NN);
        if (change < (double)p.th) {
            status = PS_OK;
            break;
        }
    }
    for (int k = tid; k < nt; k += nthr) kernel_out[k] = z[k];
    if (tid == 0) {
        if (info_iters) *info_iters = it;
        if (info_status) *info_status = status;
        if (info_change) *info_change = change;
    }
}

void launch_admm(const float *Q, const double *zf, int R, const ps_kernel_params &p,
                 float *kernel_out, int *info_iters, int *info_status, double *info_change,
                 cudaStream_t st) {
    const size_t smem = admm_smem_bytes(R);
    switch (R) {
#define PS_ADMM(RR)                                                                      \
    case RR:                                                                             \
        admm_kernel<2 * RR + 1><<<1, 1024, smem, st>>>(Q, zf, R, p, kernel_out, info_iters, \
                                                       info_status, info_change);         \
        return;
        PS_ADMM(4) PS_ADMM(6) PS_ADMM(8) PS_ADMM(14)
#undef PS_ADMM
        default:
            admm_kernel<0><<<1, 1024, smem, st>>>(Q, zf, R, p, kernel_out, info_iters,
                                                  info_status, info_change);
    }
}

cudaError_t kest_set_attrs() {
    cudaError_t e = cudaSuccess;
#define PS_ADMM_ATTR(NC)                                                                   \
    if (e == cudaSuccess)                                                                  \
        e = cudaFuncSetAttribute(admm_kernel<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)kAdmmMaxSmem);
    PS_ADMM_ATTR(0) PS_ADMM_ATTR(9) PS_ADMM_ATTR(13) PS_ADMM_ATTR(17) PS_ADMM_ATTR(29)
#undef PS_ADMM_ATTR
    return e;
}

}  // namespace ps
