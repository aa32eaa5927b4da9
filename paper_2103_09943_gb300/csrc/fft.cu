// FFT and the Fourier-domain Z-step solve (Eq. Z_solution), sm_103a.
//
// The Z step of Algorithm 2 is solved exactly in the Fourier domain, the
// single FFT-based iteration the paper takes from Zhao et al. (2016): the
// operator B^T D^T D B + lambda' L^T L is block diagonal over alias groups
// of c^2 HR frequencies, each block (1/c^2) v v^H + diag(t) with
// v_j = conj(B^_j) and t_j = lambda' S^_j^2 (S^ the Laplacian symbol).
//
// 2-D FFTs are row FFTs in shared memory (Stockham autosort, radix 4/2/3,
// one CTA per row, lengths 2^a 3^b up to 8192) with tiled transposes in
// between; the spectrum is kept in transposed layout [kx][ky]. Two real
// bands are packed as the real and imaginary parts of one complex image:
// the operator has a real kernel, so the two solves do not mix.
//
// Precision: the operator amplifies relative errors of its right-hand side
// spectrum by roughly its condition number, so the forward transforms (of the
// right-hand side and of the kernel) and the group solve run in FP64; the
// solution spectrum is rounded to FP32 (harmless: the inverse transform does
// not amplify) and the inverse transforms run in FP32.
#include <math.h>

#include "common.cuh"
#include "fft_dev.cuh"
#include "kernels.cuh"

namespace ps {

bool fft_make_plan(int L, FftPlan *plan) {
    if (L < 2 || L > kMaxFFT) return false;
    int m = L, np = 0;
    while (m % 4 == 0 && np < 16) { plan->radix[np++] = 4; m /= 4; }
    while (m % 2 == 0 && np < 16) { plan->radix[np++] = 2; m /= 2; }
    while (m % 3 == 0 && np < 16) { plan->radix[np++] = 3; m /= 3; }
    if (m != 1) return false;
    plan->L = L;
    plan->npass = np;
    return true;
}

// Twiddles tw[k] = exp(-2 pi i k / L), computed in FP64; the FP32 table is
// the FP64 one rounded once.
__global__ void fft_twiddle_kernel(int L, float2 *tw32, double2 *tw64) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L) return;
    double sn, cs;
    sincospi(-2.0 * (double)k / (double)L, &sn, &cs);
    tw64[k] = make_double2(cs, sn);
    tw32[k] = make_float2((float)cs, (float)sn);
}

void launch_fft_twiddles(int L, float2 *tw32, double2 *tw64, cudaStream_t st) {
    fft_twiddle_kernel<<<(L + 255) / 256, 256, 0, st>>>(L, tw32, tw64);
}

// One CTA per row of length L (<= 8192), blockDim = L/8 rounded up to a
// multiple of 32. If `unpack` is given (FP32 inverse only), the row is
// written as two real bands (real part -> band 2k, imaginary part ->
// band 2k+1 when it exists) instead of in place.
template <class T2>
__global__ void __launch_bounds__(1024) fft_rows_kernel(T2 *data, FftPlan plan,
                                                        const T2 *__restrict__ tw, int inverse,
                                                        float *unpack, int N, size_t HW) {
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    T2 *a = reinterpret_cast<T2 *>(fsm_raw);
    const int L = plan.L;
    const size_t row = blockIdx.x;
    T2 *src = data + row * (size_t)L;
    for (int i = threadIdx.x; i < L; i += blockDim.x) a[i] = src[i];
    __syncthreads();
    fft_row<8, T2>(a, plan, tw, inverse != 0, threadIdx.x, blockDim.x);
    if (unpack) {
        // rows are ordered (image, y); image k holds bands 2k, 2k+1
        const size_t rows_per_img = HW / (size_t)L;
        const size_t img = row / rows_per_img, y = row - img * rows_per_img;
        const int b0 = (int)(2 * img);
        float *o0 = unpack + (size_t)b0 * HW + y * L;
        float *o1 = (b0 + 1 < N) ? unpack + (size_t)(b0 + 1) * HW + y * L : nullptr;
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            o0[i] = (float)a[i].x;
            if (o1) o1[i] = (float)a[i].y;
        }
    } else {
        for (int i = threadIdx.x; i < L; i += blockDim.x) src[i] = a[i];
    }
}

static int fft_threads(int L) {
    int t = (L + 7) / 8;
    t = (t + 31) & ~31;
    if (t < 32) t = 32;
    if (t > 1024) t = 1024;
    return t;
}

void launch_fft_rows32(float2 *data, const FftPlan &plan, int rows, const float2 *tw,
                       int inverse, float *unpack, int N, size_t HW, cudaStream_t st) {
    fft_rows_kernel<float2><<<rows, fft_threads(plan.L), plan.L * sizeof(float2), st>>>(
        data, plan, tw, inverse, unpack, N, HW);
}

void launch_fft_rows64(double2 *data, const FftPlan &plan, int rows, const double2 *tw,
                       cudaStream_t st) {
    fft_rows_kernel<double2><<<rows, fft_threads(plan.L), plan.L * sizeof(double2), st>>>(
        data, plan, tw, 0, nullptr, 0, 0);
}

// out[b][c][r] = in[b][r][c] for a batch of rows x cols complex matrices.
template <class T2>
__global__ void __launch_bounds__(256) transpose_kernel(const T2 *__restrict__ in,
                                                        T2 *__restrict__ out, int rows,
                                                        int cols) {
    __shared__ T2 tile[32][33];
    const size_t bo = (size_t)blockIdx.z * rows * cols;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = in[bo + (size_t)r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[bo + (size_t)c * rows + r] = tile[threadIdx.x][k];
    }
}

void launch_transpose32(const float2 *in, float2 *out, int rows, int cols, int batch,
                        cudaStream_t st) {
    dim3 blk(32, 8), grd((cols + 31) / 32, (rows + 31) / 32, batch);
    transpose_kernel<float2><<<grd, blk, 0, st>>>(in, out, rows, cols);
}

void launch_transpose64(const double2 *in, double2 *out, int rows, int cols, int batch,
                        cudaStream_t st) {
    dim3 blk(32, 8), grd((cols + 31) / 32, (rows + 31) / 32, batch);
    transpose_kernel<double2><<<grd, blk, 0, st>>>(in, out, rows, cols);
}

// H x W complex image holding the kernel taps at (i mod H, j mod W).
__global__ void kernel_embed_kernel(const float *__restrict__ u, int R, int H, int W,
                                    double2 *out) {
    const size_t HW = (size_t)H * W;
    const int n = 2 * R + 1;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < HW;
         k += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(k / W), x = (int)(k - (k / W) * W);
        int i = y, j = x;
        if (i > H / 2) i -= H;
        if (j > W / 2) j -= W;
        double val = 0.0;
        if (i >= -R && i <= R && j >= -R && j <= R) val = (double)u[(i + R) * n + (j + R)];
        out[k] = make_double2(val, 0.0);
    }
}

void launch_kernel_embed(const float *u, int R, int H, int W, double2 *out, cudaStream_t st) {
    const size_t HW = (size_t)H * W;
    int blocks = (int)((HW + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    kernel_embed_kernel<<<blocks, 256, 0, st>>>(u, R, H, W, out);
}

// Spectrum of the kernel embedded on the H x W torus, straight from its
// (2R+1)^2 taps, layout [kx][ky] (FP64):
//   B^(kx, ky) = sum_i exp(-2 pi i ky i / H) T_i(kx),
//   T_i(kx) = sum_j u(i, j) exp(-2 pi i kx j / W),  i, j in [-R, R].
// One CTA per 32 values of kx and 128 of ky: the T_i of its columns in
// shared memory, then one output per thread along ky (coalesced), twiddles
// from the FP64 tables tw[k] = exp(-2 pi i k / L).
constexpr int kSpecCols = 32, kSpecRows = 128;
__global__ void __launch_bounds__(256) kernel_spectrum_kernel(const float *__restrict__ u, int R,
                                                              int H, int W,
                                                              const double2 *__restrict__ twW,
                                                              const double2 *__restrict__ twH,
                                                              double2 *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char ksm[];
    double2 *T = reinterpret_cast<double2 *>(ksm);  // [2R+1][kSpecCols]
    const int n = 2 * R + 1;
    const int kx0 = blockIdx.x * kSpecCols;
    for (int e = threadIdx.x; e < n * kSpecCols; e += blockDim.x) {
        const int ii = e / kSpecCols, c = e - ii * kSpecCols;
        const int kx = kx0 + c;
        double re = 0.0, im = 0.0;
        if (kx < W) {
            // twiddle index kx j mod W, stepped by kx from j = -R
            int idx = (int)(((long long)W * (R + 1) - (long long)kx * R) % W);
            for (int jj = 0; jj < n; ++jj) {
                const double2 w = twW[idx];
                const double uv = (double)u[ii * n + jj];
                re = fma(uv, w.x, re);
                im = fma(uv, w.y, im);
                idx += kx;
                if (idx >= W) idx -= W;
            }
        }
        T[ii * kSpecCols + c] = make_double2(re, im);
    }
    __syncthreads();
    const int cols = min(kSpecCols, W - kx0);
    const int ky0 = blockIdx.y * kSpecRows, nky = min(kSpecRows, H - ky0);
    for (int e = threadIdx.x; e < cols * nky; e += blockDim.x) {
        const int c = e / nky, ky = ky0 + (e - (e / nky) * nky);
        double re = 0.0, im = 0.0;
        // twiddle index ky i mod H, stepped by ky from i = -R
        int idx = (int)(((long long)H * (R + 1) - (long long)ky * R) % H);
        for (int ii = 0; ii < n; ++ii) {
            const double2 w = twH[idx];
            idx += ky;
            if (idx >= H) idx -= H;
            const double2 t = T[ii * kSpecCols + c];
            re = fma(t.x, w.x, fma(-t.y, w.y, re));
            im = fma(t.x, w.y, fma(t.y, w.x, im));
        }
        out[(size_t)(kx0 + c) * H + ky] = make_double2(re, im);
    }
}

void launch_kernel_spectrum(const float *u, int R, int H, int W, const double2 *twW,
                            const double2 *twH, double2 *out, cudaStream_t st) {
    const int n = 2 * R + 1;
    const size_t smem = (size_t)n * kSpecCols * sizeof(double2);
    const dim3 grd((W + kSpecCols - 1) / kSpecCols, (H + kSpecRows - 1) / kSpecRows);
    kernel_spectrum_kernel<<<grd, 256, smem, st>>>(u, R, H, W, twW, twH, out);
}

// Per alias group (ky0 + p h, kx0 + q w), p, q in [0, c): solve
//   ((1/c^2) v v^H + diag(t)) x = r,  v_j = conj(B^_j), t_j = lam S^_j^2.
// With s = v^H x:  x_j = (r_j - v_j s / c^2) / t_j, and s from
//   s (t_m + (|v_m|^2 + t_m sum_{j!=m} |v_j|^2/t_j) / c^2)
//     = conj(v_m) r_m + t_m sum_{j!=m} conj(v_j) r_j / t_j,
// m the member with the smallest t (both sides multiplied by t_m, so the
// DC group, where t_m = 0, needs no special case). When the data term
// dominates member m (c^2 t_m < |v_m|^2), x_m is taken from
// s = sum_j conj(v_j) x_j instead of dividing by the tiny t_m.
// The group algebra runs in FP64 (near-DC groups cancel strongly; there are
// only H W / c^2 groups per image). The result is scaled by 1/(H W) for the
// unnormalised inverse FFT.
struct cd { double x, y; };
__device__ __forceinline__ cd cd_mul(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }

__device__ __forceinline__ double symbol_t(int ky, int kx, int H, int W, double lam) {
    const double sy = (double)sinpif((float)ky / (float)H);
    const double sx = (double)sinpif((float)kx / (float)W);
    const double sh = 4.0 * (sy * sy + sx * sx);
    return lam * sh * sh;
}

__global__ void __launch_bounds__(256) alias_solve_kernel(const double2 *__restrict__ spec,
                                                          const double2 *__restrict__ bspec,
                                                          float2 *__restrict__ sol, int H,
                                                          int W, int c, float lamf,
                                                          const double *__restrict__ tsym) {
    const int h = H / c, w = W / c;
    const int gidx = blockIdx.x * blockDim.x + threadIdx.x;
    if (gidx >= h * w) return;
    const int kx0 = gidx / h, ky0 = gidx - (gidx / h) * h;
    const double2 *S = spec + (size_t)blockIdx.y * H * W;
    float2 *X = sol + (size_t)blockIdx.y * H * W;
    const double cc = (double)(c * c), icc = 1.0 / cc, lam = (double)lamf;
    int pm = 0, qm = 0;
    double tmin = 1e300;
    for (int p = 0; p < c; ++p)
        for (int q = 0; q < c; ++q) {
            const int ky = ky0 + p * h, kx = kx0 + q * w;
            const double t = tsym ? lam * tsym[(size_t)kx * H + ky] : symbol_t(ky, kx, H, W, lam);
            if (t < tmin) { tmin = t; pm = p; qm = q; }
        }
    cd num = {0.0, 0.0};
    double dsum = 0.0;
    cd rm = {0.0, 0.0}, vm = {0.0, 0.0};
    for (int p = 0; p < c; ++p)
        for (int q = 0; q < c; ++q) {
            const int ky = ky0 + p * h, kx = kx0 + q * w;
            const size_t o = (size_t)kx * H + ky;
            const double2 rf = S[o], bh = bspec[o];
            const cd r = {rf.x, rf.y};
            const cd v = {bh.x, -bh.y};
            if (p == pm && q == qm) {
                rm = r;
                vm = v;
                continue;
            }
            const double it =
                1.0 / (tsym ? lam * tsym[(size_t)kx * H + ky] : symbol_t(ky, kx, H, W, lam));
            num.x += (v.x * r.x + v.y * r.y) * it;
            num.y += (v.x * r.y - v.y * r.x) * it;
            dsum += (v.x * v.x + v.y * v.y) * it;
        }
    const double vm2 = vm.x * vm.x + vm.y * vm.y;
    const cd nn = {vm.x * rm.x + vm.y * rm.y + tmin * num.x,
                   vm.x * rm.y - vm.y * rm.x + tmin * num.y};
    const double iden = 1.0 / (tmin + (vm2 + tmin * dsum) * icc);
    const cd s = {nn.x * iden, nn.y * iden};
    const double scale = 1.0 / ((double)H * (double)W);
    cd acc = {0.0, 0.0};
    for (int p = 0; p < c; ++p)
        for (int q = 0; q < c; ++q) {
            if (p == pm && q == qm) continue;
            const int ky = ky0 + p * h, kx = kx0 + q * w;
            const size_t o = (size_t)kx * H + ky;
            const double2 rf = S[o], bh = bspec[o];
            const cd v = {bh.x, -bh.y};
            const double it =
                1.0 / (tsym ? lam * tsym[(size_t)kx * H + ky] : symbol_t(ky, kx, H, W, lam));
            const cd vs = cd_mul(v, s);
            const cd x = {(rf.x - vs.x * icc) * it, (rf.y - vs.y * icc) * it};
            acc.x += v.x * x.x + v.y * x.y;
            acc.y += v.x * x.y - v.y * x.x;
            X[o] = make_float2((float)(x.x * scale), (float)(x.y * scale));
        }
    cd xm;
    if (cc * tmin < vm2) {
        const cd d = {s.x - acc.x, s.y - acc.y};
        const double iv = 1.0 / vm2;
        xm = {(d.x * vm.x - d.y * vm.y) * iv, (d.y * vm.x + d.x * vm.y) * iv};
    } else {
        const cd vs = cd_mul(vm, s);
        xm = {(rm.x - vs.x * icc) / tmin, (rm.y - vs.y * icc) / tmin};
    }
    X[(size_t)(kx0 + qm * w) * H + (ky0 + pm * h)] =
        make_float2((float)(xm.x * scale), (float)(xm.y * scale));
}

void launch_alias_solve(const double2 *spec, const double2 *bspec, float2 *sol, int nimg, int H,
                        int W, int c, float lam, cudaStream_t st, const double *tsym) {
    const int groups = (H / c) * (W / c);
    dim3 grd((groups + 255) / 256, nimg);
    alias_solve_kernel<<<grd, 256, 0, st>>>(spec, bspec, sol, H, W, c, lam, tsym);
}

cudaError_t fft_set_attrs() {
    cudaError_t e = cudaFuncSetAttribute(fft_rows_kernel<float2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kMaxFFT * sizeof(float2)));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fft_rows_kernel<double2>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kMaxFFT * sizeof(double2)));
}

}  // namespace ps
