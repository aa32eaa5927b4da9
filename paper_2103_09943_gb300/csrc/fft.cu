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
#include <math.h>

#include "common.cuh"
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

// tw[k] = exp(-2 pi i k / L), computed in FP64 and rounded once.
__global__ void fft_twiddle_kernel(int L, float2 *tw) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L) return;
    double sn, cs;
    sincospi(-2.0 * (double)k / (double)L, &sn, &cs);
    tw[k] = make_float2((float)cs, (float)sn);
}

void launch_fft_twiddles(int L, float2 *tw, cudaStream_t st) {
    fft_twiddle_kernel<<<(L + 255) / 256, 256, 0, st>>>(L, tw);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place radix-R DFT of v with exponent sign `sg` (-1 forward, +1 inverse).
template <int R>
__device__ __forceinline__ void dft_small(float2 *v, float sg);

template <>
__device__ __forceinline__ void dft_small<2>(float2 *v, float) {
    const float2 a = v[0], b = v[1];
    v[0] = make_float2(a.x + b.x, a.y + b.y);
    v[1] = make_float2(a.x - b.x, a.y - b.y);
}

template <>
__device__ __forceinline__ void dft_small<4>(float2 *v, float sg) {
    // exp(sg * 2 pi i / 4) = (0, sg)
    const float2 a0 = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
    const float2 a1 = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
    const float2 b0 = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
    const float2 b1 = make_float2(v[1].x - v[3].x, v[1].y - v[3].y);
    // (0, sg) * b1 = (-sg b1.y, sg b1.x)
    const float2 jb1 = make_float2(-sg * b1.y, sg * b1.x);
    v[0] = make_float2(a0.x + b0.x, a0.y + b0.y);
    v[2] = make_float2(a0.x - b0.x, a0.y - b0.y);
    v[1] = make_float2(a1.x + jb1.x, a1.y + jb1.y);
    v[3] = make_float2(a1.x - jb1.x, a1.y - jb1.y);
}

template <>
__device__ __forceinline__ void dft_small<3>(float2 *v, float sg) {
    // w = exp(sg * 2 pi i / 3) = (-1/2, sg sqrt(3)/2)
    const float s3 = 0.86602540378443865f * sg;
    const float2 a = v[0], b = v[1], c = v[2];
    const float2 t = make_float2(b.x + c.x, b.y + c.y);
    const float2 d = make_float2(b.x - c.x, b.y - c.y);
    const float2 m = make_float2(a.x - 0.5f * t.x, a.y - 0.5f * t.y);
    // w b + w^2 c = -t/2 + i s3 (b - c)
    v[0] = make_float2(a.x + t.x, a.y + t.y);
    v[1] = make_float2(m.x - s3 * d.y, m.y + s3 * d.x);
    v[2] = make_float2(m.x + s3 * d.y, m.y - s3 * d.x);
}

template <int R>
__device__ __forceinline__ void stockham_pass(const float2 *a, float2 *b, int L, int Ns,
                                              const float2 *__restrict__ tw, float sg,
                                              bool inverse) {
    const int m = L / R;
    const int stride = L / (Ns * R);
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            float2 x = a[j + t * m];
            if (t > 0 && k > 0) {
                float2 w = __ldg(tw + t * k * stride);
                if (inverse) w.y = -w.y;
                x = cmul(x, w);
            }
            v[t] = x;
        }
        dft_small<R>(v, sg);
        const int idxD = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int t = 0; t < R; ++t) b[idxD + t * Ns] = v[t];
    }
}

// One CTA per row of length L. If `unpack` is given, the row is written back
// as two real bands (real part -> band 2k, imaginary part -> band 2k+1 when
// it exists) instead of in place.
__global__ void __launch_bounds__(256) fft_rows_kernel(float2 *data, FftPlan plan,
                                                       const float2 *__restrict__ tw,
                                                       int inverse, float scale, float *unpack,
                                                       int N, size_t HW) {
    extern __shared__ float2 fsm[];
    const int L = plan.L;
    float2 *a = fsm, *b = fsm + L;
    const size_t row = blockIdx.x;
    float2 *src = data + row * (size_t)L;
    for (int i = threadIdx.x; i < L; i += blockDim.x) a[i] = src[i];
    __syncthreads();
    const float sg = inverse ? 1.0f : -1.0f;
    int Ns = 1;
    for (int p = 0; p < plan.npass; ++p) {
        const int R = plan.radix[p];
        if (R == 4)
            stockham_pass<4>(a, b, L, Ns, tw, sg, inverse != 0);
        else if (R == 2)
            stockham_pass<2>(a, b, L, Ns, tw, sg, inverse != 0);
        else
            stockham_pass<3>(a, b, L, Ns, tw, sg, inverse != 0);
        __syncthreads();
        float2 *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    if (unpack) {
        // rows are ordered (image, y); image k holds bands 2k, 2k+1
        const size_t rows_per_img = HW / (size_t)L;
        const size_t img = row / rows_per_img, y = row - img * rows_per_img;
        const int b0 = (int)(2 * img);
        float *o0 = unpack + (size_t)b0 * HW + y * L;
        float *o1 = (b0 + 1 < N) ? unpack + (size_t)(b0 + 1) * HW + y * L : nullptr;
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            o0[i] = a[i].x * scale;
            if (o1) o1[i] = a[i].y * scale;
        }
    } else {
        for (int i = threadIdx.x; i < L; i += blockDim.x)
            src[i] = make_float2(a[i].x * scale, a[i].y * scale);
    }
}

void launch_fft_rows(float2 *data, const FftPlan &plan, int rows, const float2 *tw,
                     int inverse, float scale, float *unpack, int N, size_t HW,
                     cudaStream_t st) {
    const int thr = plan.L >= 1024 ? 256 : (plan.L >= 256 ? 128 : 64);
    fft_rows_kernel<<<rows, thr, 2 * plan.L * sizeof(float2), st>>>(data, plan, tw, inverse,
                                                                    scale, unpack, N, HW);
}

// out[b][c][r] = in[b][r][c] for a batch of rows x cols complex matrices.
__global__ void __launch_bounds__(256) transpose_kernel(const float2 *__restrict__ in,
                                                        float2 *__restrict__ out, int rows,
                                                        int cols) {
    __shared__ float2 tile[32][33];
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

void launch_transpose(const float2 *in, float2 *out, int rows, int cols, int batch,
                      cudaStream_t st) {
    dim3 blk(32, 8), grd((cols + 31) / 32, (rows + 31) / 32, batch);
    transpose_kernel<<<grd, blk, 0, st>>>(in, out, rows, cols);
}

// H x W complex image holding the kernel taps at (i mod H, j mod W).
__global__ void kernel_embed_kernel(const float *__restrict__ u, int R, int H, int W,
                                    float2 *out) {
    const size_t HW = (size_t)H * W;
    const int n = 2 * R + 1;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < HW;
         k += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(k / W), x = (int)(k - (k / W) * W);
        int i = y, j = x;
        if (i > H / 2) i -= H;
        if (j > W / 2) j -= W;
        float val = 0.0f;
        if (i >= -R && i <= R && j >= -R && j <= R) val = u[(i + R) * n + (j + R)];
        out[k] = make_float2(val, 0.0f);
    }
}

void launch_kernel_embed(const float *u, int R, int H, int W, float2 *out, cudaStream_t st) {
    const size_t HW = (size_t)H * W;
    int blocks = (int)((HW + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    kernel_embed_kernel<<<blocks, 256, 0, st>>>(u, R, H, W, out);
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
// The result is scaled by 1/(H W) for the unnormalised inverse FFT.
__global__ void __launch_bounds__(256) alias_solve_kernel(float2 *spec,
                                                          const float2 *__restrict__ bspec,
                                                          int H, int W, int c, float lam) {
    const int h = H / c, w = W / c;
    const int gidx = blockIdx.x * blockDim.x + threadIdx.x;
    if (gidx >= h * w) return;
    const int kx0 = gidx / h, ky0 = gidx - (gidx / h) * h;
    float2 *S = spec + (size_t)blockIdx.y * H * W;
    const float cc = (float)(c * c);
    // member with the smallest symbol
    int pm = 0, qm = 0;
    float tmin = 3.4e38f;
    for (int p = 0; p < c; ++p)
        for (int q = 0; q < c; ++q) {
            const float sy = sinpif((float)(ky0 + p * h) / (float)H);
            const float sx = sinpif((float)(kx0 + q * w) / (float)W);
            const float sh = 4.0f * (sy * sy + sx * sx);
            const float t = lam * sh * sh;
            if (t < tmin) { tmin = t; pm = p; qm = q; }
        }
    float2 num = make_float2(0.f, 0.f);
    float dsum = 0.f;
    float2 rm = make_float2(0.f, 0.f), vm = make_float2(0.f, 0.f);
    for (int p = 0; p < c; ++p)
        for (int q = 0; q < c; ++q) {
            const int ky = ky0 + p * h, kx = kx0 + q * w;
            const size_t o = (size_t)kx * H + ky;
            const float2 r = S[o];
            const float2 bh = bspec[o];
            const float2 v = make_float2(bh.x, -bh.y);
            if (p == pm && q == qm) {
                rm = r;
                vm = v;
                continue;
            }
            const float sy = sinpif((float)ky / (float)H);
            const float sx = sinpif((float)kx / (float)W);
            const float sh = 4.0f * (sy * sy + sx * sx);
            const float t = lam * sh * sh;
            // conj(v) r / t
            num.x += (v.x * r.x + v.y * r.y) / t;
            num.y += (v.x * r.y - v.y * r.x) / t;
            dsum += (v.x * v.x + v.y * v.y) / t;
        }
    const float vm2 = vm.x * vm.x + vm.y * vm.y;
    // numerator: conj(vm) rm + tmin * num
    float2 nn = make_float2(vm.x * rm.x + vm.y * rm.y + tmin * num.x,
                            vm.x * rm.y - vm.y * rm.x + tmin * num.y);
    const float den = tmin + (vm2 + tmin * dsum) / cc;
    const float2 s = make_float2(nn.x / den, nn.y / den);
    const float scale = 1.0f / ((float)H * (float)W);
    float2 acc = make_float2(0.f, 0.f);  // sum_{j != m} conj(v_j) x_j
    for (int p = 0; p < c; ++p)
        for (int q = 0; q < c; ++q) {
            if (p == pm && q == qm) continue;
            const int ky = ky0 + p * h, kx = kx0 + q * w;
            const size_t o = (size_t)kx * H + ky;
            const float2 r = S[o];
            const float2 bh = bspec[o];
            const float2 v = make_float2(bh.x, -bh.y);
            const float sy = sinpif((float)ky / (float)H);
            const float sx = sinpif((float)kx / (float)W);
            const float sh = 4.0f * (sy * sy + sx * sx);
            const float t = lam * sh * sh;
            const float2 vs = cmul(v, s);
            const float2 x = make_float2((r.x - vs.x / cc) / t, (r.y - vs.y / cc) / t);
            acc.x += v.x * x.x + v.y * x.y;
            acc.y += v.x * x.y - v.y * x.x;
            S[o] = make_float2(x.x * scale, x.y * scale);
        }
    float2 xm;
    if (cc * tmin < vm2) {
        // x_m = (s - acc) / conj(v_m)
        const float2 d = make_float2(s.x - acc.x, s.y - acc.y);
        const float2 cv = make_float2(vm.x, -vm.y);
        const float cv2 = vm2;
        xm = make_float2((d.x * cv.x + d.y * cv.y) / cv2, (d.y * cv.x - d.x * cv.y) / cv2);
    } else {
        const float2 vs = cmul(vm, s);
        xm = make_float2((rm.x - vs.x / cc) / tmin, (rm.y - vs.y / cc) / tmin);
    }
    S[(size_t)(kx0 + qm * w) * H + (ky0 + pm * h)] = make_float2(xm.x * scale, xm.y * scale);
}

void launch_alias_solve(float2 *spec, const float2 *bspec, int nimg, int H, int W, int c,
                        float lam, cudaStream_t st) {
    const int groups = (H / c) * (W / c);
    dim3 grd((groups + 255) / 256, nimg);
    alias_solve_kernel<<<grd, 256, 0, st>>>(spec, bspec, H, W, c, lam);
}

cudaError_t fft_set_attrs() {
    return cudaFuncSetAttribute(fft_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2 * kMaxFFT * sizeof(float2)));
}

}  // namespace ps
