// Warm starts of the Z0 solve (sm_103a): bicubic x c upsampling of the LR
// bands, the start point the CG runs from (and the network's input).
//
// Keys' cubic convolution (Keys 1981, a = -1/2), separable, with HR pixel
// c k + phi on LR coordinate k + phi / c (phase 0: the samples the
// decimation D keeps) and a circular boundary. One thread writes four
// consecutive HR pixels of a row (one float4 store); the LR rows it reads
// are shared by the CTA's threads through L1.
#include "common.cuh"
#include "kernels.cuh"

namespace ps {

namespace {

// W(x) of Keys' kernel for 0 <= x < 2, a = -1/2.
__device__ __forceinline__ float keys_w(float x) {
    return x <= 1.0f ? fmaf(fmaf(1.5f, x, -2.5f), x * x, 1.0f)
                     : fmaf(fmaf(fmaf(-0.5f, x, 2.5f), x, -4.0f), x, 2.0f);
}

// Weights of the taps k-1, k, k+1, k+2 at fractional position t in [0, 1).
__device__ __forceinline__ void keys_weights(float t, float w[4]) {
    w[0] = keys_w(1.0f + t);
    w[1] = keys_w(t);
    w[2] = keys_w(1.0f - t);
    w[3] = keys_w(2.0f - t);
}

__global__ void __launch_bounds__(256) bicubic_up_kernel(const float *__restrict__ X, int h,
                                                         int w, int c,
                                                         float *__restrict__ out) {
    const int W = w * c, H = h * c;
    const int x4 = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, b = blockIdx.z;
    if (4 * x4 >= W) return;
    const float *Xb = X + (size_t)b * h * w;
    const int ky = y / c;
    float wy[4];
    keys_weights((float)(y - ky * c) / (float)c, wy);
    const float *rows[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int yy = ky - 1 + i;
        yy = yy < 0 ? yy + h : (yy >= h ? yy - h : yy);
        rows[i] = Xb + (size_t)yy * w;
    }
    float res[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int x = 4 * x4 + e;
        const int kx = x / c;
        float wx[4];
        keys_weights((float)(x - kx * c) / (float)c, wx);
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int xx = kx - 1 + j;
            xx = xx < 0 ? xx + w : (xx >= w ? xx - w : xx);
            float col = 0.0f;
#pragma unroll
            for (int i = 0; i < 4; ++i) col = fmaf(wy[i], __ldg(rows[i] + xx), col);
            acc = fmaf(wx[j], col, acc);
        }
        res[e] = acc;
    }
    *reinterpret_cast<float4 *>(out + ((size_t)b * H + y) * W + 4 * x4) =
        make_float4(res[0], res[1], res[2], res[3]);
}

}  // namespace

void launch_bicubic_up(const float *X, int N, int h, int w, int c, float *out,
                       cudaStream_t st) {
    const int W4 = (w * c) / 4;
    dim3 grd((W4 + 127) / 128, h * c, N);
    bicubic_up_kernel<<<grd, 128, 0, st>>>(X, h, w, c, out);
}

}  // namespace ps
