// The warm-start network's parts on the CUDA cores (sm_103a): the first
// convolution (2 -> 32), the last one (32 -> 1) with the residual output, the
// loss and its gradient, the last layer's backward pass, the weight and bias
// gradients of every layer, and Adam. The 32 -> 32 convolutions (forward and
// backward data) run on the tensor cores (cnn.cu).
//
// Layouts: input planes and outputs are FP32 B x H x W; hidden activations
// and the gradients that flow between hidden layers are BF16 NHWC
// (B x H x W x 32). Parameters are one FP32 vector, layer after layer, each
// layer's weights (out, in, 3, 3) followed by its biases. Convolutions are
// circular 3 x 3 cross-correlations.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace ps {

namespace {

constexpr int kCh = 32;
constexpr float kScale = 255.0f;

__device__ __forceinline__ int wrapi2(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ void load_px32(const __nv_bfloat16 *p, float *v) {
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint4 u = __ldg(q + k);
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 f = __bfloat1622float2(h[e]);
            v[8 * k + 2 * e] = f.x;
            v[8 * k + 2 * e + 1] = f.y;
        }
    }
}

__device__ __forceinline__ void store_px32(__nv_bfloat16 *p, const float *v) {
    uint4 pk[4];
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(pk);
#pragma unroll
    for (int c = 0; c < kCh / 2; ++c) h[c] = __floats2bfloat162_rn(v[2 * c], v[2 * c + 1]);
    uint4 *q = reinterpret_cast<uint4 *>(p);
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = pk[k];
}

// a1 = ReLU(conv0(x) + b0), x = (up / s, pan / s). One thread per pair of
// horizontally adjacent pixels (W is even): every weight load feeds both
// pixels, and the two 3 x 3 neighbourhoods share a 3 x 4 input patch. The
// weights sit transposed in shared memory, sw[(t * 2 + i) * 32 + o] =
// w0[o][i][t], so that four output channels are one broadcast 16-byte load.
__global__ void __launch_bounds__(256, 2) cnn_first_kernel(const float *__restrict__ up,
                                                        const float *__restrict__ pan,
                                                        size_t pan_stride,
                                                        const float *__restrict__ prm, int B,
                                                        int H, int W,
                                                        __nv_bfloat16 *__restrict__ a1) {
    __shared__ __align__(16) float sw[kCh * 2 * 9 + kCh];
    for (int i = threadIdx.x; i < kCh * 18; i += blockDim.x) {
        const int o = i / 18, ci = (i / 9) % 2, t = i % 9;
        sw[(t * 2 + ci) * 32 + o] = prm[i];
    }
    if (threadIdx.x < kCh) sw[576 + threadIdx.x] = prm[576 + threadIdx.x];
    __syncthreads();
    const size_t HW = (size_t)H * W;
    const int W2 = W >> 1;
    const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)B * H * W2) return;
    const size_t HW2 = (size_t)H * W2;
    const int b = (int)(idx / HW2);
    const int rem = (int)(idx - (size_t)b * HW2), y = rem / W2, x = 2 * (rem - (rem / W2) * W2);
    const float *u = up + (size_t)b * HW;
    const float *p = pan + (size_t)b * pan_stride;
    float in[2][3][4];  // channel, row y - 1 .. y + 1, columns x - 1 .. x + 2
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
        const size_t ro = (size_t)wrapi2(y + dy - 1, H) * W;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int xx = wrapi2(x - 1 + c, W);
            in[0][dy][c] = __ldg(u + ro + xx) * (1.0f / kScale);
            in[1][dy][c] = __ldg(p + ro + xx) * (1.0f / kScale);
        }
    }
    float v0[kCh], v1[kCh];
#pragma unroll
    for (int o = 0; o < kCh; ++o) v0[o] = v1[o] = sw[576 + o];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int dy = t / 3, dx = t % 3;
#pragma unroll
        for (int ci = 0; ci < 2; ++ci) {
            const float xa = in[ci][dy][dx], xb = in[ci][dy][dx + 1];
            const float4 *w4 = reinterpret_cast<const float4 *>(sw + (t * 2 + ci) * 32);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 wv = w4[q];
                v0[4 * q] = fmaf(wv.x, xa, v0[4 * q]);
                v0[4 * q + 1] = fmaf(wv.y, xa, v0[4 * q + 1]);
                v0[4 * q + 2] = fmaf(wv.z, xa, v0[4 * q + 2]);
                v0[4 * q + 3] = fmaf(wv.w, xa, v0[4 * q + 3]);
                v1[4 * q] = fmaf(wv.x, xb, v1[4 * q]);
                v1[4 * q + 1] = fmaf(wv.y, xb, v1[4 * q + 1]);
                v1[4 * q + 2] = fmaf(wv.z, xb, v1[4 * q + 2]);
                v1[4 * q + 3] = fmaf(wv.w, xb, v1[4 * q + 3]);
            }
        }
    }
#pragma unroll
    for (int o = 0; o < kCh; ++o) {
        v0[o] = fmaxf(v0[o], 0.0f);
        v1[o] = fmaxf(v1[o], 0.0f);
    }
    __nv_bfloat16 *dst = a1 + ((size_t)b * HW + (size_t)y * W + x) * kCh;
    store_px32(dst, v0);
    store_px32(dst + kCh, v1);
}

// z = s (up / s + conv5(a5) + b5). With a target: also the loss sum
// sum w ((z - t) / s)^2 (FP64, per launch) and d5 = 2 w (z - t) / s / count,
// w the per-pixel weight (1 without one).
__global__ void __launch_bounds__(256) cnn_last_kernel(const __nv_bfloat16 *__restrict__ a5,
                                                       const float *__restrict__ up,
                                                       const float *__restrict__ prm5, int B,
                                                       int H, int W, float *__restrict__ z,
                                                       const float *__restrict__ target,
                                                       const float *__restrict__ weight,
                                                       float inv_count, float *__restrict__ d5,
                                                       double *loss) {
    __shared__ float sw[kCh * 9 + 1];
    __shared__ double red[8];
    for (int i = threadIdx.x; i < kCh * 9 + 1; i += blockDim.x) sw[i] = prm5[i];
    __syncthreads();
    const size_t HW = (size_t)H * W;
    const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    double l2 = 0.0;
    if (idx < (size_t)B * HW) {
        const int b = (int)(idx / HW);
        const int rem = (int)(idx - (size_t)b * HW), y = rem / W, x = rem - (rem / W) * W;
        float s = sw[kCh * 9];
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int yy = wrapi2(y + dy, H);
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int xx = wrapi2(x + dx, W);
                float v[kCh];
                load_px32(a5 + (((size_t)b * H + yy) * W + xx) * kCh, v);
                const int t = (dy + 1) * 3 + dx + 1;
#pragma unroll
                for (int c = 0; c < kCh; ++c) s = fmaf(sw[c * 9 + t], v[c], s);
            }
        }
        const float zv = kScale * (__ldg(up + idx) * (1.0f / kScale) + s);
        if (z) z[idx] = zv;
        if (target) {
            const float d = (zv - __ldg(target + idx)) * (1.0f / kScale);
            const float w = weight ? __ldg(weight + idx) : 1.0f;
            d5[idx] = 2.0f * w * d * inv_count;
            l2 = (double)w * (double)d * (double)d;
        }
    }
    if (!target) return;
    for (int o = 16; o > 0; o >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        atomicAdd(loss, t);
    }
}

// Backward of the last layer: D4 = conv5^T(d5) * (a5 > 0) (BF16 NHWC), and
// the gradients of w5 (32 x 9) and b5, accumulated per CTA then atomically.
__global__ void __launch_bounds__(256) cnn_last_bwd_kernel(const __nv_bfloat16 *__restrict__ a5,
                                                           const float *__restrict__ d5,
                                                           const float *__restrict__ prm5,
                                                           int B, int H, int W,
                                                           __nv_bfloat16 *__restrict__ D4,
                                                           float *__restrict__ g5) {
    __shared__ float sw[kCh * 9];
    __shared__ float acc[kCh * 9 + 1];
    for (int i = threadIdx.x; i < kCh * 9; i += blockDim.x) sw[i] = prm5[i];
    for (int i = threadIdx.x; i < kCh * 9 + 1; i += blockDim.x) acc[i] = 0.0f;
    __syncthreads();
    const size_t HW = (size_t)H * W;
    const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const bool live = idx < (size_t)B * HW;
    int b = 0, y = 0, x = 0;
    if (live) {
        b = (int)(idx / HW);
        const int rem = (int)(idx - (size_t)b * HW);
        y = rem / W;
        x = rem - (rem / W) * W;
    }
    // D4(p) = sum_t w5[c][t] d5(p - t): gather from the neighbours
    float g[kCh];
#pragma unroll
    for (int c = 0; c < kCh; ++c) g[c] = 0.0f;
    if (live) {
        const float *db = d5 + (size_t)b * HW;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int yy = wrapi2(y - dy, H);
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int xx = wrapi2(x - dx, W);
                const float dv = __ldg(db + (size_t)yy * W + xx);
                const int t = (dy + 1) * 3 + dx + 1;
#pragma unroll
                for (int c = 0; c < kCh; ++c) g[c] = fmaf(sw[c * 9 + t], dv, g[c]);
            }
        }
        float a[kCh];
        load_px32(a5 + idx * kCh, a);
#pragma unroll
        for (int c = 0; c < kCh; ++c)
            if (!(a[c] > 0.0f)) g[c] = 0.0f;
        store_px32(D4 + idx * kCh, g);
    }
    // dw5[c][t] += d5(p) a5(p + t)[c]: this thread's pixel p, all 9 taps
    if (live) {
        const float dv = __ldg(d5 + idx);
        atomicAdd(&acc[kCh * 9], dv);
        if (dv != 0.0f) {
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const int yy = wrapi2(y + dy, H);
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const int xx = wrapi2(x + dx, W);
                    float a[kCh];
                    load_px32(a5 + (((size_t)b * H + yy) * W + xx) * kCh, a);
                    const int t = (dy + 1) * 3 + dx + 1;
#pragma unroll
                    for (int c = 0; c < kCh; ++c) atomicAdd(&acc[c * 9 + t], dv * a[c]);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kCh * 9 + 1; i += blockDim.x) atomicAdd(&g5[i], acc[i]);
}

// Weight and bias gradients of a 32 -> 32 layer: dW[o][i][t] = sum_p D(p)[o]
// a(p + t)[i], db[o] = sum_p D(p)[o]. A CTA takes one row segment of 64
// pixels at a time (persistent over many), with the three input rows and the
// gradient rows staged in shared memory as FP32; thread (t, o4, i8) owns a
// 4 x 8 block of (out, in) for tap t: 9 x 8 x 4 = 288 threads.
constexpr int kWgSeg = 64;
__global__ void __launch_bounds__(288) cnn_wgrad32_kernel(const __nv_bfloat16 *__restrict__ act,
                                                          const __nv_bfloat16 *__restrict__ D,
                                                          int B, int H, int W,
                                                          float *__restrict__ gw) {
    __shared__ float sa[3][kWgSeg + 2][kCh + 1];
    __shared__ float sd[kWgSeg][kCh + 1];
    const int tid = threadIdx.x;
    const int t = tid / 32, o4 = (tid >> 2) & 7, i8 = tid & 3;
    const int dy = t / 3 - 1, dx = t % 3 - 1;
    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[a][c] = 0.0f;
    const int segs = (W + kWgSeg - 1) / kWgSeg;
    const long long items = (long long)B * H * segs;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int b = (int)(it / ((long long)H * segs));
        const int rem = (int)(it - (long long)b * H * segs);
        const int y = rem / segs, x0 = (rem - (rem / segs) * segs) * kWgSeg;
        __syncthreads();
        for (int e = tid; e < 3 * (kWgSeg + 2) * (kCh / 8); e += blockDim.x) {
            const int r = e / ((kWgSeg + 2) * 4), q = e - r * (kWgSeg + 2) * 4;
            const int p = q >> 2, j = q & 3;
            const int yy = wrapi2(y + r - 1, H);
            const int xx = ((x0 - 1 + p) % W + W) % W;
            const uint4 u = __ldg(reinterpret_cast<const uint4 *>(
                act + (((size_t)b * H + yy) * W + xx) * kCh + 8 * j));
            const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = __bfloat1622float2(h[k]);
                sa[r][p][8 * j + 2 * k] = f.x;
                sa[r][p][8 * j + 2 * k + 1] = f.y;
            }
        }
        for (int e = tid; e < kWgSeg * 4; e += blockDim.x) {
            const int p = e >> 2, j = e & 3;
            const int xx = x0 + p;
            uint4 u = make_uint4(0u, 0u, 0u, 0u);
            if (xx < W)
                u = __ldg(reinterpret_cast<const uint4 *>(D + (((size_t)b * H + y) * W + xx) * kCh +
                                                          8 * j));
            const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = __bfloat1622float2(h[k]);
                sd[p][8 * j + 2 * k] = f.x;
                sd[p][8 * j + 2 * k + 1] = f.y;
            }
        }
        __syncthreads();
        for (int p = 0; p < kWgSeg; ++p) {
            float dv[4], av[8];
#pragma unroll
            for (int a = 0; a < 4; ++a) dv[a] = sd[p][4 * o4 + a];
#pragma unroll
            for (int c = 0; c < 8; ++c) av[c] = sa[dy + 1][p + 1 + dx][8 * i8 + c];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(dv[a], av[c], acc[a][c]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c)
            atomicAdd(&gw[((size_t)(4 * o4 + a) * kCh + 8 * i8 + c) * 9 + t], acc[a][c]);
}

// Bias gradient of a 32-channel layer: db[o] = sum_p D(p)[o].
__global__ void __launch_bounds__(256) cnn_bgrad32_kernel(const __nv_bfloat16 *__restrict__ D,
                                                          size_t P, float *__restrict__ gb) {
    __shared__ float acc[kCh];
    if (threadIdx.x < kCh) acc[threadIdx.x] = 0.0f;
    __syncthreads();
    float loc[kCh];
#pragma unroll
    for (int c = 0; c < kCh; ++c) loc[c] = 0.0f;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P;
         p += (size_t)gridDim.x * blockDim.x) {
        float v[kCh];
        load_px32(D + p * kCh, v);
#pragma unroll
        for (int c = 0; c < kCh; ++c) loc[c] += v[c];
    }
#pragma unroll
    for (int c = 0; c < kCh; ++c) {
        float s = loc[c];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&acc[c], s);
    }
    __syncthreads();
    if (threadIdx.x < kCh) atomicAdd(&gb[threadIdx.x], acc[threadIdx.x]);
}

// Weight and bias gradients of the first layer (2 -> 32): dW0[o][i][t] =
// sum_p D0(p)[o] x_i(p + t), x = (up / s, pan / s). One thread per pixel,
// per-CTA sums in shared memory.
__global__ void __launch_bounds__(256) cnn_wgrad_first_kernel(
    const float *__restrict__ up, const float *__restrict__ pan, size_t pan_stride,
    const __nv_bfloat16 *__restrict__ D0, int B, int H, int W, float *__restrict__ g0) {
    __shared__ float acc[kCh * 18 + kCh];
    for (int i = threadIdx.x; i < kCh * 18 + kCh; i += blockDim.x) acc[i] = 0.0f;
    __syncthreads();
    const size_t HW = (size_t)H * W;
    const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx < (size_t)B * HW) {
        const int b = (int)(idx / HW);
        const int rem = (int)(idx - (size_t)b * HW), y = rem / W, x = rem - (rem / W) * W;
        const float *u = up + (size_t)b * HW;
        const float *pp = pan + (size_t)b * pan_stride;
        float in[2][9];
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int yy = wrapi2(y + dy, H);
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int xx = wrapi2(x + dx, W);
                in[0][(dy + 1) * 3 + dx + 1] = __ldg(u + (size_t)yy * W + xx) * (1.0f / kScale);
                in[1][(dy + 1) * 3 + dx + 1] = __ldg(pp + (size_t)yy * W + xx) * (1.0f / kScale);
            }
        }
        float d[kCh];
        load_px32(D0 + idx * kCh, d);
        for (int o = 0; o < kCh; ++o) {
            if (d[o] == 0.0f) continue;
            atomicAdd(&acc[kCh * 18 + o], d[o]);
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                atomicAdd(&acc[(o * 2) * 9 + t], d[o] * in[0][t]);
                atomicAdd(&acc[(o * 2 + 1) * 9 + t], d[o] * in[1][t]);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kCh * 18 + kCh; i += blockDim.x) atomicAdd(&g0[i], acc[i]);
}

// Adam (Kingma & Ba 2015, Algorithm 1) over the parameter vector.
__global__ void cnn_adam_kernel(float *__restrict__ p, const float *__restrict__ g,
                                float *__restrict__ m, float *__restrict__ v, int n, float lr,
                                float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

int blocks_for(size_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// Offsets of each layer's weights and biases in the parameter vector.
void cnn_layout(int *w_off, int *b_off) {
    static const int widths[7] = {2, 32, 32, 32, 32, 32, 1};
    int o = 0;
    for (int l = 0; l < 6; ++l) {
        w_off[l] = o;
        o += widths[l + 1] * widths[l] * 9;
        b_off[l] = o;
        o += widths[l + 1];
    }
    w_off[6] = o;  // total
}

void launch_cnn_first(const float *up, const float *pan, size_t pan_stride, const float *prm,
                      int B, int H, int W, __nv_bfloat16 *a1, cudaStream_t st) {
    const size_t P = (size_t)B * H * (W / 2);
    cnn_first_kernel<<<blocks_for(P, 256), 256, 0, st>>>(up, pan, pan_stride, prm, B, H, W, a1);
}

void launch_cnn_last(const __nv_bfloat16 *a5, const float *up, const float *prm5, int B, int H,
                     int W, float *z, const float *target, const float *weight, float *d5,
                     double *loss, cudaStream_t st) {
    const size_t P = (size_t)B * H * W;
    cnn_last_kernel<<<blocks_for(P, 256), 256, 0, st>>>(a5, up, prm5, B, H, W, z, target, weight,
                                                        1.0f / (float)P, d5, loss);
}

void launch_cnn_last_bwd(const __nv_bfloat16 *a5, const float *d5, const float *prm5, int B,
                         int H, int W, __nv_bfloat16 *D4, float *g5, cudaStream_t st) {
    const size_t P = (size_t)B * H * W;
    cnn_last_bwd_kernel<<<blocks_for(P, 256), 256, 0, st>>>(a5, d5, prm5, B, H, W, D4, g5);
}

void launch_cnn_wgrad32(const __nv_bfloat16 *act, const __nv_bfloat16 *D, int B, int H, int W,
                        float *gw, float *gb, int num_sms, cudaStream_t st) {
    const int segs = (W + kWgSeg - 1) / kWgSeg;
    const long long items = (long long)B * H * segs;
    int grid = 2 * num_sms;
    if (grid > items) grid = (int)items;
    cnn_wgrad32_kernel<<<grid, 288, 0, st>>>(act, D, B, H, W, gw);
    const size_t P = (size_t)B * H * W;
    int gb_blocks = blocks_for(P, 256 * 16);
    if (gb_blocks > 4 * num_sms) gb_blocks = 4 * num_sms;
    cnn_bgrad32_kernel<<<gb_blocks, 256, 0, st>>>(D, P, gb);
}

void launch_cnn_wgrad_first(const float *up, const float *pan, size_t pan_stride,
                            const __nv_bfloat16 *D0, int B, int H, int W, float *g0,
                            cudaStream_t st) {
    const size_t P = (size_t)B * H * W;
    cnn_wgrad_first_kernel<<<blocks_for(P, 256), 256, 0, st>>>(up, pan, pan_stride, D0, B, H, W,
                                                               g0);
}

void launch_cnn_adam(float *p, const float *g, float *m, float *v, int n, int step, float lr,
                     float b1, float b2, float eps, cudaStream_t st) {
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    cnn_adam_kernel<<<blocks_for(n, 256), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
}

}  // namespace ps
