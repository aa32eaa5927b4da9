// The learned warm start's 3 x 3 convolutions with 32 input and 32 output
// channels on the 5th-generation tensor cores (tcgen05, BF16 operands, FP32
// accumulators in TMEM), sm_103a.
//
// Implicit GEMM per tile of 128 consecutive pixels of one row:
//   D[128 px][32 out] = sum over 9 taps of A_tap[128 px][32 in] B_tap[32 in][32 out]
// i.e. 18 MMAs of M = 128, N = 32, K = 16. Activations are NHWC BF16 (64 B
// per pixel). Three input rows of 130 pixels (the tile and its halo) sit in
// shared memory as four planes of 8-channel chunks, plane[j][p] = channels
// 8j .. 8j+7 of pixel p (16 B): in this layout the A operand of every tap is
// a canonical no-swizzle K-major matrix (core matrices of 8 pixels x 16 B,
// 128 B apart along M, one plane apart along K) whose start address is the
// tap's pixel shift, so no im2col copy is made. The B operand (weights) is
// packed once per launch in the same core-matrix form.
//
// Each CTA walks a vertical strip 128 pixels wide, row after row, with a
// ring of five input rows: the load of row y + 3 (cp.async) and the
// epilogue of row y - 1 (tcgen05.ld, bias + ReLU or the backward mask, BF16
// store) overlap the MMAs of row y, which go to one of two TMEM accumulators.
// Every wait is bounded: on a timeout the kernel sets an error flag and
// stops.
#include <cuda_bf16.h>

#include "cnn_tc.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace ps {

namespace {

constexpr int kCh = 32;
constexpr int kTileM = 128;
constexpr int kHalo = kTileM + 2;
constexpr int kPlane = kHalo * 16;      // bytes of one 8-channel plane of a halo row
constexpr int kRowB = 4 * kPlane;       // bytes of one halo row
constexpr int kRing = 5;
constexpr int kWTap = 4 * kCh * 16;     // bytes of one tap's B operand
constexpr int kWBytes = 9 * kWTap;
constexpr int kConvSmem = kWBytes + kRing * kRowB + 256;
constexpr uint32_t kIdesc = umma_idesc_bf16(128, 32);

__device__ __forceinline__ int ring_slot(int y) { return ((y % kRing) + kRing) % kRing; }

__device__ __forceinline__ int wrapm(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// The B operand of one layer: element (tap, k, n) at byte
// tap * kWTap + (k / 8) * 512 + n * 16 + (k % 8) * 2, k the input and n the
// output channel of the GEMM. Forward: n = out, k = in, the tap as is.
// Backward data (the adjoint): n = in, k = out and the tap mirrored.
__global__ void pack_w32_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ out,
                                int adjoint) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 9 * kCh * kCh) return;
    const int tap = i / 1024, r = i - tap * 1024;
    const int j = r / 256, n = (r - j * 256) / 8, e = r & 7;
    const int k = 8 * j + e;
    const float v = adjoint ? w[((size_t)k * kCh + n) * 9 + (8 - tap)]
                            : w[((size_t)n * kCh + k) * 9 + tap];
    out[i] = __float2bfloat16_rn(v);
}

// Extra shared memory of the fused last layer: its parameters (289 floats,
// padded) and the exchange of its per-tap partial sums (128 pixels x 9).
constexpr int kExtraW5 = 304 * 4;
constexpr int kExtraX = kTileM * 9 * 4;
constexpr int kConvSmemFused = kConvSmem + kExtraW5 + kExtraX;

template <int MODE>
__global__ void __launch_bounds__(128, 3) conv32_tc_kernel(Conv32Args a) {
    extern __shared__ __align__(1024) uint8_t csm[];
    uint8_t *wsm = csm;
    uint8_t *ring = csm + kWBytes;
    float *sbias = reinterpret_cast<float *>(ring + kRing * kRowB);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sbias + kCh);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
    float *sw5 = reinterpret_cast<float *>(csm + kConvSmem);
    float *sxc = reinterpret_cast<float *>(csm + kConvSmem + kExtraW5);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int H = a.H, W = a.W;

    for (int i = tid; i < kWBytes / 16; i += 128)
        reinterpret_cast<uint4 *>(wsm)[i] = __ldg(reinterpret_cast<const uint4 *>(a.wpack) + i);
    if (tid < kCh) sbias[tid] = a.bias ? a.bias[tid] : 0.0f;
    // the fused last layer's weights transposed so that four input channels
    // are one 16-byte load: sw5[t * 32 + c] = w5[c][t], bias at 288
    if (MODE == CONV_LAST) {
        for (int i = tid; i < 288; i += 128) sw5[(i % 9) * 32 + i / 9] = a.w5[i];
        if (tid == 0) sw5[288] = a.w5[288];
    }
    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(tslot), 64);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t w_u32 = smem_u32(wsm), ring_u32 = smem_u32(ring);
    const uint32_t mb[2] = {smem_u32(&mbar[0]), smem_u32(&mbar[1])};
    uint32_t parity[2] = {0u, 0u};
    bool ok = true;

    // tiles of 128 pixels; the fused last layer keeps the 126 whose 3 x 3
    // neighbourhood lies in the tile, so its tiles start one pixel early and
    // advance by 126
    constexpr int TS = (MODE == CONV_LAST) ? kTileM - 2 : kTileM;
    const int strips = (W + TS - 1) / TS;
    const int chunks = (H + a.rpi - 1) / a.rpi;
    const int items = a.N * strips * chunks;
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
        const int b = item / (strips * chunks);
        const int rem = item - b * strips * chunks;
        const int sx = rem / chunks, ch = rem - (rem / chunks) * chunks;
        const int x0 = sx * TS - (MODE == CONV_LAST ? 1 : 0);
        const int ya = ch * a.rpi, yb = min(H, ya + a.rpi);
        // rows of this layer's output computed by the item
        const int ys = ya - (MODE == CONV_LAST ? 1 : 0), ye = yb + (MODE == CONV_LAST ? 1 : 0);
        const __nv_bfloat16 *inb = a.in + (size_t)b * H * W * kCh;
        float racc[3] = {0.f, 0.f, 0.f};  // last layer: output rows y - 1, y, y + 1

        auto load_row = [&](int yabs) {
            const int yy = wrapm(yabs, H);
            const uint32_t dst = ring_u32 + ring_slot(yabs) * kRowB;
            {
                const __nv_bfloat16 *src = inb + (size_t)yy * W * kCh;
                for (int idx = tid; idx < kHalo * 4; idx += 128) {
                    const int p = idx >> 2, j = idx & 3;
                    const int x = wrapm(x0 - 1 + p, W);
                    cp_async16(dst + j * kPlane + p * 16, src + (size_t)x * kCh + j * 8);
                }
            }
        };
        auto epilogue = [&](int y, int buf) {
            float v[32];
            tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(buf * 32), v);
            const int x = x0 + tid;
            if (MODE == CONV_LAST) {
                // act5 = ReLU(conv + bias) at this pixel, then its 9 per-tap
                // partial sums of the last layer, exchanged through shared
                // memory: output (y - dy, x - dx) takes tap (dy, dx) of (y, x)
#pragma unroll
                for (int c = 0; c < kCh; ++c) v[c] = fmaxf(v[c] + sbias[c], 0.0f);
#pragma unroll
                for (int t = 0; t < 9; ++t) {
                    const float4 *w4 = reinterpret_cast<const float4 *>(sw5 + t * 32);
                    float s = 0.0f;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 wv = w4[q];
                        s = fmaf(wv.x, v[4 * q], s);
                        s = fmaf(wv.y, v[4 * q + 1], s);
                        s = fmaf(wv.z, v[4 * q + 2], s);
                        s = fmaf(wv.w, v[4 * q + 3], s);
                    }
                    sxc[t * kTileM + tid] = s;
                }
                __syncthreads();
                if (tid >= 1 && tid <= kTileM - 2) {
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
                        // tap (dy, dx) of pixel tid + dx feeds output row y - dy
                        racc[0] += sxc[(2 * 3 + dx + 1) * kTileM + tid + dx];  // dy = +1
                        racc[1] += sxc[(1 * 3 + dx + 1) * kTileM + tid + dx];  // dy = 0
                        racc[2] += sxc[(0 * 3 + dx + 1) * kTileM + tid + dx];  // dy = -1
                    }
                    const int yo = y - 1;
                    if (yo >= ya && yo < yb && x < W) {
                        const size_t o = ((size_t)b * H + yo) * W + x;
                        a.z[o] = __ldg(a.up + o) + 255.0f * (racc[0] + sw5[288]);
                    }
                }
                racc[0] = racc[1];
                racc[1] = racc[2];
                racc[2] = 0.0f;
                __syncthreads();
                return;
            }
            if (x >= W) return;
            const size_t o = (((size_t)b * H + y) * W + x) * kCh;
            if (a.mask) {
                const uint4 *mp = reinterpret_cast<const uint4 *>(a.mask + o);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 m = __ldg(mp + q);
                    const __nv_bfloat16 *mh = reinterpret_cast<const __nv_bfloat16 *>(&m);
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        if (!(__bfloat162float(mh[e]) > 0.0f)) v[8 * q + e] = 0.0f;
                }
            }
#pragma unroll
            for (int c = 0; c < kCh; ++c) {
                v[c] += sbias[c];
                if (a.relu) v[c] = fmaxf(v[c], 0.0f);
            }
            uint4 pk[4];
            __nv_bfloat162 *ph = reinterpret_cast<__nv_bfloat162 *>(pk);
#pragma unroll
            for (int c = 0; c < kCh / 2; ++c) ph[c] = __floats2bfloat162_rn(v[2 * c], v[2 * c + 1]);
            uint4 *op = reinterpret_cast<uint4 *>(a.out + o);
#pragma unroll
            for (int q = 0; q < 4; ++q) op[q] = pk[q];
        };

        load_row(ys - 1);
        load_row(ys);
        load_row(ys + 1);
        cp_async_commit();
        load_row(ys + 2);
        cp_async_commit();
        for (int y = ys; y < ye; ++y) {
            const int buf = (y - ys) & 1;
            cp_async_wait<1>();  // rows y - 1 .. y + 1 are in
            fence_async_smem();
            ok = __syncthreads_and(ok) != 0;
            if (!ok) break;
            if (tid == 0) {
                tc_fence_after();
                const uint32_t d = tbase + (uint32_t)(buf * 32);
                int kk = 0;
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy) {
                    const uint32_t rb = ring_u32 + ring_slot(y + dy) * kRowB;
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int tap = (dy + 1) * 3 + (dx + 1);
#pragma unroll
                        for (int s = 0; s < 2; ++s) {
                            const uint64_t ad = umma_desc(rb + 2 * s * kPlane + (dx + 1) * 16,
                                                          kPlane, 128);
                            const uint64_t bd = umma_desc(w_u32 + tap * kWTap + 2 * s * 512, 512,
                                                          128);
                            umma_bf16(d, ad, bd, kIdesc, kk > 0 ? 1u : 0u);
                            ++kk;
                        }
                    }
                }
                umma_commit(mb[buf]);
            }
            if (y > ys) {
                // MMAs of row y - 1 done: its accumulator is readable and the
                // ring slot of row y - 2 is free
                const int pb = buf ^ 1;
                if (!mbar_wait_bounded(mb[pb], parity[pb])) {
                    ok = false;
                    if (a.err) atomicExch(a.err, 1);
                }
                ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
                parity[pb] ^= 1u;
                tc_fence_after();
            }
            // the fused last layer's epilogue holds CTA barriers: its
            // condition must be uniform across the CTA
            if (MODE == CONV_LAST) ok = __syncthreads_and(ok) != 0;
            load_row(y + 3);
            cp_async_commit();
            if (y > ys && ok) epilogue(y - 1, buf ^ 1);
            tc_fence_before();
        }
        if (ok) {
            const int lb = (ye - 1 - ys) & 1;
            if (!mbar_wait_bounded(mb[lb], parity[lb])) {
                ok = false;
                if (a.err) atomicExch(a.err, 1);
            }
            ok = __all_sync(0xffffffffu, ok);
            parity[lb] ^= 1u;
            tc_fence_after();
            if (MODE == CONV_LAST) ok = __syncthreads_and(ok) != 0;
            if (ok) epilogue(ye - 1, lb);
            tc_fence_before();
        }
        cp_async_wait<0>();
        ok = __syncthreads_and(ok) != 0;
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, 64);
    }
}

}  // namespace

size_t conv32_smem_bytes() { return (size_t)kConvSmemFused; }

void launch_pack_w32(const float *w, void *out, int adjoint, cudaStream_t st) {
    pack_w32_kernel<<<(9 * kCh * kCh + 255) / 256, 256, 0, st>>>(
        w, static_cast<__nv_bfloat16 *>(out), adjoint);
}

void launch_conv32(const Conv32Args &a, int num_sms, cudaStream_t st) {
    const int ts = a.mode == CONV_LAST ? kTileM - 2 : kTileM;
    const int strips = (a.W + ts - 1) / ts;
    const int chunks = (a.H + a.rpi - 1) / a.rpi;
    const int items = a.N * strips * chunks;
    int grid = 3 * num_sms;
    if (grid > items) grid = items;
    switch (a.mode) {
        case CONV_LAST: conv32_tc_kernel<CONV_LAST><<<grid, 128, kConvSmemFused, st>>>(a); break;
        default: conv32_tc_kernel<CONV_PLAIN><<<grid, 128, kConvSmem, st>>>(a); break;
    }
}

cudaError_t cnn_set_attrs() {
    cudaError_t e = cudaFuncSetAttribute(conv32_tc_kernel<CONV_PLAIN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(conv32_tc_kernel<CONV_LAST>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmemFused);
    return e;
}

}  // namespace ps
