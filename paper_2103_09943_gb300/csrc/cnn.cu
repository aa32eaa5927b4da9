// The learned warm start's 3 x 3 convolutions with 32 input and 32 output
// channels on the 5th-generation tensor cores (tcgen05, BF16 operands, FP32
// accumulators in TMEM), sm_103a.
//
// Implicit GEMM per tile of 128 consecutive pixels of one row:
//   D[128 px][32 out] = sum over 9 taps of A_tap[128 px][32 in] B_tap[32 in][32 out]
// i.e. 18 MMAs of M = 128, N = 32, K = 16 per row, issued as 24 MMAs (N = 32
// and 64) per pair of rows. Activations are NHWC BF16 (64 B
// per pixel). Three input rows of 130 pixels (the tile and its halo) sit in
// shared memory as four planes of 8-channel chunks, plane[j][p] = channels
// 8j .. 8j+7 of pixel p (16 B): in this layout the A operand of every tap is
// a canonical no-swizzle K-major matrix (core matrices of 8 pixels x 16 B,
// 128 B apart along M, one plane apart along K) whose start address is the
// tap's pixel shift, so no im2col copy is made. The B operand (weights) is
// packed once per launch in the same core-matrix form, the three vertical
// taps of each dx stacked along N.
//
// Each CTA walks vertical strips 128 pixels wide, row after row, as a
// warp-specialised pipeline (a cp.async producer warp, one MMA-issuing
// thread, four epilogue warps) coupled by mbarriers; see conv32_tc_kernel.
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
constexpr int kWStack = 3 * kCh;         // B rows of one dx: W(dy = 1), W(0), W(-1)
constexpr int kWChunk = kWStack * 16;    // bytes of one 8-channel K chunk of a dx block
constexpr int kWdx = 4 * kWChunk;        // bytes of one dx block
constexpr int kWBytes = 3 * kWdx;
constexpr uint32_t kIdesc32 = umma_idesc_bf16(128, 32);
constexpr uint32_t kIdesc64 = umma_idesc_bf16(128, 64);

__device__ __forceinline__ int wrapm(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// The B operand of one layer, K-major: for each horizontal tap offset dx the
// three vertical taps are stacked along N, rows 32 (1 - dy) + n, so that
// W(dy = 1) | W(0) and W(0) | W(-1) are each one N = 64 operand. Element
// (dx, dy, k, n) sits at byte (dx + 1) * kWdx + (k / 8) * kWChunk
// + (32 (1 - dy) + n) * 16 + (k % 8) * 2, k the input and n the output
// channel of the GEMM. Forward: n = out, k = in, the tap as is. Backward data
// (the adjoint): n = in, k = out and the tap mirrored.
__global__ void pack_w32_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ out,
                                int adjoint) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 9 * kCh * kCh) return;
    const int dxi = i / (kWdx / 2), r = i - dxi * (kWdx / 2);
    const int j = r / (kWChunk / 2), r2 = r - j * (kWChunk / 2);
    const int ns = r2 / 8, e = r2 & 7;
    const int dy = 1 - ns / kCh, n = ns % kCh;
    const int k = 8 * j + e;
    const int tap = (dy + 1) * 3 + dxi;
    const float v = adjoint ? w[((size_t)k * kCh + n) * 9 + (8 - tap)]
                            : w[((size_t)n * kCh + k) * 9 + tap];
    out[i] = __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------------------
// Warp-specialised pipeline. Each CTA (six warps) walks its work items, each
// a vertical strip 128 pixels wide and a run of rows, with three roles that
// only meet at mbarriers:
//   warp 0     producer: cp.async of input rows (130 pixels with the halo)
//              into a ring of kRingWs slots; kDepth rows in flight per lane;
//              a row is announced on full[slot] (32 lane arrivals) once its
//              copies have landed and been fenced for the async proxy
//   warp 1     MMA issuer (one thread): per pair of output rows k, k + 1,
//              one of kAcc TMEM accumulators of 64 columns (row k in 0..31,
//              k + 1 in 32..63). Input row k - 1 feeds only row k and row k + 2
//              only row k + 1 (N = 32, each starts its half); rows k and k + 1
//              feed both (N = 64 with the weights stacked along N): 24 MMAs
//              of K = 16 for two rows instead of 36. Then commits to
//              acc_full[acc] and to empty[slot] of input rows no longer needed
//   warps 2-9  epilogue, two groups of four warps taking alternate output
//              rows (the fused last layer, whose rows chain, uses group 0
//              only): warp w reads TMEM lanes 32 (w mod 4) .. + 31 (one pixel
//              per thread), releases the accumulator on acc_empty[acc] (4 warp
//              arrivals), then bias + ReLU (or the backward mask) and the BF16
//              store, or the fused last layer
// All three roles follow the same item and row sequence, so slot and
// accumulator phases are counted, not exchanged. Every wait is bounded and
// also ends when another role has set the CTA's abort flag.
// ---------------------------------------------------------------------------
constexpr int kRingWs = 8;
constexpr int kDepth = 4;
// an MMA group reads four input rows and frees two; the producer holds
// kDepth - 1 issued rows unannounced: the ring must hold kDepth + 3 rows
static_assert(kRingWs >= kDepth + 3, "ring too short for the prefetch depth");
constexpr int kAcc = 4;
constexpr int kWsThreads = 320;
constexpr int kExtraW5 = 304 * 4;
constexpr int kExtraX = kTileM * 9 * 4;
constexpr int kOffRing = kWBytes;
constexpr int kOffBias = kOffRing + kRingWs * kRowB;
constexpr int kOffW5 = kOffBias + kCh * 4;
constexpr int kOffX = kOffW5 + kExtraW5;
constexpr int kOffBar = kOffX + kExtraX;  // 8-byte aligned
constexpr int kNumBar = 2 * kRingWs + 2 * kAcc + 1;
constexpr int kConvSmemWs = kOffBar + kNumBar * 8 + 16;
static_assert(kOffBar % 8 == 0, "mbarriers need 8-byte alignment");

struct ConvItem {
    int b, x0, ys, ye, ya, yb;
};

template <int MODE>
__device__ __forceinline__ ConvItem conv_item(const Conv32Args &a, int item, int strips,
                                              int chunks) {
    constexpr int TS = (MODE == CONV_LAST) ? kTileM - 2 : kTileM;
    ConvItem it;
    it.b = item / (strips * chunks);
    const int rem = item - it.b * strips * chunks;
    const int sx = rem / chunks, ch = rem - (rem / chunks) * chunks;
    // the fused last layer keeps the 126 pixels whose 3 x 3 neighbourhood
    // lies in the tile: its tiles start one pixel early and advance by 126,
    // and it computes one extra layer-4 row above and below its rows
    it.x0 = sx * TS - (MODE == CONV_LAST ? 1 : 0);
    it.ya = ch * a.rpi;
    it.yb = min(a.H, it.ya + a.rpi);
    it.ys = it.ya - (MODE == CONV_LAST ? 1 : 0);
    it.ye = it.yb + (MODE == CONV_LAST ? 1 : 0);
    return it;
}

template <int MODE>
__global__ void __launch_bounds__(kWsThreads, 2) conv32_tc_kernel(Conv32Args a) {
    extern __shared__ __align__(1024) uint8_t csm[];
    uint8_t *wsm = csm;
    float *sbias = reinterpret_cast<float *>(csm + kOffBias);
    float *sw5 = reinterpret_cast<float *>(csm + kOffW5);
    float *sxc = reinterpret_cast<float *>(csm + kOffX);
    uint64_t *bars = reinterpret_cast<uint64_t *>(csm + kOffBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + kNumBar);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int H = a.H, W = a.W;

    for (int i = tid; i < kWBytes / 16; i += kWsThreads)
        reinterpret_cast<uint4 *>(wsm)[i] = __ldg(reinterpret_cast<const uint4 *>(a.wpack) + i);
    if (tid < kCh) sbias[tid] = a.bias ? a.bias[tid] : 0.0f;
    // the fused last layer's weights transposed so that four input channels
    // are one 16-byte load: sw5[t * 32 + c] = w5[c][t], bias at 288
    if (MODE == CONV_LAST) {
        for (int i = tid; i < 288; i += kWsThreads) sw5[(i % 9) * 32 + i / 9] = a.w5[i];
        if (tid == 0) sw5[288] = a.w5[288];
    }
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (uint32_t)(kRingWs + s); };
    auto accf_bar = [&](int k) { return bar0 + 8u * (uint32_t)(2 * kRingWs + k); };
    auto acce_bar = [&](int k) { return bar0 + 8u * (uint32_t)(2 * kRingWs + kAcc + k); };
    const uint32_t done_bar = bar0 + 8u * (uint32_t)(2 * kRingWs + 2 * kAcc);
    if (tid == 0) {
        for (int s = 0; s < kRingWs; ++s) {
            mbar_init(full_bar(s), 32);
            mbar_init(empty_bar(s), 1);
        }
        for (int k = 0; k < kAcc; ++k) {
            mbar_init(accf_bar(k), 1);
            // the epilogue warps that read an accumulator: both groups in the
            // plain form, group 0 alone in the fused last layer
            mbar_init(acce_bar(k), MODE == CONV_LAST ? 4 : 8);
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(smem_u32(tslot), 64 * kAcc);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t w_u32 = smem_u32(wsm), ring_u32 = smem_u32(csm + kOffRing);

    constexpr int TS = (MODE == CONV_LAST) ? kTileM - 2 : kTileM;
    const int strips = (W + TS - 1) / TS;
    const int chunks = (H + a.rpi - 1) / a.rpi;
    const int items = a.N * strips * chunks;
    auto fail = [&]() {
        *abort_flag = 1;
        if (a.err) atomicExch(a.err, 1);
    };

    if (warp == 0) {
        // ---------------- producer ----------------
        uint32_t q = 0;  // input rows issued by this CTA
        int pend = 0;    // issued rows not yet announced
        bool ok = true;
        // a lane's 16-byte chunks of a halo row: chunk idx = lane + 32 m is
        // plane j = idx & 3 of pixel p = idx >> 2; the same columns for every
        // row of an item, so their offsets are computed once per item
        constexpr int kChunks = (kHalo * 4 + 31) / 32;
        uint32_t soff[kChunks], doff[kChunks];
        for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
            const ConvItem it = conv_item<MODE>(a, item, strips, chunks);
            const __nv_bfloat16 *inb = a.in + (size_t)it.b * H * W * kCh;
            const int n_in = it.ye - it.ys + 2;
#pragma unroll
            for (int m = 0; m < kChunks; ++m) {
                const int idx = lane + 32 * m;
                const int p = idx >> 2, j = idx & 3;
                soff[m] = (uint32_t)(wrapm(it.x0 - 1 + p, W) * kCh + j * 8);
                doff[m] = (uint32_t)(j * kPlane + p * 16);
            }
            for (int i = 0; i < n_in; ++i, ++q) {
                const int s = (int)(q % kRingWs);
                const uint32_t u = q / kRingWs;
                if (u >= 1)
                    ok = __all_sync(0xffffffffu,
                                    mbar_wait_or_abort(empty_bar(s), (u - 1) & 1u, abort_flag));
                if (!ok) break;
                const int yy = wrapm(it.ys - 1 + i, H);
                const __nv_bfloat16 *src = inb + (size_t)yy * W * kCh;
                const uint32_t dst = ring_u32 + s * kRowB;
#pragma unroll
                for (int m = 0; m < kChunks; ++m)
                    if (lane + 32 * m < kHalo * 4) cp_async16(dst + doff[m], src + soff[m]);
                cp_async_commit();
                if (pend == kDepth - 1) {
                    // the row issued kDepth - 1 rows ago has landed
                    cp_async_wait<kDepth - 1>();
                    fence_async_smem();
                    mbar_arrive(full_bar((int)((q - (kDepth - 1)) % kRingWs)));
                } else {
                    ++pend;
                }
            }
        }
        cp_async_wait<0>();
        fence_async_smem();
        if (ok) {
            for (int k = pend; k >= 1; --k) mbar_arrive(full_bar((int)((q - k) % kRingWs)));
        } else {
            fail();
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            uint32_t q = 0, o = 0;
            bool ok = true;
            auto wait_full = [&](uint32_t row) {
                return mbar_wait_or_abort(full_bar((int)(row % kRingWs)), (row / kRingWs) & 1u,
                                          abort_flag);
            };
            // descriptors: B per (dx, K half, stacked slice) fixed, slice 0 at
            // W(1) (N = 64: W(1) | W(0)), 1 at W(0) (W(0) | W(-1)), 2 at W(-1);
            // A is the ring base descriptor plus the 16-byte-unit offset of
            // slot, K half and dx
            uint64_t bdesc[3][2][3];
#pragma unroll
            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                for (int sk = 0; sk < 2; ++sk)
#pragma unroll
                    for (int sl = 0; sl < 3; ++sl)
                        bdesc[dx][sk][sl] =
                            umma_desc(w_u32 + dx * kWdx + 2 * sk * kWChunk + sl * kCh * 16,
                                      kWChunk, 128);
            const uint64_t adesc0 = umma_desc(ring_u32, kPlane, 128);
            // one input row times one stacked slice into D columns dcol ..
            auto mma_row = [&](uint32_t in_seq, uint32_t d, int sl, uint32_t idesc, bool &first) {
                const uint64_t ar = adesc0 + (uint64_t)((in_seq % kRingWs) * (kRowB >> 4));
#pragma unroll
                for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                    for (int sk = 0; sk < 2; ++sk) {
                        const uint64_t ad = ar + (uint64_t)((2 * sk * kPlane + dx * 16) >> 4);
                        umma_bf16(d, ad, bdesc[dx][sk][sl], idesc, first ? 0u : 1u);
                        first = false;
                    }
            };
            for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
                const ConvItem it = conv_item<MODE>(a, item, strips, chunks);
                const int n_out = it.ye - it.ys, n_in = n_out + 2;
                int waited = 0, freed = 0;  // input rows of the item waited for, released
                // output rows k, k + 1 (one MMA group, one accumulator of 64
                // columns: row k in columns 0..31, row k + 1 in 32..63) read
                // input rows k .. k + 3
                for (int k = 0; k < n_out && ok; k += 2, ++o) {
                    const int cnt = min(2, n_out - k);
                    for (; waited < k + cnt + 2 && ok; ++waited) ok = wait_full(q + waited);
                    const int acc = (int)(o % kAcc);
                    const uint32_t v = o / kAcc;
                    if (ok && v >= 1)
                        ok = mbar_wait_or_abort(acce_bar(acc), (v - 1) & 1u, abort_flag);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t d = tbase + (uint32_t)(acc * 64);
                    const uint32_t r0 = q + (uint32_t)k;
                    if (cnt == 2) {
                        // each D half starts fresh with its one-tap input row,
                        // then the two shared rows add to both halves at once
                        bool f0 = true, f1 = true, f2 = false;
                        mma_row(r0, d, 2, kIdesc32, f0);            // row k - 1: W(-1) -> k
                        mma_row(r0 + 3, d + 32, 0, kIdesc32, f1);   // row k + 2: W(1) -> k + 1
                        mma_row(r0 + 1, d, 1, kIdesc64, f2);        // row k: W(0) | W(-1)
                        mma_row(r0 + 2, d, 0, kIdesc64, f2);        // row k + 1: W(1) | W(0)
                    } else {
                        bool f0 = true;
                        mma_row(r0, d, 2, kIdesc32, f0);
                        mma_row(r0 + 1, d, 1, kIdesc32, f0);
                        mma_row(r0 + 2, d, 0, kIdesc32, f0);
                    }
                    umma_commit(accf_bar(acc));
                    // input rows below the next group's first are not read again
                    const int keep = (k + cnt < n_out) ? k + cnt : n_in;
                    for (; freed < keep; ++freed)
                        umma_commit(empty_bar((int)((q + freed) % kRingWs)));
                }
                q += (uint32_t)n_in;
            }
            if (!ok) fail();
            // every MMA issued has completed before the CTA frees its TMEM
            if (o > 0) {
                umma_commit(done_bar);
                mbar_wait_bounded(done_bar, 0);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue ----------------
        const int eg = warp & 3;             // TMEM lane group of this warp
        const int pix = 32 * eg + lane;      // pixel of the tile
        const int grp = (warp - 2) >> 2;     // row k + grp of each MMA group
        uint32_t o = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < items && ok && (MODE != CONV_LAST || grp == 0);
             item += gridDim.x) {
            const ConvItem it = conv_item<MODE>(a, item, strips, chunks);
            const int n_out = it.ye - it.ys;
            const int x = it.x0 + pix;
            float racc[3] = {0.f, 0.f, 0.f};  // last layer: output rows y - 1, y, y + 1
            // the fused last layer's row (exchange with the neighbours of the
            // row, 3 running output rows) or the plain store of one row
            auto process_row = [&](int y, float *vals) {
                if (MODE == CONV_LAST) {
                    // act5 = ReLU(conv + bias) at this pixel, then its 9
                    // per-tap partial sums of the last layer: output
                    // (y - dy, x - dx) takes tap (dy, dx) of (y, x)
#pragma unroll
                    for (int c = 0; c < kCh; ++c) vals[c] = fmaxf(vals[c] + sbias[c], 0.0f);
#pragma unroll
                    for (int t = 0; t < 9; ++t) {
                        const float4 *w4 = reinterpret_cast<const float4 *>(sw5 + t * 32);
                        float sacc = 0.0f;
#pragma unroll
                        for (int qq = 0; qq < 8; ++qq) {
                            const float4 wv = w4[qq];
                            sacc = fmaf(wv.x, vals[4 * qq], sacc);
                            sacc = fmaf(wv.y, vals[4 * qq + 1], sacc);
                            sacc = fmaf(wv.z, vals[4 * qq + 2], sacc);
                            sacc = fmaf(wv.w, vals[4 * qq + 3], sacc);
                        }
                        sxc[t * kTileM + pix] = sacc;
                    }
                    named_sync(1, 128);
                    if (pix >= 1 && pix <= kTileM - 2) {
#pragma unroll
                        for (int dx = -1; dx <= 1; ++dx) {
                            // tap (dy, dx) of pixel pix + dx feeds output row y - dy
                            racc[0] += sxc[(2 * 3 + dx + 1) * kTileM + pix + dx];  // dy = +1
                            racc[1] += sxc[(1 * 3 + dx + 1) * kTileM + pix + dx];  // dy = 0
                            racc[2] += sxc[(0 * 3 + dx + 1) * kTileM + pix + dx];  // dy = -1
                        }
                        const int yo = y - 1;
                        if (yo >= it.ya && yo < it.yb && x < W) {
                            const size_t oo = ((size_t)it.b * H + yo) * W + x;
                            a.z[oo] = __ldg(a.up + oo) + 255.0f * (racc[0] + sw5[288]);
                        }
                    }
                    racc[0] = racc[1];
                    racc[1] = racc[2];
                    racc[2] = 0.0f;
                    named_sync(1, 128);
                    return;
                }
                if (x >= W) return;
                const size_t oo = (((size_t)it.b * H + y) * W + x) * kCh;
                if (a.mask) {
                    const uint4 *mp = reinterpret_cast<const uint4 *>(a.mask + oo);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        const uint4 m = __ldg(mp + qq);
                        const __nv_bfloat16 *mh = reinterpret_cast<const __nv_bfloat16 *>(&m);
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (!(__bfloat162float(mh[e]) > 0.0f)) vals[8 * qq + e] = 0.0f;
                    }
                }
#pragma unroll
                for (int c = 0; c < kCh; ++c) {
                    vals[c] += sbias[c];
                    if (a.relu) vals[c] = fmaxf(vals[c], 0.0f);
                }
                uint4 pk[4];
                __nv_bfloat162 *ph = reinterpret_cast<__nv_bfloat162 *>(pk);
#pragma unroll
                for (int c = 0; c < kCh / 2; ++c)
                    ph[c] = __floats2bfloat162_rn(vals[2 * c], vals[2 * c + 1]);
                uint4 *op = reinterpret_cast<uint4 *>(a.out + oo);
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) op[qq] = pk[qq];
            };
            // one accumulator per pair of output rows (k in columns 0..31,
            // k + 1 in 32..63): group g of the plain epilogue takes row
            // k + g; the fused last layer takes both rows in order
            for (int k = 0; k < n_out; k += 2, ++o) {
                const int cnt = min(2, n_out - k);
                const int acc = (int)(o % kAcc);
                const uint32_t v = o / kAcc;
                ok = mbar_wait_or_abort(accf_bar(acc), v & 1u, abort_flag);
                // the fused last layer exchanges partial sums among the four
                // epilogue warps: they must agree to go on
                if (MODE == CONV_LAST) ok = named_and(1, 128, ok);
                ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
                if (!ok) break;
                tc_fence_after();
                const uint32_t tl = tbase + ((uint32_t)(32 * eg) << 16) + (uint32_t)(acc * 64);
                float vals[32];
                if (MODE == CONV_LAST) {
                    for (int h = 0; h < cnt; ++h) {
                        tmem_ld32(tl + (uint32_t)(32 * h), vals);
                        process_row(it.ys + k + h, vals);
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(acce_bar(acc));
                } else {
                    const bool mine = grp < cnt;
                    if (mine) tmem_ld32(tl + (uint32_t)(32 * grp), vals);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(acce_bar(acc));
                    if (mine) process_row(it.ys + k + grp, vals);
                }
            }
        }
        if (!ok) fail();
    }
    // every role is done: its MMAs were committed and waited on by the
    // epilogue, its copies waited for by the producer
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, 64 * kAcc);
    }
}

}  // namespace

size_t conv32_smem_bytes() { return (size_t)kConvSmemWs; }

void launch_pack_w32(const float *w, void *out, int adjoint, cudaStream_t st) {
    pack_w32_kernel<<<(9 * kCh * kCh + 255) / 256, 256, 0, st>>>(
        w, static_cast<__nv_bfloat16 *>(out), adjoint);
}

void launch_conv32(const Conv32Args &a, int num_sms, cudaStream_t st) {
    const int ts = a.mode == CONV_LAST ? kTileM - 2 : kTileM;
    const int strips = (a.W + ts - 1) / ts;
    const int chunks = (a.H + a.rpi - 1) / a.rpi;
    const int items = a.N * strips * chunks;
    int grid = 2 * num_sms;
    if (grid > items) grid = items;
    switch (a.mode) {
        case CONV_LAST:
            conv32_tc_kernel<CONV_LAST><<<grid, kWsThreads, kConvSmemWs, st>>>(a);
            break;
        default: conv32_tc_kernel<CONV_PLAIN><<<grid, kWsThreads, kConvSmemWs, st>>>(a); break;
    }
}

cudaError_t cnn_set_attrs() {
    cudaError_t e = cudaFuncSetAttribute(conv32_tc_kernel<CONV_PLAIN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmemWs);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(conv32_tc_kernel<CONV_LAST>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmemWs);
    return e;
}

}  // namespace ps
