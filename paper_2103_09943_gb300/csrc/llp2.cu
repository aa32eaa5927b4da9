// The prior part of the Z0 operator inside the CG loop, q = lam L M L p with
// p^T q per band (Eq. Z_ini_matting, matrix-free M of Eq. matting_matrix),
// two pixels per lane (sm_103a). Three forms, chosen per size by the
// autotuner: the general walk below (any window radius, one or two bands a
// CTA, loads ahead in registers or in a cp.async ring), and for 3 x 3
// windows the lean walks with two or four columns a lane (further down).
//
// Same register-streaming scheme as the general LLP kernel (a warp walks
// down a strip of columns keeping every stage of the chain -- Laplacian,
// window sums, affine fit, window sums, Laplacian -- as short rolling
// buffers of rows), but lane l owns the two adjacent columns 2l and 2l + 1
// of a 64-column strip. A horizontal neighbour at offset d of column 2l + e
// lives in lane l + floor((e + d) / 2): the shuffles per row stay those of
// one pixel per lane while each warp row yields 64 - 2G outputs instead of
// 32 - 2G, and the loads become one float2 of p and two float4 of
// statistics per lane.
#include "common.cuh"
#include "kernels.cuh"

namespace ps {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 4;

__device__ __forceinline__ int wrap2(int i, int n) {
    int m = i % n;
    return m < 0 ? m + n : m;
}

// Value at column 2 lane + E + D of the pair (v0, v1) held at columns
// 2 lane, 2 lane + 1.
template <int E, int D>
__device__ __forceinline__ float nbr(float v0, float v1) {
    constexpr int c = E + D;
    constexpr int o = (c >= 0) ? c / 2 : -((1 - c) / 2);  // floor(c / 2)
    constexpr int el = c - 2 * o;
    const float src = el ? v1 : v0;
    if constexpr (o == 0) return src;
    else if constexpr (o < 0) return __shfl_up_sync(kFull, src, (unsigned)(-o));
    else return __shfl_down_sync(kFull, src, (unsigned)o);
}

// Horizontal window sum over [-RW, RW] at both columns of the pair.
template <int RW, int E, int D = -RW>
__device__ __forceinline__ float hsum(float v0, float v1) {
    if constexpr (D > RW) {
        return 0.0f;
    } else {
        return nbr<E, D>(v0, v1) + hsum<RW, E, D + 1>(v0, v1);
    }
}

// Output rows per warp, two lengths per radius (the autotuner picks): longer
// walks spend less on the 2G halo rows, shorter ones give more warps. UNR is
// the depth of the rolling buffers that the walk's unrolled blocks must
// respect (3 for r = 1).
template <int RW>
struct Llp2Rows {
    static constexpr int LONG = (RW == 1) ? 66 : 64;
    static constexpr int SHORT = (RW == 1) ? 33 : 32;
    static constexpr int UNR = (RW == 1) ? 3 : 1;
};

// rows per warp of the lean kernels (r = 1): long and short walks
constexpr int kQ4Long = 64;
constexpr int kQ4Short = 32;

constexpr int llp_gcd(int a, int b) { return b ? llp_gcd(b, a % b) : a; }
constexpr int llp_lcm(int a, int b) { return a / llp_gcd(a, b) * b; }

// Asynchronous copies global -> shared (sm_80+ cp.async); each lane copies
// and later reads only its own bytes, so waiting on its own groups suffices.
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One ring slot of a warp: its 64 columns of p and the statistics of both
// columns of every lane, each array contiguous over the lanes.
struct LlpSlot {
    float2 p[32];
    float4 s0[32], s1[32];
};
constexpr int kRing = 8;  // rows the ring holds (PF = kRing selects it)

// Last CTA of a band: p^T A p = ||D B p||^2 + p^T (lam L^T M L) p, then
// alpha = rho / p^T A p, or the band stops with its status.
__device__ void llp_cg_finish(CgBand *bd, double tot, unsigned int nblk) {
    atomicAdd(&bd->pAp, tot);
    __threadfence();
    const unsigned int t = atomicAdd(&bd->cnt_apply, 1u);
    if (t == nblk - 1) {
        __threadfence();
        const double pAp = atomicAdd(&bd->pAp, 0.0) + bd->vv;
        const double rho = bd->rho;
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
            bd->alpha = rho / pAp;
        }
    }
}

template <int RW, int TY, int PF>
__global__ void __launch_bounds__(128) llp_cgq2_kernel(LlpArgs a) {
    // PF < kRing: the loads run PF rows ahead in registers; PF == kRing: they
    // run kRing - 1 rows ahead as asynchronous copies into a ring of kRing
    // rows per warp in shared memory
    constexpr bool RING = (PF == kRing);
    __shared__ LlpSlot ring[RING ? kWarps * kRing : 1];
    constexpr int G = 2 * RW + 2;
    constexpr int VALID = 64 - 2 * G;
    constexpr int NB = 2 * RW + 1;
    constexpr float nw = (float)(NB * NB);
    constexpr float inw = 1.0f / nw;
    __shared__ double red[kWarps];
    // band-minor grid: the CTAs of all bands of one strip run together and
    // read the shared PAN statistics once from memory, the rest from L2
    const int b = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (a.g->stop || a.bands[b].done) return;
    const int H = a.H, W = a.W;
    const int HWi = H * W;
    const size_t HW = (size_t)HWi;
    const int x0 = blockIdx.y * VALID;
    const int y0 = (blockIdx.z * kWarps + warp) * TY;
    const int xl = x0 - G + 2 * lane;  // even; W is even, so xl + 1 wraps with xl
    const int gx = wrap2(xl, W);
    const bool out_lane = lane >= G / 2 && lane < 32 - G / 2 && xl < W;
    const float *in = a.in + (size_t)b * HW;
    const float4 *st4 = a.st4;
    float part = 0.0f;

    if (y0 < H) {
        int rowIn = wrap2(y0 - G, H) * W;
        int rowA = wrap2(y0 - G - 1, H) * W;
        int rowD = wrap2(y0, H) * W;
        float pm2[2] = {0.f, 0.f}, pm1[2] = {0.f, 0.f}, p0[2] = {0.f, 0.f};
        float hA[2][NB], hIA[2][NB], ab[2][NB], ib[2][NB], ha[2][NB], hb[2][NB];
        float mub[2][RW + 1], sb[2][RW + 1];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
#pragma unroll
            for (int d = 0; d < NB; ++d) hA[e][d] = hIA[e][d] = ab[e][d] = ib[e][d] = ha[e][d] = hb[e][d] = 0.f;
#pragma unroll
            for (int d = 0; d <= RW; ++d) mub[e][d] = sb[e][d] = 0.f;
        }
        float mm2[2] = {0.f, 0.f}, mm1[2] = {0.f, 0.f}, m0[2] = {0.f, 0.f};
        // loads run PF rows ahead of their use (registers), or kRing - 1
        // rows ahead (the ring)
        constexpr int PFR = RING ? 1 : PF;
        float2 qp[PFR];
        float4 qs0[PFR], qs1[PFR];
        constexpr int PH = ((G + 1 + 2) / 3) * 3;
        float2 ph[PH];
#pragma unroll
        for (int d = 0; d < PH; ++d) ph[d] = make_float2(0.f, 0.f);
        LlpSlot *wr = ring + (RING ? warp * kRing : 0);
        int slot = 0;
        auto issue = [&](int sl) {
            cp_async8(&wr[sl].p[lane], in + rowIn + gx);
            cp_async16(&wr[sl].s0[lane], st4 + rowA + gx);
            cp_async16(&wr[sl].s1[lane], st4 + rowA + gx + 1);
            cp_async_commit();
            rowIn += W;
            if (rowIn == HWi) rowIn = 0;
            rowA += W;
            if (rowA == HWi) rowA = 0;
        };
        if constexpr (RING) {
#pragma unroll
            for (int k = 0; k < kRing - 1; ++k) issue(k);
        } else {
#pragma unroll
            for (int k = 0; k < PF; ++k) {
                qp[k] = *reinterpret_cast<const float2 *>(in + rowIn + gx);
                qs0[k] = st4[rowA + gx];
                qs1[k] = st4[rowA + gx + 1];
                rowIn += W;
                if (rowIn == HWi) rowIn = 0;
                rowA += W;
                if (rowA == HWi) rowA = 0;
            }
        }

        auto advance = [&]() -> float2 {
            float2 pin;
            float4 s0, s1;
            if constexpr (RING) {
                // this row's copies have landed once at most kRing - 2
                // younger groups are pending; its slot is read, then the
                // slot consumed one step earlier is refilled
                cp_async_wait<kRing - 2>();
                pin = wr[slot].p[lane];
                s0 = wr[slot].s0[lane];
                s1 = wr[slot].s1[lane];
                issue(slot == 0 ? kRing - 1 : slot - 1);
                slot = (slot == kRing - 1) ? 0 : slot + 1;
            } else {
                pin = qp[0];
                s0 = qs0[0];
                s1 = qs1[0];
#pragma unroll
                for (int k = 0; k < PF - 1; ++k) {
                    qp[k] = qp[k + 1];
                    qs0[k] = qs0[k + 1];
                    qs1[k] = qs1[k + 1];
                }
                qp[PF - 1] = *reinterpret_cast<const float2 *>(in + rowIn + gx);
                qs0[PF - 1] = st4[rowA + gx];
                qs1[PF - 1] = st4[rowA + gx + 1];
                rowIn += W;
                if (rowIn == HWi) rowIn = 0;
                rowA += W;
                if (rowA == HWi) rowA = 0;
            }
#pragma unroll
            for (int d = 0; d < PH - 1; ++d) ph[d] = ph[d + 1];
            ph[PH - 1] = pin;
            // alpha = L p on the row behind the input row
            pm2[0] = pm1[0]; pm1[0] = p0[0]; p0[0] = pin.x;
            pm2[1] = pm1[1]; pm1[1] = p0[1]; p0[1] = pin.y;
            const float l0 = nbr<0, -1>(pm1[0], pm1[1]), r0 = pm1[1];
            const float l1 = pm1[0], r1 = nbr<1, 1>(pm1[0], pm1[1]);
            float al[2], iv[2], ia[2];
            al[0] = 4.0f * pm1[0] - pm2[0] - p0[0] - l0 - r0;
            al[1] = 4.0f * pm1[1] - pm2[1] - p0[1] - l1 - r1;
            iv[0] = s0.x;
            iv[1] = s1.x;
            ia[0] = iv[0] * al[0];
            ia[1] = iv[1] * al[1];
            const float h10 = hsum<RW, 0>(al[0], al[1]), h11 = hsum<RW, 1>(al[0], al[1]);
            const float h20 = hsum<RW, 0>(ia[0], ia[1]), h21 = hsum<RW, 1>(ia[0], ia[1]);
            const float h1[2] = {h10, h11}, h2[2] = {h20, h21};
            const float mu_in[2] = {s0.y, s1.y}, s_in[2] = {s0.z, s1.z};
            float av[2], bv[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
#pragma unroll
                for (int d = 0; d < NB - 1; ++d) {
                    hA[e][d] = hA[e][d + 1];
                    hIA[e][d] = hIA[e][d + 1];
                    ab[e][d] = ab[e][d + 1];
                    ib[e][d] = ib[e][d + 1];
                }
                hA[e][NB - 1] = h1[e];
                hIA[e][NB - 1] = h2[e];
                ab[e][NB - 1] = al[e];
                ib[e][NB - 1] = iv[e];
#pragma unroll
                for (int d = 0; d < RW; ++d) {
                    mub[e][d] = mub[e][d + 1];
                    sb[e][d] = sb[e][d + 1];
                }
                mub[e][RW] = mu_in[e];
                sb[e][RW] = s_in[e];
                float v1 = 0.f, v2 = 0.f;
#pragma unroll
                for (int d = 0; d < NB; ++d) {
                    v1 += hA[e][d];
                    v2 += hIA[e][d];
                }
                const float mu = mub[e][0], sv = sb[e][0];
                const float ma = v1 * inw, mia = v2 * inw;
                av[e] = (mia - mu * ma) * sv;
                bv[e] = ma - av[e] * mu;
            }
            const float g10 = hsum<RW, 0>(av[0], av[1]), g11 = hsum<RW, 1>(av[0], av[1]);
            const float g20 = hsum<RW, 0>(bv[0], bv[1]), g21 = hsum<RW, 1>(bv[0], bv[1]);
            const float g1[2] = {g10, g11}, g2[2] = {g20, g21};
            float mv[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
#pragma unroll
                for (int d = 0; d < NB - 1; ++d) {
                    ha[e][d] = ha[e][d + 1];
                    hb[e][d] = hb[e][d + 1];
                }
                ha[e][NB - 1] = g1[e];
                hb[e][NB - 1] = g2[e];
                float sa = 0.f, sbb = 0.f;
#pragma unroll
                for (int d = 0; d < NB; ++d) {
                    sa += ha[e][d];
                    sbb += hb[e][d];
                }
                // M alpha = |w| alpha - Sa I - Sb on the row of ab[0], ib[0]
                mv[e] = nw * ab[e][0] - sa * ib[e][0] - sbb;
                mm2[e] = mm1[e];
                mm1[e] = m0[e];
                m0[e] = mv[e];
            }
            const float ql0 = nbr<0, -1>(mm1[0], mm1[1]), qr0 = mm1[1];
            const float ql1 = mm1[0], qr1 = nbr<1, 1>(mm1[0], mm1[1]);
            return make_float2(4.0f * mm1[0] - mm2[0] - m0[0] - ql0 - qr0,
                               4.0f * mm1[1] - mm2[1] - m0[1] - ql1 - qr1);
        };

        float2 *outb = reinterpret_cast<float2 *>(a.out + (size_t)b * HW);
        // The walk: 2G rows that fill the chain (unrolled), then TY output
        // rows. Every rolling buffer shifts by one slot a row; in loop blocks
        // of U rows, U a multiple of every buffer's depth, each slot keeps one
        // register across the loop, so no register holding a load in flight
        // is copied (a copy would wait for that load). The TY % U rows left
        // over are unrolled after the loop.
#pragma unroll
        for (int k = 0; k < 2 * G; ++k) (void)advance();
        constexpr int U = llp_lcm(Llp2Rows<RW>::UNR, PFR);
        int yy = 0;
        auto row = [&]() {
            float2 val = advance();
            if (out_lane && y0 + yy < H) {
                val.x *= a.lam;
                val.y *= a.lam;
                outb[(rowD + gx) >> 1] = val;
                // the output row is the input row of G steps ago
                const float2 pv = ph[PH - 1 - G];
                part = fmaf(pv.x, val.x, fmaf(pv.y, val.y, part));
            }
            rowD += W;
            if (rowD == HWi) rowD = 0;
            ++yy;
        };
        for (int blk = 0; blk < TY / U; ++blk) {
#pragma unroll
            for (int u = 0; u < U; ++u) row();
        }
#pragma unroll
        for (int u = 0; u < TY % U; ++u) row();
        if constexpr (RING) cp_async_wait<0>();
    }
    double pd = (double)part;
    for (int o = 16; o > 0; o >>= 1) pd += __shfl_xor_sync(kFull, pd, o);
    if (lane == 0) red[warp] = pd;
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0;
        for (int k = 0; k < kWarps; ++k) tot += red[k];
        llp_cg_finish(a.bands + b, tot, gridDim.y * gridDim.z);  // CTAs of this band
    }
}

// Horizontal 3-sums of a row held as C adjacent columns a lane; the columns
// beyond the lane's come from its neighbours.
template <int C>
__device__ __forceinline__ void hsumc(const float v[C], float h[C]) {
    const float l = __shfl_up_sync(kFull, v[C - 1], 1u);
    const float r = __shfl_down_sync(kFull, v[0], 1u);
    if constexpr (C == 4) {
        const float s01 = v[0] + v[1], s23 = v[2] + v[3];
        h[0] = l + s01;
        h[1] = s01 + v[2];
        h[2] = v[1] + s23;
        h[3] = s23 + r;
    } else {
        const float s01 = v[0] + v[1];
        h[0] = l + s01;
        h[1] = s01 + r;
    }
}

template <int C> struct VecC;
template <> struct VecC<2> {
    using T = float2;
    __device__ static void get(const T &v, float *o) { o[0] = v.x; o[1] = v.y; }
    __device__ static T make(const float *o, float s) { return make_float2(o[0] * s, o[1] * s); }
};
template <> struct VecC<4> {
    using T = float4;
    __device__ static void get(const T &v, float *o) {
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    __device__ static T make(const float *o, float s) {
        return make_float4(o[0] * s, o[1] * s, o[2] * s, o[3] * s);
    }
};

// The same chain for 3 x 3 windows (r = 1) with C = 2 or 4 adjacent columns
// a lane, written for few registers: the vertical 3-sums keep two registers a
// quantity (the newest row and the sum of the two newest), and since the
// periodic L is symmetric, p^T (L M L p) = (L p)^T M (L p): the partial sums
// take alpha . (M alpha) at each output pixel, so p needs no delay buffer.
// A strip is 32 C columns with G / C lanes of halo on each side (56 output
// columns for C = 2, 120 for C = 4), one vector of C values of p a row.
// Requires W % C == 0 (a lane's columns never wrap apart).
template <int C, int TY, int PF>
__global__ void __launch_bounds__(128) llp_cgqc_kernel(LlpArgs a) {
    using V = VecC<C>;
    using VT = typename V::T;
    constexpr int G = 4;
    constexpr int GL = G / C;  // halo lanes
    constexpr int VALID = 32 * C - 2 * G;
    constexpr float nw = 9.0f;
    constexpr float inw = 1.0f / 9.0f;
    __shared__ double red[kWarps];
    const int b = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (a.g->stop || a.bands[b].done) return;
    const int H = a.H, W = a.W;
    const int HWi = H * W;
    const size_t HW = (size_t)HWi;
    const int x0 = blockIdx.y * VALID;
    const int y0 = (blockIdx.z * kWarps + warp) * TY;
    const int xl = x0 - G + C * lane;  // a multiple of C, as is W
    const int gx = wrap2(xl, W);
    const bool out_lane = lane >= GL && lane < 32 - GL && xl < W;
    const float *in = a.in + (size_t)b * HW;
    const float4 *st4 = a.st4;
    float part = 0.0f;

    if (y0 < H) {
        int rowIn = wrap2(y0 - G, H) * W;
        int rowA = wrap2(y0 - G - 1, H) * W;
        int rowD = wrap2(y0, H) * W;
        // with input row i: p of rows i-2, i-1; the vertical 3-sum state of
        // the first windows (alpha, I alpha: newest row i-2 and the sum of
        // rows i-2, i-3), mu and s of row i-2, the second windows' state
        // (a, b), alpha and I of rows i-3, i-2, M alpha of rows i-5, i-4 and
        // alpha of row i-4
        float pA[C], pB[C], h1n[C], h1s[C], h2n[C], h2s[C], mup[C], sp[C];
        float g1n[C], g1s[C], g2n[C], g2s[C], aA[C], aB[C], iA[C], iB[C];
        float mm2[C], mm1[C], ap1[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            pA[c] = pB[c] = h1n[c] = h1s[c] = h2n[c] = h2s[c] = mup[c] = sp[c] = 0.f;
            g1n[c] = g1s[c] = g2n[c] = g2s[c] = aA[c] = aB[c] = iA[c] = iB[c] = 0.f;
            mm2[c] = mm1[c] = ap1[c] = 0.f;
        }
        VT qp[PF];
        float4 qs[PF][C];
        auto load = [&](int k) {
            qp[k] = *reinterpret_cast<const VT *>(in + rowIn + gx);
#pragma unroll
            for (int c = 0; c < C; ++c) qs[k][c] = st4[rowA + gx + c];
            rowIn += W;
            if (rowIn == HWi) rowIn = 0;
            rowA += W;
            if (rowA == HWi) rowA = 0;
        };
#pragma unroll
        for (int k = 0; k < PF; ++k) load(k);

        // one row: consumes input row i (stats row i-1), returns L M alpha of
        // row i-4 and alpha . M alpha of that row in *dot
        auto advance = [&](float *dot) -> VT {
            float pin[C];
            V::get(qp[0], pin);
            float4 sv[C];
#pragma unroll
            for (int c = 0; c < C; ++c) sv[c] = qs[0][c];
#pragma unroll
            for (int k = 0; k < PF - 1; ++k) {
                qp[k] = qp[k + 1];
#pragma unroll
                for (int c = 0; c < C; ++c) qs[k][c] = qs[k + 1][c];
            }
            load(PF - 1);
            // alpha = L p on row i-1
            const float pl = __shfl_up_sync(kFull, pB[C - 1], 1u);
            const float pr = __shfl_down_sync(kFull, pB[0], 1u);
            float al[C], iv[C], ia[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float left = c ? pB[c - 1] : pl;
                const float right = c < C - 1 ? pB[c + 1] : pr;
                al[c] = 4.0f * pB[c] - pA[c] - pin[c] - left - right;
                iv[c] = sv[c].x;
                ia[c] = iv[c] * al[c];
            }
#pragma unroll
            for (int c = 0; c < C; ++c) {  // after every column read its neighbours
                pA[c] = pB[c];
                pB[c] = pin[c];
            }
            float h1[C], h2[C];
            hsumc<C>(al, h1);
            hsumc<C>(ia, h2);
            // first windows, centred on row i-2: a, b of Eq. matting_matrix
            float av[C], bv[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float v1 = h1[c] + h1s[c], v2 = h2[c] + h2s[c];
                h1s[c] = h1[c] + h1n[c];
                h1n[c] = h1[c];
                h2s[c] = h2[c] + h2n[c];
                h2n[c] = h2[c];
                const float ma = v1 * inw, mia = v2 * inw;
                av[c] = (mia - mup[c] * ma) * sp[c];
                bv[c] = ma - av[c] * mup[c];
                mup[c] = sv[c].y;
                sp[c] = sv[c].z;
            }
            float g1[C], g2[C];
            hsumc<C>(av, g1);
            hsumc<C>(bv, g2);
            // second windows, centred on row i-3: M alpha there
            float m0[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float sa = g1[c] + g1s[c], sb = g2[c] + g2s[c];
                g1s[c] = g1[c] + g1n[c];
                g1n[c] = g1[c];
                g2s[c] = g2[c] + g2n[c];
                g2n[c] = g2[c];
                m0[c] = nw * aA[c] - sa * iA[c] - sb;
            }
            // L M alpha on row i-4
            const float ml = __shfl_up_sync(kFull, mm1[C - 1], 1u);
            const float mr = __shfl_down_sync(kFull, mm1[0], 1u);
            float q[C], d = 0.0f;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float left = c ? mm1[c - 1] : ml;
                const float right = c < C - 1 ? mm1[c + 1] : mr;
                q[c] = 4.0f * mm1[c] - mm2[c] - m0[c] - left - right;
                d = fmaf(ap1[c], mm1[c], d);
            }
#pragma unroll
            for (int c = 0; c < C; ++c) {
                mm2[c] = mm1[c];
                mm1[c] = m0[c];
                ap1[c] = aA[c];
                aA[c] = aB[c];
                aB[c] = al[c];
                iA[c] = iB[c];
                iB[c] = iv[c];
            }
            *dot = d;
            return V::make(q, 1.0f);
        };

        // unrolled fill of the chain, then loop blocks of U rows (every
        // rotating buffer has depth 2 or PF) and the unrolled rest
        float dot;
#pragma unroll
        for (int k = 0; k < 2 * G; ++k) (void)advance(&dot);
        constexpr int U = llp_lcm(2, PF);
        VT *outb = reinterpret_cast<VT *>(a.out + (size_t)b * HW);
        int yy = 0;
        auto row = [&]() {
            const VT val = advance(&dot);
            if (out_lane && y0 + yy < H) {
                float o[C];
                V::get(val, o);
                outb[(rowD + gx) / C] = V::make(o, a.lam);
                part += dot;
            }
            rowD += W;
            if (rowD == HWi) rowD = 0;
            ++yy;
        };
        for (int blk = 0; blk < TY / U; ++blk) {
#pragma unroll
            for (int u = 0; u < U; ++u) row();
        }
#pragma unroll
        for (int u = 0; u < TY % U; ++u) row();
    }
    double pd = (double)part * (double)a.lam;
    for (int o = 16; o > 0; o >>= 1) pd += __shfl_xor_sync(kFull, pd, o);
    if (lane == 0) red[warp] = pd;
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0;
        for (int k = 0; k < kWarps; ++k) tot += red[k];
        llp_cg_finish(a.bands + b, tot, gridDim.y * gridDim.z);
    }
}

// The same walk for two bands at once (bands 2z and 2z + 1 of blockIdx.z):
// the PAN statistics and their rolling buffers are loaded and kept once for
// both, and the two bands' chains give each lane twice the independent work.
// A band that has stopped still runs (its outputs and partial sums are not
// used); the CTA leaves only when both have.
template <int RW, int TY, int PF>
__global__ void __launch_bounds__(128) llp_cgq2b_kernel(LlpArgs a) {
    constexpr int G = 2 * RW + 2;
    constexpr int VALID = 64 - 2 * G;
    constexpr int NB = 2 * RW + 1;
    constexpr float nw = (float)(NB * NB);
    constexpr float inw = 1.0f / nw;
    __shared__ double red[2][kWarps];
    const int b0 = 2 * blockIdx.z;
    const bool two = b0 + 1 < a.N;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (a.g->stop || (a.bands[b0].done && (!two || a.bands[b0 + 1].done))) return;
    const int H = a.H, W = a.W;
    const int HWi = H * W;
    const size_t HW = (size_t)HWi;
    const int x0 = blockIdx.x * VALID;
    const int y0 = (blockIdx.y * kWarps + warp) * TY;
    const int xl = x0 - G + 2 * lane;
    const int gx = wrap2(xl, W);
    const bool out_lane = lane >= G / 2 && lane < 32 - G / 2 && xl < W;
    const float *in0 = a.in + (size_t)b0 * HW;
    const float *in1 = two ? in0 + HW : in0;
    const float4 *st4 = a.st4;
    float part[2] = {0.f, 0.f};

    if (y0 < H) {
        int rowIn = wrap2(y0 - G, H) * W;
        int rowA = wrap2(y0 - G - 1, H) * W;
        int rowD = wrap2(y0, H) * W;
        // per band q, pixel e
        float pm2[2][2], pm1[2][2], p0[2][2], mm2[2][2], mm1[2][2], m0[2][2];
        float hA[2][2][NB], hIA[2][2][NB], ab[2][2][NB], ha[2][2][NB], hb[2][2][NB];
        // shared by the bands
        float ib[2][NB], mub[2][RW + 1], sb[2][RW + 1];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
#pragma unroll
            for (int d = 0; d < NB; ++d) ib[e][d] = 0.f;
#pragma unroll
            for (int d = 0; d <= RW; ++d) mub[e][d] = sb[e][d] = 0.f;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                pm2[q][e] = pm1[q][e] = p0[q][e] = mm2[q][e] = mm1[q][e] = m0[q][e] = 0.f;
#pragma unroll
                for (int d = 0; d < NB; ++d)
                    hA[q][e][d] = hIA[q][e][d] = ab[q][e][d] = ha[q][e][d] = hb[q][e][d] = 0.f;
            }
        }
        float2 qp[2][PF];
        float4 qs0[PF], qs1[PF];
        constexpr int PH = ((G + 1 + 2) / 3) * 3;
        float2 ph[2][PH];
#pragma unroll
        for (int d = 0; d < PH; ++d) ph[0][d] = ph[1][d] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            qp[0][k] = *reinterpret_cast<const float2 *>(in0 + rowIn + gx);
            qp[1][k] = *reinterpret_cast<const float2 *>(in1 + rowIn + gx);
            qs0[k] = st4[rowA + gx];
            qs1[k] = st4[rowA + gx + 1];
            rowIn += W;
            if (rowIn == HWi) rowIn = 0;
            rowA += W;
            if (rowA == HWi) rowA = 0;
        }

        auto advance = [&](float2 *res) {
            float2 pin[2];
            pin[0] = qp[0][0];
            pin[1] = qp[1][0];
            const float4 s0 = qs0[0], s1 = qs1[0];
#pragma unroll
            for (int k = 0; k < PF - 1; ++k) {
                qp[0][k] = qp[0][k + 1];
                qp[1][k] = qp[1][k + 1];
                qs0[k] = qs0[k + 1];
                qs1[k] = qs1[k + 1];
            }
            qp[0][PF - 1] = *reinterpret_cast<const float2 *>(in0 + rowIn + gx);
            qp[1][PF - 1] = *reinterpret_cast<const float2 *>(in1 + rowIn + gx);
            qs0[PF - 1] = st4[rowA + gx];
            qs1[PF - 1] = st4[rowA + gx + 1];
            rowIn += W;
            if (rowIn == HWi) rowIn = 0;
            rowA += W;
            if (rowA == HWi) rowA = 0;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
#pragma unroll
                for (int d = 0; d < PH - 1; ++d) ph[q][d] = ph[q][d + 1];
                ph[q][PH - 1] = pin[q];
            }
            const float iv[2] = {s0.x, s1.x};
            const float mu_in[2] = {s0.y, s1.y}, s_in[2] = {s0.z, s1.z};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
#pragma unroll
                for (int d = 0; d < NB - 1; ++d) ib[e][d] = ib[e][d + 1];
                ib[e][NB - 1] = iv[e];
#pragma unroll
                for (int d = 0; d < RW; ++d) {
                    mub[e][d] = mub[e][d + 1];
                    sb[e][d] = sb[e][d + 1];
                }
                mub[e][RW] = mu_in[e];
                sb[e][RW] = s_in[e];
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                // alpha = L p on the row behind the input row
                pm2[q][0] = pm1[q][0]; pm1[q][0] = p0[q][0]; p0[q][0] = pin[q].x;
                pm2[q][1] = pm1[q][1]; pm1[q][1] = p0[q][1]; p0[q][1] = pin[q].y;
                const float l0 = nbr<0, -1>(pm1[q][0], pm1[q][1]), r0 = pm1[q][1];
                const float l1 = pm1[q][0], r1 = nbr<1, 1>(pm1[q][0], pm1[q][1]);
                float al[2], ia[2];
                al[0] = 4.0f * pm1[q][0] - pm2[q][0] - p0[q][0] - l0 - r0;
                al[1] = 4.0f * pm1[q][1] - pm2[q][1] - p0[q][1] - l1 - r1;
                ia[0] = iv[0] * al[0];
                ia[1] = iv[1] * al[1];
                const float h10 = hsum<RW, 0>(al[0], al[1]), h11 = hsum<RW, 1>(al[0], al[1]);
                const float h20 = hsum<RW, 0>(ia[0], ia[1]), h21 = hsum<RW, 1>(ia[0], ia[1]);
                const float h1[2] = {h10, h11}, h2[2] = {h20, h21};
                float av[2], bv[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
#pragma unroll
                    for (int d = 0; d < NB - 1; ++d) {
                        hA[q][e][d] = hA[q][e][d + 1];
                        hIA[q][e][d] = hIA[q][e][d + 1];
                        ab[q][e][d] = ab[q][e][d + 1];
                    }
                    hA[q][e][NB - 1] = h1[e];
                    hIA[q][e][NB - 1] = h2[e];
                    ab[q][e][NB - 1] = al[e];
                    float v1 = 0.f, v2 = 0.f;
#pragma unroll
                    for (int d = 0; d < NB; ++d) {
                        v1 += hA[q][e][d];
                        v2 += hIA[q][e][d];
                    }
                    const float mu = mub[e][0], sv = sb[e][0];
                    const float ma = v1 * inw, mia = v2 * inw;
                    av[e] = (mia - mu * ma) * sv;
                    bv[e] = ma - av[e] * mu;
                }
                const float g10 = hsum<RW, 0>(av[0], av[1]), g11 = hsum<RW, 1>(av[0], av[1]);
                const float g20 = hsum<RW, 0>(bv[0], bv[1]), g21 = hsum<RW, 1>(bv[0], bv[1]);
                const float g1[2] = {g10, g11}, g2[2] = {g20, g21};
#pragma unroll
                for (int e = 0; e < 2; ++e) {
#pragma unroll
                    for (int d = 0; d < NB - 1; ++d) {
                        ha[q][e][d] = ha[q][e][d + 1];
                        hb[q][e][d] = hb[q][e][d + 1];
                    }
                    ha[q][e][NB - 1] = g1[e];
                    hb[q][e][NB - 1] = g2[e];
                    float sa = 0.f, sbb = 0.f;
#pragma unroll
                    for (int d = 0; d < NB; ++d) {
                        sa += ha[q][e][d];
                        sbb += hb[q][e][d];
                    }
                    const float mv = nw * ab[q][e][0] - sa * ib[e][0] - sbb;
                    mm2[q][e] = mm1[q][e];
                    mm1[q][e] = m0[q][e];
                    m0[q][e] = mv;
                }
                const float ql0 = nbr<0, -1>(mm1[q][0], mm1[q][1]), qr0 = mm1[q][1];
                const float ql1 = mm1[q][0], qr1 = nbr<1, 1>(mm1[q][0], mm1[q][1]);
                res[q] = make_float2(4.0f * mm1[q][0] - mm2[q][0] - m0[q][0] - ql0 - qr0,
                                     4.0f * mm1[q][1] - mm2[q][1] - m0[q][1] - ql1 - qr1);
            }
        };

        float2 *out0 = reinterpret_cast<float2 *>(a.out + (size_t)b0 * HW);
        float2 *out1 = reinterpret_cast<float2 *>(a.out + (size_t)(b0 + 1) * HW);
        // the walk as in the one-band kernel: unrolled fill, loop blocks of
        // U rows, unrolled rest
        float2 val[2];
#pragma unroll
        for (int k = 0; k < 2 * G; ++k) advance(val);
        constexpr int U = llp_lcm(Llp2Rows<RW>::UNR, PF);
        int yy = 0;
        auto row = [&]() {
            advance(val);
            if (out_lane && y0 + yy < H) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    if (q == 1 && !two) break;
                    val[q].x *= a.lam;
                    val[q].y *= a.lam;
                    (q ? out1 : out0)[(rowD + gx) >> 1] = val[q];
                    // the output row is the input row of G steps ago
                    const float2 pv = ph[q][PH - 1 - G];
                    part[q] = fmaf(pv.x, val[q].x, fmaf(pv.y, val[q].y, part[q]));
                }
            }
            rowD += W;
            if (rowD == HWi) rowD = 0;
            ++yy;
        };
        for (int blk = 0; blk < TY / U; ++blk) {
#pragma unroll
            for (int u = 0; u < U; ++u) row();
        }
#pragma unroll
        for (int u = 0; u < TY % U; ++u) row();
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        double pd = (double)part[q];
        for (int o = 16; o > 0; o >>= 1) pd += __shfl_xor_sync(kFull, pd, o);
        if (lane == 0) red[q][warp] = pd;
    }
    __syncthreads();
    if (tid >= 2 || (tid == 1 && !two)) return;
    // thread q finishes band b0 + q
    const int q = tid;
    double tot = 0.0;
    for (int k = 0; k < kWarps; ++k) tot += red[q][k];
    CgBand *bd = a.bands + b0 + q;
    atomicAdd(&bd->pAp, tot);
    __threadfence();
    const unsigned int nblk = gridDim.x * gridDim.y;
    const unsigned int t = atomicAdd(&bd->cnt_apply, 1u);
    if (t == nblk - 1) {
        __threadfence();
        // p^T A p = ||D B p||^2 + p^T (lam L^T M L) p
        const double pAp = atomicAdd(&bd->pAp, 0.0) + bd->vv;
        const double rho = bd->rho;
        bd->cnt_apply = 0u;
        if (bd->done) return;
        if (!isfinite(pAp)) {
            bd->status = PS_ERR_NONFINITE;
            bd->done = 1;
            bd->alpha = 0.0;
        } else if (!(pAp > 0.0)) {
            bd->status = PS_ERR_BREAKDOWN;
            bd->done = 1;
            bd->alpha = 0.0;
        } else {
            bd->alpha = rho / pAp;
        }
    }
}

template <int RW, int TY, int PF>
void launch_ty2(const LlpArgs &a, int N, cudaStream_t st) {
    constexpr int G = 2 * RW + 2, VALID = 64 - 2 * G;
    const int rows = TY * kWarps;
    dim3 grd((a.W + VALID - 1) / VALID, (a.H + rows - 1) / rows, (N + 1) / 2);
    llp_cgq2b_kernel<RW, TY, PF><<<grd, 32 * kWarps, 0, st>>>(a);
}

template <int RW, int TY, int PF>
void launch_ty(const LlpArgs &a, int N, cudaStream_t st) {
    constexpr int G = 2 * RW + 2, VALID = 64 - 2 * G;
    const int rows = TY * kWarps;
    dim3 grd(N, (a.W + VALID - 1) / VALID, (a.H + rows - 1) / rows);
    llp_cgq2_kernel<RW, TY, PF><<<grd, 32 * kWarps, 0, st>>>(a);
}

template <int C, int TY, int PF>
void launch_qc(const LlpArgs &a, int N, cudaStream_t st) {
    constexpr int VALID = 32 * C - 8;
    const int rows = TY * kWarps;
    dim3 grd(N, (a.W + VALID - 1) / VALID, (a.H + rows - 1) / rows);
    llp_cgqc_kernel<C, TY, PF><<<grd, 32 * kWarps, 0, st>>>(a);
}

template <int C, int TY>
void launch_qc_pf(const LlpArgs &a, int N, cudaStream_t st) {
    if (a.pf == 4)
        launch_qc<C, TY, 4>(a, N, st);
    else
        launch_qc<C, TY, 2>(a, N, st);
}

template <int RW, int TY>
void launch_pf(const LlpArgs &a, int N, cudaStream_t st) {
    if (a.nbd == 2)
        launch_ty2<RW, TY, 2>(a, N, st);
    else if (a.pf == kRing)
        launch_ty<RW, TY, kRing>(a, N, st);
    else if (a.pf == 3)
        launch_ty<RW, TY, 3>(a, N, st);
    else if (a.pf == 4)
        launch_ty<RW, TY, 4>(a, N, st);
    else
        launch_ty<RW, TY, 2>(a, N, st);
}

template <int RW>
void launch_r(const LlpArgs &a, int N, cudaStream_t st) {
    if (a.ty == Llp2Rows<RW>::SHORT)
        launch_pf<RW, Llp2Rows<RW>::SHORT>(a, N, st);
    else
        launch_pf<RW, Llp2Rows<RW>::LONG>(a, N, st);
}

}  // namespace

int llp_lean_rows(int which) { return which ? kQ4Short : kQ4Long; }

int llp_cgq2_rows(int r, int which) {
    switch (r) {
        case 1: return which ? Llp2Rows<1>::SHORT : Llp2Rows<1>::LONG;
        case 2: return which ? Llp2Rows<2>::SHORT : Llp2Rows<2>::LONG;
        case 3: return which ? Llp2Rows<3>::SHORT : Llp2Rows<3>::LONG;
        default: return which ? Llp2Rows<4>::SHORT : Llp2Rows<4>::LONG;
    }
}

bool llp_lean_supported(int form, int r, int W) {
    return r == 1 && (form == 2 ? W % 2 == 0 : form == 4 && W % 4 == 0);
}

void launch_llp_cgq2(const LlpArgs &a, int r, int N, cudaStream_t st) {
    if (a.nbd != 2 && llp_lean_supported(a.form, r, a.W)) {
        if (a.form == 4) {
            if (a.ty == kQ4Short)
                launch_qc_pf<4, kQ4Short>(a, N, st);
            else
                launch_qc_pf<4, kQ4Long>(a, N, st);
        } else {
            if (a.ty == kQ4Short)
                launch_qc_pf<2, kQ4Short>(a, N, st);
            else
                launch_qc_pf<2, kQ4Long>(a, N, st);
        }
        return;
    }
    switch (r) {
        case 1: launch_r<1>(a, N, st); break;
        case 2: launch_r<2>(a, N, st); break;
        case 3: launch_r<3>(a, N, st); break;
        default: launch_r<4>(a, N, st); break;
    }
}

}  // namespace ps
