// Register-resident passes of the Z0 preconditioner P^{-1} (and of the FP32
// Z step, which applies the same operator at weight lambda) for the sides
// 256 .. 4096 that are powers of two and 384, 768, 1536 (3 * 2^k), ratios 2
// and 4; other sizes keep the shared-memory passes of precond.cu.
//
// P = B^T D^T D B + lam L^T L is block diagonal over alias groups of c^2
// frequencies (ky0 + p h, kx0 + q w), p, q < c (Eq. Z_solution's structure):
// z = P^{-1} r is a forward 2-D FFT, one rank-one solve per group, an inverse
// 2-D FFT. Three kernels, as before: row FFTs of r (two bands packed as one
// complex image) stored transposed, the column pass (column FFTs, the group
// solves, inverse column FFTs), and the inverse row FFTs with z and r^T z.
//
// Each length-L transform (L = P T) is held by T threads, P values each, in
// registers (P = 16 for powers of two, 24 for 3 * 2^k): three Stockham
// stages (radix 16, 16, L / 256, two for L = 256; or 24, then 4 or 8 twice)
// with two exchanges (one) through shared memory. The first stage reads its inputs,
// positions t + T e (e < 16), straight from global memory, and the last
// leaves its outputs, positions t + T i (i < 16), in registers. In the
// column pass the members ky0 + p h of a group then lie in the registers of
// one thread for every column q (h is a multiple of T when c divides P), and
// the c threads of the c columns sit in adjacent lanes: the group solve runs
// in registers with lane shuffles, and the inverse transform starts from the
// registers it leaves.
#include <math.h>

#include "common.cuh"
#include "fft_dev.cuh"
#include "kernels.cuh"

namespace ps {

namespace {

constexpr int kRegRows = 4;  // rows per CTA of the row passes

// Shared-memory row stride (float2) for a padded row of length L: prow_len
// rounded up to 4 mod 16, so that rows r = 0..3 of a CTA start 8 r banks
// apart and the accesses of a warp (4 rows x 8 consecutive positions) take
// the minimum two wavefronts.
__host__ __device__ constexpr int reg_ld(int L) {
    return ((prow_len(L) + 11) / 16) * 16 + 4;
}

__device__ __forceinline__ float2 cmul2(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // conj(a) b
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// Radix-3 and radix-24 DFTs in registers (y_k = sum_n x_n w^{nk}, w =
// exp(sg 2 pi i / R)), for the lengths 3 * 2^k.
__device__ __forceinline__ void dft3_reg(float2 *x, float sg) {
    constexpr float s3 = 0.86602540378443864676f;  // sin(2 pi / 3)
    const float2 a = x[0], b = x[1], c = x[2];
    const float2 t = make_float2(b.x + c.x, b.y + c.y), d = make_float2(b.x - c.x, b.y - c.y);
    const float2 m = make_float2(a.x - 0.5f * t.x, a.y - 0.5f * t.y);
    x[0] = make_float2(a.x + t.x, a.y + t.y);
    x[1] = make_float2(m.x - sg * s3 * d.y, m.y + sg * s3 * d.x);
    x[2] = make_float2(m.x + sg * s3 * d.y, m.y - sg * s3 * d.x);
}

// cos and sin of 2 pi m / 24 for m in [0, 14] (the products n2 k1 of the
// radix-24 split), as literals so the multiplications fold to constants
__device__ __forceinline__ float2 cs24(int m) {
    constexpr float c1 = 0.96592582628906829f, s1 = 0.25881904510252076f;  // 15 deg
    constexpr float c2 = 0.86602540378443864f, s2 = 0.5f;                 // 30
    constexpr float c3 = 0.70710678118654752f;                              // 45
    switch (m) {
        case 0: return make_float2(1.f, 0.f);
        case 1: return make_float2(c1, s1);
        case 2: return make_float2(c2, s2);
        case 3: return make_float2(c3, c3);
        case 4: return make_float2(s2, c2);
        case 5: return make_float2(s1, c1);
        case 6: return make_float2(0.f, 1.f);
        case 7: return make_float2(-s1, c1);
        case 8: return make_float2(-s2, c2);
        case 9: return make_float2(-c3, c3);
        case 10: return make_float2(-c2, s2);
        case 11: return make_float2(-c1, s1);
        case 12: return make_float2(-1.f, 0.f);
        case 13: return make_float2(-c1, -s1);
        default: return make_float2(-c2, -s2);
    }
}

// 24 = 8 x 3: n = 3 n1 + n2, k = k1 + 8 k2:
//   y_{k1 + 8 k2} = sum_{n2} w_3^{n2 k2} w_24^{n2 k1} [DFT_8 over n1 of x_{3 n1 + n2}]_{k1}
__device__ __forceinline__ void dft24_reg(float2 *x, float sg) {
    float2 a[3][8];
#pragma unroll
    for (int n2 = 0; n2 < 3; ++n2) {
        float2 v[8];
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) v[n1] = x[3 * n1 + n2];
        dft_reg<8>(v, sg);
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) {
            if (n2 * k1 == 0) {
                a[n2][k1] = v[k1];
            } else {
                const float2 cs = cs24(n2 * k1);
                a[n2][k1] = cmul2(v[k1], make_float2(cs.x, sg * cs.y));
            }
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
        float2 v[3] = {a[0][k1], a[1][k1], a[2][k1]};
        dft3_reg(v, sg);
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2) x[k1 + 8 * k2] = v[k2];
    }
}

template <int R>
__device__ __forceinline__ void dftR_reg(float2 *x, float sg) {
    if constexpr (R == 24) dft24_reg(x, sg);
    else dft_reg<R>(x, sg);
}

// Stage plan of a length-L transform held P values a thread (T = L / P
// threads): P = 16 for powers of two, radices 16, 16, L / 256 (two stages
// for L = 256); P = 24 for L = 3 * 2^k, radices 24, R2, R3 with R2 R3 = T,
// R2 and R3 in {4, 8}. Spans NS2 = R1, NS3 = R1 R2.
template <int L, int P>
struct RegPlan {
    static constexpr int T = L / P;
    static constexpr int R1 = P;
    static constexpr int R2 = (P == 16) ? 16 : ((T >= 64) ? 8 : 4);
    static constexpr int R3 = (P == 16) ? ((L >= 512) ? L / 256 : 1) : T / R2;
    static constexpr int NS2 = R1, NS3 = R1 * R2;
    static_assert(R1 * R2 * R3 == L, "stage plan");
};

// w^e for e = 1 .. R-1 from the table tw (tw[m] = exp(-2 pi i m / L)):
// w = tw[k s] and its powers 2, 4, 8 read from the table, the others their
// products (at most three factors), conjugated for the inverse.
template <int R>
__device__ __forceinline__ void twiddle_powers(const float2 *__restrict__ tw, int ks, int L,
                                               bool inverse, float2 (&w)[R]) {
    const float sgn = inverse ? -1.0f : 1.0f;
    auto ld = [&](int m) {
        float2 v = __ldg(tw + (m >= L ? m - L : m));
        v.y *= sgn;
        return v;
    };
    w[0] = make_float2(1.f, 0.f);
    if (R > 1) w[1] = ld(ks);
    if (R > 2) w[2] = ld(2 * ks);
    if (R > 4) w[4] = ld(4 * ks);
    if (R > 8) w[8] = ld(8 * ks);
#pragma unroll
    for (int e = 3; e < R; ++e) {
        if (e == 4 || e == 8) continue;
        const int hi = (e >= 8) ? 8 : ((e >= 4) ? 4 : 2);
        w[e] = cmul2(w[hi], w[e - hi]);
    }
}

// One Stockham stage of radix R and span NS on the P values of this thread:
// butterfly b (j = t + b T, k = j mod NS) holds its R inputs in v[b R + e].
// Twiddles w_{NS R}^{e k}, then the radix-R DFT in registers.
template <int L, int P, int R, int NS>
__device__ __forceinline__ void reg_stage(float2 (&v)[P], int t, const float2 *__restrict__ tw,
                                          bool inverse) {
    constexpr int T = L / P, NB = P / R;
    const float sg = inverse ? 1.0f : -1.0f;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * T, k = (int)((unsigned)j % (unsigned)NS);
        if (NS > 1) {
            float2 w[R];
            twiddle_powers<R>(tw, k * (L / (NS * R)), L, inverse, w);
#pragma unroll
            for (int e = 1; e < R; ++e) v[b * R + e] = cmul2(v[b * R + e], w[e]);
        }
        dftR_reg<R>(&v[b * R], sg);
    }
}

// Outputs of a stage (NS, R) to the shared row: element e of butterfly j to
// position (j - k) R + k + e NS.
template <int L, int P, int R, int NS>
__device__ __forceinline__ void reg_write(float2 *a, const float2 (&v)[P], int t) {
    constexpr int T = L / P, NB = P / R;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * T, k = (int)((unsigned)j % (unsigned)NS), base = (j - k) * R + k;
#pragma unroll
        for (int e = 0; e < R; ++e) a[prow(base + e * NS)] = v[b * R + e];
    }
}

// Inputs of a radix-R stage from the shared row: element e of butterfly j at
// position j + e L / R.
template <int L, int P, int R>
__device__ __forceinline__ void reg_read(const float2 *a, float2 (&v)[P], int t) {
    constexpr int T = L / P, NB = P / R, M = L / R;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * T;
#pragma unroll
        for (int e = 0; e < R; ++e) v[b * R + e] = a[prow(j + e * M)];
    }
}

// The whole transform of one row of length L in place on v: inputs v[e] at
// positions t + T e, outputs v[i] at positions t + T i. `a` is this row's
// shared buffer (prow-padded). Every thread of the CTA must call it; it
// begins with the first stage in registers and ends in registers. With
// `reused`, a barrier precedes its first shared write (the buffer is still
// being read by a previous transform); none follows its last read.
template <int L, int P>
__device__ __forceinline__ void reg_fft(float2 (&v)[P], float2 *a, int t,
                                        const float2 *__restrict__ tw, bool inverse,
                                        bool reused) {
    using Pl = RegPlan<L, P>;
    constexpr int R3 = Pl::R3, NB3 = (R3 > 1) ? P / R3 : 1;
    reg_stage<L, P, Pl::R1, 1>(v, t, tw, inverse);
    if (reused) __syncthreads();
    reg_write<L, P, Pl::R1, 1>(a, v, t);
    __syncthreads();
    reg_read<L, P, Pl::R2>(a, v, t);
    reg_stage<L, P, Pl::R2, Pl::NS2>(v, t, tw, inverse);
    if constexpr (R3 == 1) {
        return;  // the second stage was the last: v[e] at t + T e
    } else {
        __syncthreads();
        reg_write<L, P, Pl::R2, Pl::NS2>(a, v, t);
        __syncthreads();
        reg_read<L, P, R3>(a, v, t);
        reg_stage<L, P, R3, Pl::NS3>(v, t, tw, inverse);
        // butterfly b's output e sits at t + T (b + e NB3): reorder to v[i]
        if (NB3 > 1) {
            float2 o[P];
#pragma unroll
            for (int b = 0; b < NB3; ++b)
#pragma unroll
                for (int e = 0; e < R3; ++e) o[b + e * NB3] = v[b * R3 + e];
#pragma unroll
            for (int i = 0; i < P; ++i) v[i] = o[i];
        }
    }
}

__device__ __forceinline__ bool reg_image_idle(const PrecArgs &a, int k) {
    if (!a.bands) return false;
    if (a.g->stop) return true;
    const bool d0 = a.bands[2 * k].done != 0;
    const bool d1 = (2 * k + 1 >= a.N) || a.bands[2 * k + 1].done != 0;
    return d0 && d1;
}

// Values a thread holds for a transform of length L: 16 for powers of two,
// 24 for 3 * 2^k.
__host__ __device__ constexpr int reg_p(int L) { return (L & (L - 1)) == 0 ? 16 : 24; }
// Minimum CTAs an SM for NT threads: 64 registers a thread for the 16-value
// transforms, about 96 for the 24-value ones.
__host__ __device__ constexpr int reg_minb(int NT, int P) {
    return (P == 16 ? 65536 / 64 : 65536 / 96) / NT > 0 ? (P == 16 ? 65536 / 64 : 65536 / 96) / NT
                                                         : 1;
}

// Lane layout of the row passes: the kRegRows rows of a CTA interleave in
// every warp (row = lane mod kRegRows), so that the transposed spectrum
// accesses of a warp cover whole 32-byte runs of kRegRows rows.
__device__ __forceinline__ void row_lane(int &row, int &t) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    row = lane % kRegRows;
    t = lane / kRegRows + (32 / kRegRows) * warp;
}

// ---------------------------------------------------------------------------
// Forward row pass: rows y0 .. y0 + 3 of bands 2k (real part) and 2k + 1
// (imaginary part), stored transposed: spec[k][kx][y].
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kRegRows * W / reg_p(W),
                                  reg_minb(kRegRows * W / reg_p(W), reg_p(W)))
    prec_rows_fwd_reg_kernel(PrecArgs a) {
    constexpr int P = reg_p(W), T = W / P, LD = reg_ld(W);
    extern __shared__ __align__(16) float2 rsm[];
    const int k = blockIdx.y;
    if (reg_image_idle(a, k)) return;
    int row, t;
    row_lane(row, t);
    const int H = a.H, y = blockIdx.x * kRegRows + row;
    const size_t HW = (size_t)H * W;
    // a finished band enters as zeros, so that it cannot disturb the band it
    // shares the image with
    const float *r0 = a.r + (size_t)(2 * k) * HW + (size_t)y * W;
    const float *r1 = (2 * k + 1 < a.N) ? r0 + HW : nullptr;
    if (a.bands && a.bands[2 * k].done) r0 = nullptr;
    if (a.bands && r1 && a.bands[2 * k + 1].done) r1 = nullptr;
    float2 v[P];
#pragma unroll
    for (int e = 0; e < P; ++e) {
        const int x = t + T * e;
        v[e] = make_float2(r0 ? __ldg(r0 + x) : 0.f, r1 ? __ldg(r1 + x) : 0.f);
    }
    reg_fft<W, P>(v, rsm + row * LD, t, a.twW, false, false);
    float2 *S = a.spec + (size_t)k * HW + y;
#pragma unroll
    for (int i = 0; i < P; ++i) S[(size_t)(t + T * i) * H] = v[i];
}

// ---------------------------------------------------------------------------
// Column pass: columns kx0 + q w (q < C) of image k. Lane q + C u of warp
// w serves column q, t = u + (32 / C) w.
// ---------------------------------------------------------------------------
__constant__ float2 c_cs32[16];  // (cos, sin) of pi i / 16
__constant__ float2 c_cs48[24];  // (cos, sin) of pi i / 24

// The group solve of ((1/C^2) v v^H + diag(t)) x = s for every group whose
// members this thread holds (ky0 = t + T g, p = 0 .. C-1 at ky0 + p h, in
// registers v[g + (16 / C) p]); the C columns are the C adjacent lanes.
// v_j = conj(B^_j), t_j = lam S^_j^2, S^ = 4 sin^2(pi ky / H) + 4 sin^2(pi kx
// / W). With m the member of smallest t (the separable minimum: smallest
// sin^2 in ky, then in kx) the system is solved as the Z step's rank-one
// form, which stays exact for t_m = 0 (the DC group):
//   s = (conj(v_m) r_m + t_m n) / (t_m + (|v_m|^2 + t_m d) / C^2),
//   n = sum_{j != m} conj(v_j) r_j / t_j,  d = sum_{j != m} |v_j|^2 / t_j,
//   x_j = (r_j - v_j s / C^2) / t_j  (j != m),
//   x_m = (s - sum_{j != m} conj(v_j) x_j) / conj(v_m)  if C^2 t_m < |v_m|^2,
//         (r_m - v_m s / C^2) / t_m                     otherwise.
// `scale` folds in 1/(H W) of the inverse transform.
template <int H, int C, int P>
__device__ __forceinline__ void reg_group_solve(float2 (&v)[P], int t, int q, int kx, int W,
                                                const float2 *__restrict__ bcol, float lam,
                                                float scale) {
    constexpr int T = H / P, G = P / C;
    constexpr float icc = 1.0f / (float)(C * C);
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, base = lane - q;
    // sin^2 in x for this column; the column of the group's smallest one
    const float sxv = sinpif((float)kx / (float)W);
    const float sx2 = sxv * sxv;
    float best = sx2;
    int qm = q;
#pragma unroll
    for (int o = 1; o < C; o <<= 1) {
        const float ob = __shfl_xor_sync(full, best, o);
        const int oq = __shfl_xor_sync(full, qm, o);
        if (ob < best || (ob == best && oq < qm)) {
            best = ob;
            qm = oq;
        }
    }
    // sin(pi (t + T i) / H) = sin(pi t / H + pi i / P) by angle addition
    float s0, c0;
    sincospif((float)t / (float)H, &s0, &c0);
#pragma unroll
    for (int g = 0; g < G; ++g) {
        // (indices into the register arrays stay compile-time constants: the
        // member m is selected by comparisons, never by a computed index)
        float tj[C];
        float2 vj[C];
        int pm = 0;
        float smin = 0.f;
#pragma unroll
        for (int p = 0; p < C; ++p) {
            const int i = g + G * p;
            const float2 cs = (P == 16) ? c_cs32[i] : c_cs48[i];
            const float sy = s0 * cs.x + c0 * cs.y;
            const float sy2 = sy * sy;
            if (p == 0 || sy2 < smin) {
                smin = sy2;
                pm = p;
            }
            const float S = 4.0f * (sy2 + sx2);
            tj[p] = lam * S * S;
            const float2 b = __ldg(bcol + t + T * i);
            vj[p] = make_float2(b.x, -b.y);
        }
        const bool mlane = (q == qm);
        // n and d over the members other than m
        float2 num = make_float2(0.f, 0.f);
        float dsum = 0.f;
#pragma unroll
        for (int p = 0; p < C; ++p) {
            if (mlane && p == pm) continue;
            const float it = __frcp_rn(tj[p]);
            const float2 cr = cmulc(vj[p], v[g + G * p]);
            num.x = fmaf(cr.x, it, num.x);
            num.y = fmaf(cr.y, it, num.y);
            dsum = fmaf(vj[p].x * vj[p].x + vj[p].y * vj[p].y, it, dsum);
        }
#pragma unroll
        for (int o = 1; o < C; o <<= 1) {
            num.x += __shfl_xor_sync(full, num.x, o);
            num.y += __shfl_xor_sync(full, num.y, o);
            dsum += __shfl_xor_sync(full, dsum, o);
        }
        float2 sv = make_float2(0.f, 0.f), vm = make_float2(0.f, 0.f), rm = sv;
        float tm = 0.f;
        if (mlane) {
#pragma unroll
            for (int p = 0; p < C; ++p)
                if (p == pm) {
                    vm = vj[p];
                    rm = v[g + G * p];
                    tm = tj[p];
                }
            const float vm2 = vm.x * vm.x + vm.y * vm.y;
            const float iden = 1.0f / (tm + (vm2 + tm * dsum) * icc);
            const float2 cr = cmulc(vm, rm);
            sv = make_float2((cr.x + tm * num.x) * iden, (cr.y + tm * num.y) * iden);
        }
        sv.x = __shfl_sync(full, sv.x, base + qm);
        sv.y = __shfl_sync(full, sv.y, base + qm);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int p = 0; p < C; ++p) {
            if (mlane && p == pm) continue;
            const float it = __frcp_rn(tj[p]);
            const float2 vs = cmul2(vj[p], sv);
            const float2 r = v[g + G * p];
            const float2 x = make_float2((r.x - vs.x * icc) * it, (r.y - vs.y * icc) * it);
            const float2 cx = cmulc(vj[p], x);
            acc.x += cx.x;
            acc.y += cx.y;
            v[g + G * p] = make_float2(x.x * scale, x.y * scale);
        }
#pragma unroll
        for (int o = 1; o < C; o <<= 1) {
            acc.x += __shfl_xor_sync(full, acc.x, o);
            acc.y += __shfl_xor_sync(full, acc.y, o);
        }
        if (mlane) {
            const float vm2 = vm.x * vm.x + vm.y * vm.y;
            float2 xm;
            if ((float)(C * C) * tm < vm2) {
                const float2 d = make_float2(sv.x - acc.x, sv.y - acc.y);
                const float iv = 1.0f / vm2;
                xm = make_float2((d.x * vm.x - d.y * vm.y) * iv, (d.y * vm.x + d.x * vm.y) * iv);
            } else {
                const float2 vs = cmul2(vm, sv);
                xm = make_float2((rm.x - vs.x * icc) / tm, (rm.y - vs.y * icc) / tm);
            }
#pragma unroll
            for (int p = 0; p < C; ++p)
                if (p == pm) v[g + G * p] = make_float2(xm.x * scale, xm.y * scale);
        }
    }
}

template <int H, int C>
__global__ void __launch_bounds__(C * H / reg_p(H), reg_minb(C * H / reg_p(H), reg_p(H)))
    prec_cols_reg_kernel(PrecArgs a, float scale) {
    constexpr int P = reg_p(H), T = H / P, LD = reg_ld(H);
    extern __shared__ __align__(16) float2 csm[];
    const int k = blockIdx.y, kx0 = blockIdx.x;
    if (reg_image_idle(a, k)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane % C, t = lane / C + (32 / C) * warp;
    const int W = a.W, kx = kx0 + q * (W / C);
    float2 *S = a.spec + (size_t)k * H * W + (size_t)kx * H;
    float2 v[P];
#pragma unroll
    for (int e = 0; e < P; ++e) v[e] = S[t + T * e];
    float2 *col = csm + q * LD;
    reg_fft<H, P>(v, col, t, a.twH, false, false);
    reg_group_solve<H, C, P>(v, t, q, kx, W, a.bh + (size_t)kx * H, a.lam, scale);
    reg_fft<H, P>(v, col, t, a.twH, true, true);
#pragma unroll
    for (int i = 0; i < P; ++i) S[t + T * i] = v[i];
}

// ---------------------------------------------------------------------------
// Inverse row pass: transposed load, inverse row FFTs, z = (real, imaginary)
// of the two bands, and their r^T z; the band pair's last CTA sets beta and
// the next alpha numerator (preconditioned CG).
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kRegRows * W / reg_p(W),
                                  reg_minb(kRegRows * W / reg_p(W), reg_p(W)))
    prec_rows_inv_reg_kernel(PrecArgs a) {
    constexpr int P = reg_p(W), T = W / P, LD = reg_ld(W);
    extern __shared__ __align__(16) float2 rsm[];
    __shared__ double red[2][32];
    const int k = blockIdx.y;
    if (reg_image_idle(a, k)) return;
    int row, t;
    row_lane(row, t);
    const int H = a.H, y = blockIdx.x * kRegRows + row;
    const size_t HW = (size_t)H * W;
    const float2 *S = a.spec + (size_t)k * HW + y;
    float2 v[P];
#pragma unroll
    for (int e = 0; e < P; ++e) v[e] = S[(size_t)(t + T * e) * H];
    reg_fft<W, P>(v, rsm + row * LD, t, a.twW, true, false);
    const size_t o0 = (size_t)(2 * k) * HW + (size_t)y * W;
    const bool two = 2 * k + 1 < a.N;
    float *__restrict__ z0 = a.z + o0;
    float *__restrict__ z1 = a.z + o0 + HW;
    const float *__restrict__ q0 = a.r + o0;
    const float *__restrict__ q1 = a.r + o0 + HW;
    float d0 = 0.f, d1 = 0.f;
    // r for r^T z in chunks of 8 positions, all loads of a chunk in flight
    // before its stores
#pragma unroll
    for (int i0 = 0; i0 < P; i0 += 8) {
        float ra[8], rb[8];
        if (a.bands) {
#pragma unroll
            for (int ii = 0; ii < 8; ++ii) {
                const int x = t + T * (i0 + ii);
                ra[ii] = __ldg(q0 + x);
                rb[ii] = two ? __ldg(q1 + x) : 0.f;
            }
        }
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) {
            const int x = t + T * (i0 + ii);
            z0[x] = v[i0 + ii].x;
            if (two) z1[x] = v[i0 + ii].y;
            if (a.bands) {
                d0 = fmaf(ra[ii], v[i0 + ii].x, d0);
                d1 = fmaf(rb[ii], v[i0 + ii].y, d1);
            }
        }
    }
    if (!a.bands) return;
    double s0 = d0, s1 = d1;
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        red[0][warp] = s0;
        red[1][warp] = s1;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double t0 = 0.0, t1 = 0.0;
    for (int j = 0; j < nw; ++j) {
        t0 += red[0][j];
        t1 += red[1][j];
    }
    CgBand *b0 = a.bands + 2 * k;
    CgBand *b1 = two ? b0 + 1 : nullptr;
    atomicAdd(&b0->rz_new, t0);
    if (b1) atomicAdd(&b1->rz_new, t1);
    __threadfence();
    const unsigned int cnt = atomicAdd(&b0->cnt_prec, 1u);
    if (cnt != gridDim.x - 1) return;
    __threadfence();
    b0->cnt_prec = 0u;
    for (int j = 0; j < (two ? 2 : 1); ++j) {
        CgBand *bd = b0 + j;
        const double rz = atomicAdd(&bd->rz_new, 0.0);
        bd->rz_new = 0.0;
        if (bd->done) continue;
        if (!isfinite(rz)) {
            bd->status = PS_ERR_NONFINITE;
            bd->done = 1;
        } else if (!(rz > 0.0)) {
            bd->status = PS_ERR_BREAKDOWN;
            bd->done = 1;
        } else {
            // first application (before any iteration): p = z
            bd->beta = bd->iters > 0 ? rz / bd->rho : 0.0;
            bd->rho = rz;
        }
    }
}

template <int L>
size_t reg_row_smem() {
    return (size_t)kRegRows * reg_ld(L) * sizeof(float2);
}

template <int H, int C>
size_t reg_col_smem() {
    return (size_t)C * reg_ld(H) * sizeof(float2);
}

template <int W>
void launch_rows_reg(const PrecArgs &a, bool inverse, cudaStream_t st) {
    const dim3 grd(a.H / kRegRows, (a.N + 1) / 2), blk(kRegRows * W / reg_p(W));
    if (inverse)
        prec_rows_inv_reg_kernel<W><<<grd, blk, reg_row_smem<W>(), st>>>(a);
    else
        prec_rows_fwd_reg_kernel<W><<<grd, blk, reg_row_smem<W>(), st>>>(a);
}

template <int H, int C>
void launch_cols_reg(const PrecArgs &a, float scale, cudaStream_t st) {
    const dim3 grd(a.W / C, (a.N + 1) / 2), blk(C * H / reg_p(H));
    prec_cols_reg_kernel<H, C><<<grd, blk, reg_col_smem<H, C>(), st>>>(a, scale);
}

bool reg_len_ok(int L) {
    return L == 256 || L == 512 || L == 1024 || L == 2048 || L == 4096 || L == 384 || L == 768 ||
           L == 1536;
}

template <int W>
bool rows_dispatch(const PrecArgs &a, bool inverse, cudaStream_t st) {
    if (a.W != W) return false;
    launch_rows_reg<W>(a, inverse, st);
    return true;
}

template <int H>
bool cols_dispatch(const PrecArgs &a, float scale, cudaStream_t st) {
    if (a.H != H) return false;
    if (a.c == 2) launch_cols_reg<H, 2>(a, scale, st);
    else launch_cols_reg<H, 4>(a, scale, st);
    return true;
}

template <class F>
cudaError_t reg_attr(F *f, size_t bytes) {
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int L>
cudaError_t reg_attrs_len() {
    cudaError_t e = reg_attr(prec_rows_fwd_reg_kernel<L>, reg_row_smem<L>());
    if (e == cudaSuccess) e = reg_attr(prec_rows_inv_reg_kernel<L>, reg_row_smem<L>());
    if (e == cudaSuccess) e = reg_attr(prec_cols_reg_kernel<L, 2>, reg_col_smem<L, 2>());
    if (e == cudaSuccess) e = reg_attr(prec_cols_reg_kernel<L, 4>, reg_col_smem<L, 4>());
    return e;
}

}  // namespace

bool precond_reg_supported(int H, int W, int c) {
    return reg_len_ok(H) && reg_len_ok(W) && (c == 2 || c == 4) && H % kRegRows == 0;
}

bool launch_precond_reg(const PrecArgs &a, cudaStream_t st) {
    if (!precond_reg_supported(a.H, a.W, a.c)) return false;
    const float scale = 1.0f / ((float)a.H * (float)a.W);
    rows_dispatch<256>(a, false, st) || rows_dispatch<512>(a, false, st) ||
        rows_dispatch<1024>(a, false, st) || rows_dispatch<2048>(a, false, st) ||
        rows_dispatch<4096>(a, false, st) || rows_dispatch<384>(a, false, st) ||
        rows_dispatch<768>(a, false, st) || rows_dispatch<1536>(a, false, st);
    cols_dispatch<256>(a, scale, st) || cols_dispatch<512>(a, scale, st) ||
        cols_dispatch<1024>(a, scale, st) || cols_dispatch<2048>(a, scale, st) ||
        cols_dispatch<4096>(a, scale, st) || cols_dispatch<384>(a, scale, st) ||
        cols_dispatch<768>(a, scale, st) || cols_dispatch<1536>(a, scale, st);
    rows_dispatch<256>(a, true, st) || rows_dispatch<512>(a, true, st) ||
        rows_dispatch<1024>(a, true, st) || rows_dispatch<2048>(a, true, st) ||
        rows_dispatch<4096>(a, true, st) || rows_dispatch<384>(a, true, st) ||
        rows_dispatch<768>(a, true, st) || rows_dispatch<1536>(a, true, st);
    return true;
}

cudaError_t precond_reg_set_attrs() {
    float2 cs[16];
    for (int i = 0; i < 16; ++i) {
        const double th = M_PI * i / 16.0;
        cs[i] = make_float2((float)cos(th), (float)sin(th));
    }
    cudaError_t e = cudaMemcpyToSymbol(c_cs32, cs, sizeof(cs));
    float2 cs3[24];
    for (int i = 0; i < 24; ++i) {
        const double th = M_PI * i / 24.0;
        cs3[i] = make_float2((float)cos(th), (float)sin(th));
    }
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_cs48, cs3, sizeof(cs3));
    if (e == cudaSuccess) e = reg_attrs_len<384>();
    if (e == cudaSuccess) e = reg_attrs_len<768>();
    if (e == cudaSuccess) e = reg_attrs_len<1536>();
    if (e == cudaSuccess) e = reg_attrs_len<256>();
    if (e == cudaSuccess) e = reg_attrs_len<512>();
    if (e == cudaSuccess) e = reg_attrs_len<1024>();
    if (e == cudaSuccess) e = reg_attrs_len<2048>();
    if (e == cudaSuccess) e = reg_attrs_len<4096>();
    return e;
}

}  // namespace ps
