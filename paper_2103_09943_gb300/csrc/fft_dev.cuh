// Device building blocks of the shared-memory FFTs (sm_103a): complex helpers,
// radix-2/3/4 butterflies and Stockham autosort passes over rows held in
// shared memory. Used by the Z-step transforms and by the CG preconditioner.
#pragma once

#include "common.cuh"
#include "kernels.cuh"

namespace ps {

template <class T2> struct Cplx;
template <> struct Cplx<float2> {
    using R = float;
    static __device__ __forceinline__ float2 make(float x, float y) { return make_float2(x, y); }
};
template <> struct Cplx<double2> {
    using R = double;
    static __device__ __forceinline__ double2 make(double x, double y) { return make_double2(x, y); }
};

template <class T2>
__device__ __forceinline__ T2 cmulT(T2 a, T2 b) {
    return Cplx<T2>::make(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place radix-R DFT of v with exponent sign `sg` (-1 forward, +1 inverse).
template <int R, class T2>
struct Dft;

template <class T2>
struct Dft<2, T2> {
    static __device__ __forceinline__ void run(T2 *v, typename Cplx<T2>::R) {
        const T2 a = v[0], b = v[1];
        v[0] = Cplx<T2>::make(a.x + b.x, a.y + b.y);
        v[1] = Cplx<T2>::make(a.x - b.x, a.y - b.y);
    }
};

template <class T2>
struct Dft<4, T2> {
    static __device__ __forceinline__ void run(T2 *v, typename Cplx<T2>::R sg) {
        // exp(sg 2 pi i / 4) = (0, sg)
        const T2 a0 = Cplx<T2>::make(v[0].x + v[2].x, v[0].y + v[2].y);
        const T2 a1 = Cplx<T2>::make(v[0].x - v[2].x, v[0].y - v[2].y);
        const T2 b0 = Cplx<T2>::make(v[1].x + v[3].x, v[1].y + v[3].y);
        const T2 b1 = Cplx<T2>::make(v[1].x - v[3].x, v[1].y - v[3].y);
        const T2 jb1 = Cplx<T2>::make(-sg * b1.y, sg * b1.x);
        v[0] = Cplx<T2>::make(a0.x + b0.x, a0.y + b0.y);
        v[2] = Cplx<T2>::make(a0.x - b0.x, a0.y - b0.y);
        v[1] = Cplx<T2>::make(a1.x + jb1.x, a1.y + jb1.y);
        v[3] = Cplx<T2>::make(a1.x - jb1.x, a1.y - jb1.y);
    }
};

template <class T2>
struct Dft<3, T2> {
    static __device__ __forceinline__ void run(T2 *v, typename Cplx<T2>::R sg) {
        // w = exp(sg 2 pi i / 3) = (-1/2, sg sqrt(3)/2); w b + w^2 c = -t/2 + i s3 (b - c)
        using Rl = typename Cplx<T2>::R;
        const Rl s3 = (Rl)0.86602540378443864676 * sg;
        const T2 a = v[0], b = v[1], c = v[2];
        const T2 t = Cplx<T2>::make(b.x + c.x, b.y + c.y);
        const T2 d = Cplx<T2>::make(b.x - c.x, b.y - c.y);
        const T2 m = Cplx<T2>::make(a.x - (Rl)0.5 * t.x, a.y - (Rl)0.5 * t.y);
        v[0] = Cplx<T2>::make(a.x + t.x, a.y + t.y);
        v[1] = Cplx<T2>::make(m.x - s3 * d.y, m.y + s3 * d.x);
        v[2] = Cplx<T2>::make(m.x + s3 * d.y, m.y - s3 * d.x);
    }
};

// One Stockham pass of radix R over a row `a` of L values, in place: every
// thread first reads the inputs of its butterflies into registers, then
// (after a barrier of the whole CTA) writes the outputs, so a single buffer of
// L values suffices. Thread t of the nt threads serving this row takes
// butterflies t, t + nt, ...; PER bounds the values a thread holds, so
// nt >= L / PER is required.
template <int R, int PER, class T2>
__device__ __forceinline__ void stockham_pass(T2 *a, int L, int Ns, const T2 *__restrict__ tw,
                                              bool inverse, int t, int nt) {
    constexpr int MAXB = (PER + R - 1) / R;
    using Rl = typename Cplx<T2>::R;
    const Rl sg = inverse ? (Rl)1 : (Rl)-1;
    const int m = L / R;
    const int stride = L / (Ns * R);
    T2 v[MAXB][R];
#pragma unroll
    for (int bi = 0; bi < MAXB; ++bi) {
        const int j = t + bi * nt;
        if (j < m) {
            const int k = j % Ns;
#pragma unroll
            for (int e = 0; e < R; ++e) {
                T2 x = a[j + e * m];
                if (e > 0 && k > 0) {
                    T2 w = tw[e * k * stride];
                    if (inverse) w.y = -w.y;
                    x = cmulT(x, w);
                }
                v[bi][e] = x;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int bi = 0; bi < MAXB; ++bi) {
        const int j = t + bi * nt;
        if (j < m) {
            const int k = j % Ns;
            Dft<R, T2>::run(v[bi], sg);
            const int idxD = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int e = 0; e < R; ++e) a[idxD + e * Ns] = v[bi][e];
        }
    }
    __syncthreads();
}

// All passes of the plan on one row; every thread of the CTA must call it
// (the passes end on CTA barriers), with rows of equal length.
template <int PER, class T2>
__device__ __forceinline__ void fft_row(T2 *a, const FftPlan &plan, const T2 *__restrict__ tw,
                                        bool inverse, int t, int nt) {
    const int L = plan.L;
    int Ns = 1;
    for (int p = 0; p < plan.npass; ++p) {
        const int R = plan.radix[p];
        if (R == 4)
            stockham_pass<4, PER, T2>(a, L, Ns, tw, inverse, t, nt);
        else if (R == 2)
            stockham_pass<2, PER, T2>(a, L, Ns, tw, inverse, t, nt);
        else
            stockham_pass<3, PER, T2>(a, L, Ns, tw, inverse, t, nt);
        Ns *= R;
    }
}

}  // namespace ps

namespace ps {

// ---------------------------------------------------------------------------
// Register FFT for power-of-two lengths L >= 16: every thread holds 16 values
// per stage and runs radix-16 (or 8/4/2 for the last stage) butterflies in
// registers; stages exchange through shared memory. Rows are stored padded,
// one float2 of padding per 16 values (prow), which keeps the strided stores
// of the early stages free of bank conflicts. T = L / 16 threads per row.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int prow(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int prow_len(int L) { return L + (L >> 4); }

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// y_k = sum_n x_n w^{nk}, w = exp(sg 2 pi i / R), in place; sg = -1 forward.
template <int R>
__device__ __forceinline__ void dft_reg(float2 *x, float sg);

template <>
__device__ __forceinline__ void dft_reg<2>(float2 *x, float) {
    const float2 a = x[0], b = x[1];
    x[0] = make_float2(a.x + b.x, a.y + b.y);
    x[1] = make_float2(a.x - b.x, a.y - b.y);
}

template <>
__device__ __forceinline__ void dft_reg<4>(float2 *x, float sg) {
    const float2 a0 = make_float2(x[0].x + x[2].x, x[0].y + x[2].y);
    const float2 a1 = make_float2(x[0].x - x[2].x, x[0].y - x[2].y);
    const float2 b0 = make_float2(x[1].x + x[3].x, x[1].y + x[3].y);
    const float2 b1 = make_float2(x[1].x - x[3].x, x[1].y - x[3].y);
    // w = exp(sg i pi / 2) = (0, sg): w b1 = (-sg b1.y, sg b1.x)
    const float2 jb = make_float2(-sg * b1.y, sg * b1.x);
    x[0] = make_float2(a0.x + b0.x, a0.y + b0.y);
    x[2] = make_float2(a0.x - b0.x, a0.y - b0.y);
    x[1] = make_float2(a1.x + jb.x, a1.y + jb.y);
    x[3] = make_float2(a1.x - jb.x, a1.y - jb.y);
}

// cos and sin of 2 pi m / 16 (m taken mod 16), as literals so that the
// butterflies' internal twiddles fold to constants.
__device__ __forceinline__ float2 cs16(int m) {
    constexpr float c1 = 0.92387953251128674f, c2 = 0.70710678118654752f,
                    c3 = 0.38268343236508977f;
    switch (m & 15) {
        case 0: return make_float2(1.f, 0.f);
        case 1: return make_float2(c1, c3);
        case 2: return make_float2(c2, c2);
        case 3: return make_float2(c3, c1);
        case 4: return make_float2(0.f, 1.f);
        case 5: return make_float2(-c3, c1);
        case 6: return make_float2(-c2, c2);
        case 7: return make_float2(-c1, c3);
        case 8: return make_float2(-1.f, 0.f);
        case 9: return make_float2(-c1, -c3);
        case 10: return make_float2(-c2, -c2);
        case 11: return make_float2(-c3, -c1);
        case 12: return make_float2(0.f, -1.f);
        case 13: return make_float2(c3, -c1);
        case 14: return make_float2(c2, -c2);
        default: return make_float2(c1, -c3);
    }
}

// R = R1 R2 (R1 = 2 or 4, R2 = 4): n = R2 n1 + n2, k = k1 + R1 k2:
//   y_{k1 + R1 k2} = sum_{n2} w_R^{n2 k1} [DFT_R1 over n1 of x_{R2 n1 + n2}]_{k1} w_R2^{n2 k2}
template <int R1>
__device__ __forceinline__ void dft_split(float2 *x, float sg) {
    constexpr int R2 = 4, R = R1 * R2;
    float2 a[R2][R1];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
        float2 v[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) v[n1] = x[R2 * n1 + n2];
        dft_reg<R1>(v, sg);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            if (n2 * k1 == 0) {
                a[n2][k1] = v[k1];
            } else {
                const float2 cs = cs16(n2 * k1 * (16 / R));
                a[n2][k1] = cmulf(v[k1], make_float2(cs.x, sg * cs.y));
            }
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
        float2 v[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) v[n2] = a[n2][k1];
        dft_reg<R2>(v, sg);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) x[k1 + R1 * k2] = v[k2];
    }
}

template <>
__device__ __forceinline__ void dft_reg<8>(float2 *x, float sg) { dft_split<2>(x, sg); }
template <>
__device__ __forceinline__ void dft_reg<16>(float2 *x, float sg) { dft_split<4>(x, sg); }

// One Stockham stage of radix R on a padded row: butterfly j (k = j mod Ns)
// reads a[j + e L / R], multiplies by w_{Ns R}^{e k} (table tw of length L,
// conjugated for the inverse), transforms, and writes a[(j - k) R + k + e Ns].
// Each of the T threads takes 16 / R butterflies; all inputs are read before
// the barrier and all outputs written after it.
template <int R>
__device__ __forceinline__ void p2_stage(float2 *a, int L, int Ns, const float2 *__restrict__ tw,
                                         float sg, int t, int T) {
    constexpr int NB = 16 / R;
    float2 x[NB][R];
    const int m = L / R, stride = L / (Ns * R);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * T;
        const int k = j & (Ns - 1);
#pragma unroll
        for (int e = 0; e < R; ++e) {
            float2 v = a[prow(j + e * m)];
            if (e > 0 && k > 0) {
                float2 w = __ldg(tw + e * k * stride);
                w.y *= -sg;  // table holds exp(-2 pi i k / L)
                v = cmulf(v, w);
            }
            x[b][e] = v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * T;
        const int k = j & (Ns - 1);
        dft_reg<R>(x[b], sg);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int e = 0; e < R; ++e) a[prow(base + e * Ns)] = x[b][e];
    }
    __syncthreads();
}

// Stages of the register FFT from span Ns0 up to span Ns1 (powers of two,
// Ns0 < Ns1 <= L): the first log(Ns1 / Ns0) stages of a transform that starts
// at Ns0. With Ns0 = 1 and Ns1 = L it is the whole transform.
__device__ __forceinline__ void fft_p2_range(float2 *a, int L, int Ns0, int Ns1,
                                             const float2 *__restrict__ tw, bool inverse, int t,
                                             int T) {
    const float sg = inverse ? 1.0f : -1.0f;
    int Ns = Ns0;
    while (Ns < Ns1) {
        const int rem = Ns1 / Ns;
        if (rem >= 16) {
            p2_stage<16>(a, L, Ns, tw, sg, t, T);
            Ns *= 16;
        } else if (rem == 8) {
            p2_stage<8>(a, L, Ns, tw, sg, t, T);
            Ns *= 8;
        } else if (rem == 4) {
            p2_stage<4>(a, L, Ns, tw, sg, t, T);
            Ns *= 4;
        } else {
            p2_stage<2>(a, L, Ns, tw, sg, t, T);
            Ns *= 2;
        }
    }
}

// Whole transform of one padded row of power-of-two length L (16 <= L),
// natural order in and out. Every thread of the CTA must call it with the
// same L (the stages end on CTA barriers).
__device__ __forceinline__ void fft_p2_row(float2 *a, int L, const float2 *__restrict__ tw,
                                           bool inverse, int t, int T) {
    const float sg = inverse ? 1.0f : -1.0f;
    int Ns = 1;
    while (Ns < L) {
        const int rem = L / Ns;
        if (rem >= 16) {
            p2_stage<16>(a, L, Ns, tw, sg, t, T);
            Ns *= 16;
        } else if (rem == 8) {
            p2_stage<8>(a, L, Ns, tw, sg, t, T);
            Ns *= 8;
        } else if (rem == 4) {
            p2_stage<4>(a, L, Ns, tw, sg, t, T);
            Ns *= 4;
        } else {
            p2_stage<2>(a, L, Ns, tw, sg, t, T);
            Ns *= 2;
        }
    }
}

}  // namespace ps
