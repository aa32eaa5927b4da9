// Preconditioner of the Z0 solve (Eq. Z_ini_matting), sm_103a.
//
// The Z0 system A = B^T D^T D B + lam L^T M L differs from the Z-step
// operator of Eq. Z_solution only in the matting matrix M. With M replaced by
// gamma I the operator
//     P = B^T D^T D B + lam gamma L^T L
// is SPD and, in Fourier space, block diagonal over alias groups of c^2 HR
// frequencies (the same structure the Z step is solved with), so z = P^{-1} r
// is applied exactly: one forward 2-D FFT, one small solve per group, one
// inverse 2-D FFT. This is an extension beyond the paper (which runs plain
// CG): it changes the iterates, not the solution the CG converges to.
//
// Three kernels per application, all FP32 (a preconditioner needs no more:
// its rounding only perturbs the search directions):
//   prec_rows_fwd   TR rows of two bands packed as one complex image (band
//                   2k real, 2k+1 imaginary; P has a real kernel so the two do
//                   not mix), row FFTs in shared memory, stored transposed
//                   ([kx][ky]) in runs of TR values
//   prec_cols<C>    one CTA per LR column index kx0 and image: the C columns
//                   kx0 + q w are exactly the HR columns of the alias groups
//                   (ky0 + p h, kx0 + q w); column FFTs, the group solves and
//                   the inverse column FFTs all stay in shared memory
//   prec_rows_inv   transposed load, inverse row FFTs, unpack to z, and the
//                   per-band r^T z whose last CTA sets beta and the next alpha
//                   numerator (preconditioned CG)
// Sizes whose C columns do not fit one CTA take a fallback: column FFTs and
// the group solve as separate passes over global memory.
#include <math.h>
#include <string.h>

#include <cooperative_groups.h>

#include "common.cuh"
#include "fft_dev.cuh"
#include "kernels.cuh"

namespace ps {

namespace {

constexpr int kPrecPad = 4;  // float2 padding of shared rows (spreads banks)
// Row stride of the row passes, in float2, is a multiple of 16 plus kRowPad.
// Their transposed global accesses move two rows per 16 bytes: a warp covers
// TR / 2 row pairs (rows 2 j, 2 j + 1) times 64 / TR consecutive columns. With
// the stride 4 mod 16, row pair j starts 8 j float2 (mod 16) into the banks,
// so for TR = 8 the four pairs land two on each half of the 16 bank pairs and
// the 256-byte access takes the minimum two wavefronts; TR <= 4 is
// conflict-free for any stride.
constexpr int kRowPad = 4;
constexpr int kPrecMaxSmem = 192 * 1024;
// CTA size of the fused column pass: C columns of H / 16 (or H / PER) threads,
// rounded up to one of three launch shapes, all at 64 registers a thread
constexpr int kPrecColThreads = 1024;
__host__ __device__ constexpr int col_shape(int threads) {
    return threads <= 256 ? 256 : (threads <= 512 ? 512 : 1024);
}
// the 512- and 1024-thread shapes are built for ratios 2 and 4 only
constexpr int col_threads_max(int C) { return (C == 2 || C == 4) ? kPrecColThreads : 256; }

__device__ __forceinline__ bool image_idle(const PrecArgs &a, int k) {
    if (!a.bands) return false;
    if (a.g->stop) return true;
    const bool d0 = a.bands[2 * k].done != 0;
    const bool d1 = (2 * k + 1 >= a.N) || a.bands[2 * k + 1].done != 0;
    return d0 && d1;
}

// Solve ((1/C^2) v v^H + diag(t)) x = s over the alias group (ky0, kx0),
// in place; v_j = conj(B^_j), t_j = lam S^_j^2 with the Laplacian symbol
// S^ = 4 sin^2(pi ky / H) + 4 sin^2(pi kx / W). The algebra is that of the
// Z-step solve: m the member with the smallest t, both sides multiplied by
// t_m (the DC group, t_m = 0, needs no special case), x_m by substitution
// when c^2 t_m < |v_m|^2. `scale` folds in 1/(H W) of the inverse FFT.
template <int C, class At>
__device__ __forceinline__ void group_solve_f(At at, const float2 *__restrict__ bh, int ky0,
                                              int kx0, int H, int W, float lam, float scale) {
    const int h = H / C, w = W / C;
    float sy2[C], sx2[C];
#pragma unroll
    for (int p = 0; p < C; ++p) {
        const float s = sinpif((float)(ky0 + p * h) / (float)H);
        sy2[p] = s * s;
    }
#pragma unroll
    for (int q = 0; q < C; ++q) {
        const float s = sinpif((float)(kx0 + q * w) / (float)W);
        sx2[q] = s * s;
    }
    auto tval = [&](int p, int q) {
        const float S = 4.0f * (sy2[p] + sx2[q]);
        return lam * S * S;
    };
    auto vval = [&](int p, int q) {
        const float2 b = bh[(size_t)(kx0 + q * w) * H + ky0 + p * h];
        return make_float2(b.x, -b.y);
    };
    float tmin = INFINITY;
    int jm = 0;
#pragma unroll(C <= 4 ? C : 1)
    for (int p = 0; p < C; ++p)
#pragma unroll
        for (int q = 0; q < C; ++q) {
            const float tj = tval(p, q);
            if (tj < tmin) {
                tmin = tj;
                jm = p * C + q;
            }
        }
    constexpr float icc = 1.0f / (float)(C * C);
    float2 num = make_float2(0.f, 0.f), vm = make_float2(0.f, 0.f), rm = make_float2(0.f, 0.f);
    float dsum = 0.f;
#pragma unroll(C <= 4 ? C : 1)
    for (int p = 0; p < C; ++p)
#pragma unroll
        for (int q = 0; q < C; ++q) {
            const float2 vj = vval(p, q), rj = at(p, q);
            if (p * C + q == jm) {
                vm = vj;
                rm = rj;
            } else {
                const float it = __frcp_rn(tval(p, q));
                num.x = fmaf(vj.x * rj.x + vj.y * rj.y, it, num.x);
                num.y = fmaf(vj.x * rj.y - vj.y * rj.x, it, num.y);
                dsum = fmaf(vj.x * vj.x + vj.y * vj.y, it, dsum);
            }
        }
    const float vm2 = vm.x * vm.x + vm.y * vm.y;
    const float iden = 1.0f / (tmin + (vm2 + tmin * dsum) * icc);
    const float2 s = make_float2((vm.x * rm.x + vm.y * rm.y + tmin * num.x) * iden,
                                 (vm.x * rm.y - vm.y * rm.x + tmin * num.y) * iden);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll(C <= 4 ? C : 1)
    for (int p = 0; p < C; ++p)
#pragma unroll
        for (int q = 0; q < C; ++q) {
            if (p * C + q == jm) continue;
            const float2 vj = vval(p, q), rj = at(p, q);
            const float it = __frcp_rn(tval(p, q));
            const float2 vs = make_float2(vj.x * s.x - vj.y * s.y, vj.x * s.y + vj.y * s.x);
            const float2 x = make_float2((rj.x - vs.x * icc) * it, (rj.y - vs.y * icc) * it);
            acc.x += vj.x * x.x + vj.y * x.y;
            acc.y += vj.x * x.y - vj.y * x.x;
            at(p, q) = make_float2(x.x * scale, x.y * scale);
        }
    float2 xm;
    if ((float)(C * C) * tmin < vm2) {
        const float2 d = make_float2(s.x - acc.x, s.y - acc.y);
        const float iv = 1.0f / vm2;
        xm = make_float2((d.x * vm.x - d.y * vm.y) * iv, (d.y * vm.x + d.x * vm.y) * iv);
    } else {
        const float2 vs = make_float2(vm.x * s.x - vm.y * s.y, vm.x * s.y + vm.y * s.x);
        xm = make_float2((rm.x - vs.x * icc) / tmin, (rm.y - vs.y * icc) / tmin);
    }
    const int pm = jm / C, qm = jm - (jm / C) * C;
    at(pm, qm) = make_float2(xm.x * scale, xm.y * scale);
}

// Row transform of one row in shared memory: the register FFT on padded rows
// for powers of two (P2), the shared-memory Stockham passes otherwise.
template <bool P2>
__device__ __forceinline__ int ix(int i) {
    return P2 ? prow(i) : i;
}

template <bool P2>
__device__ __forceinline__ void row_fft(float2 *row, int L, const FftPlan &plan,
                                        const float2 *__restrict__ tw, bool inverse, int t,
                                        int nt) {
    if (P2)
        fft_p2_row(row, L, tw, inverse, t, nt);
    else
        fft_row<8, float2>(row, plan, tw, inverse, t, nt);
}

// ---------------------------------------------------------------------------
// Row pass, forward: rows y0 .. y0 + TR - 1 of image k (bands 2k, 2k+1).
// ---------------------------------------------------------------------------
struct RowGeom {
    int TR;   // rows per CTA
    int tpr;  // threads per row
    int ld;   // shared-memory row stride (float2), 4 mod 16: see kRowPad
};

template <bool P2>
__global__ void __launch_bounds__(1024) prec_rows_fwd_kernel(PrecArgs a, RowGeom g) {
    extern __shared__ __align__(16) float2 psm[];
    const int k = blockIdx.y;
    if (image_idle(a, k)) return;
    const int H = a.H, W = a.W, TR = g.TR, ld = g.ld;
    const size_t HW = (size_t)H * W;
    const int y0 = blockIdx.x * TR;
    // a finished band (converged, or stopped on a non-finite value) enters as
    // zeros, so that it cannot disturb the band it shares the image with
    const float *r0 = a.r + (size_t)(2 * k) * HW + (size_t)y0 * W;
    const float *r1 = (2 * k + 1 < a.N) ? r0 + HW : nullptr;
    if (a.bands && a.bands[2 * k].done) r0 = nullptr;
    if (a.bands && r1 && a.bands[2 * k + 1].done) r1 = nullptr;
    // four pixels of both bands per thread and step (W % 4 == 0), four steps
    // in flight
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int n4 = TR * W / 4;
#pragma unroll 4
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        const float4 u = r0 ? __ldg(reinterpret_cast<const float4 *>(r0) + i) : z4;
        const float4 v = r1 ? __ldg(reinterpret_cast<const float4 *>(r1) + i) : z4;
        const int rr = (4 * i) / W, x = 4 * i - rr * W;
        float2 *d = psm + rr * ld;
        d[ix<P2>(x)] = make_float2(u.x, v.x);
        d[ix<P2>(x + 1)] = make_float2(u.y, v.y);
        d[ix<P2>(x + 2)] = make_float2(u.z, v.z);
        d[ix<P2>(x + 3)] = make_float2(u.w, v.w);
    }
    __syncthreads();
    const int row = threadIdx.x / g.tpr, t = threadIdx.x - row * g.tpr;
    if (P2)
        fft_p2_range(psm + row * ld, W, 1, W, a.twW, false, t, g.tpr);
    else
        fft_row<8, float2>(psm + row * ld, a.pw, a.twW, false, t, g.tpr);
    __syncthreads();
    float2 *S = a.spec + (size_t)k * HW;
    if (TR % 2 == 0) {
        // two rows per 16-byte store
        const int hp = TR / 2;
        for (int i = threadIdx.x; i < hp * W; i += blockDim.x) {
            const int r2 = i % hp, kx = i / hp;
            const float2 e0 = psm[(2 * r2) * ld + ix<P2>(kx)];
            const float2 e1 = psm[(2 * r2 + 1) * ld + ix<P2>(kx)];
            *reinterpret_cast<float4 *>(S + (size_t)kx * H + y0 + 2 * r2) =
                make_float4(e0.x, e0.y, e1.x, e1.y);
        }
    } else {
        for (int i = threadIdx.x; i < TR * W; i += blockDim.x) {
            const int rr = i % TR, kx = i / TR;
            S[(size_t)kx * H + y0 + rr] = psm[rr * ld + ix<P2>(kx)];
        }
    }
}

// ---------------------------------------------------------------------------
// Column pass with the group solves: columns kx0 + q w, q < C, of image k.
// ---------------------------------------------------------------------------
template <int C, int PER, bool P2, int MAXT>
__global__ void __launch_bounds__(MAXT, 1024 / MAXT) prec_cols_kernel(PrecArgs a, int tpr, int ld,
                                                                      float scale) {
    extern __shared__ __align__(16) float2 psm[];
    const int k = blockIdx.y, kx0 = blockIdx.x;
    if (image_idle(a, k)) return;
    const int H = a.H, W = a.W, h = H / C, w = W / C;
    float2 *S = a.spec + (size_t)k * H * W;
    // two complex values per 16-byte access (H even), four accesses in flight
#pragma unroll 4
    for (int i = threadIdx.x; i < C * H / 2; i += blockDim.x) {
        const int q = (2 * i) / H, y = 2 * i - q * H;
        const float4 v = *reinterpret_cast<const float4 *>(S + (size_t)(kx0 + q * w) * H + y);
        psm[q * ld + ix<P2>(y)] = make_float2(v.x, v.y);
        psm[q * ld + ix<P2>(y + 1)] = make_float2(v.z, v.w);
    }
    __syncthreads();
    const int row = threadIdx.x / tpr, t = threadIdx.x - row * tpr;
    if (P2)
        fft_p2_row(psm + row * ld, H, a.twH, false, t, tpr);
    else
        fft_row<PER, float2>(psm + row * ld, a.ph, a.twH, false, t, tpr);
    for (int ky0 = threadIdx.x; ky0 < h; ky0 += blockDim.x) {
        auto at = [&](int p, int q) -> float2 & { return psm[q * ld + ix<P2>(ky0 + p * h)]; };
        group_solve_f<C>(at, a.bh, ky0, kx0, H, W, a.lam, scale);
    }
    __syncthreads();
    if (P2)
        fft_p2_row(psm + row * ld, H, a.twH, true, t, tpr);
    else
        fft_row<PER, float2>(psm + row * ld, a.ph, a.twH, true, t, tpr);
    for (int i = threadIdx.x; i < C * H / 2; i += blockDim.x) {
        const int q = (2 * i) / H, y = 2 * i - q * H;
        const float2 e0 = psm[q * ld + ix<P2>(y)], e1 = psm[q * ld + ix<P2>(y + 1)];
        *reinterpret_cast<float4 *>(S + (size_t)(kx0 + q * w) * H + y) =
            make_float4(e0.x, e0.y, e1.x, e1.y);
    }
}

// The same column pass for power-of-two sides whose C columns do not fit one
// CTA (H = 8192 at ratio 4): the C columns of an alias-group set are split
// over a cluster of two CTAs, C / 2 each. Each CTA transforms its own columns
// in its shared memory; the group solves read and write the other CTA's
// columns through distributed shared memory, each CTA taking half of the
// groups; the cluster's barriers order the three phases, so no CTA writes a
// peer's columns before they are transformed or leaves while its own are read.
template <int C>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(1024, 1)
    prec_cols_cluster_kernel(PrecArgs a, int tpr, int ld, float scale) {
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) float2 psm[];
    constexpr int CL = C / 2;  // columns a CTA
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int k = blockIdx.y, kx0 = blockIdx.x >> 1;
    if (image_idle(a, k)) return;  // both CTAs of a cluster see the same image
    const int H = a.H, W = a.W, h = H / C, w = W / C;
    float2 *S = a.spec + (size_t)k * H * W;
#pragma unroll 4
    for (int i = threadIdx.x; i < CL * H / 2; i += blockDim.x) {
        const int ql = (2 * i) / H, y = 2 * i - ql * H;
        const float4 v =
            *reinterpret_cast<const float4 *>(S + (size_t)(kx0 + (rank * CL + ql) * w) * H + y);
        psm[ql * ld + ix<true>(y)] = make_float2(v.x, v.y);
        psm[ql * ld + ix<true>(y + 1)] = make_float2(v.z, v.w);
    }
    __syncthreads();
    const int row = threadIdx.x / tpr, t = threadIdx.x - row * tpr;
    fft_p2_row(psm + row * ld, H, a.twH, false, t, tpr);
    cluster.sync();
    float2 *cols0 = rank == 0 ? psm : cluster.map_shared_rank(psm, 0);
    float2 *cols1 = rank == 1 ? psm : cluster.map_shared_rank(psm, 1);
    const int g0 = rank * (h / 2), g1 = g0 + h / 2;
    for (int ky0 = g0 + threadIdx.x; ky0 < g1; ky0 += blockDim.x) {
        auto at = [&](int p, int q) -> float2 & {
            return (q < CL ? cols0 : cols1)[(q % CL) * ld + ix<true>(ky0 + p * h)];
        };
        group_solve_f<C>(at, a.bh, ky0, kx0, H, W, a.lam, scale);
    }
    cluster.sync();
    fft_p2_row(psm + row * ld, H, a.twH, true, t, tpr);
    for (int i = threadIdx.x; i < CL * H / 2; i += blockDim.x) {
        const int ql = (2 * i) / H, y = 2 * i - ql * H;
        const float2 e0 = psm[ql * ld + ix<true>(y)], e1 = psm[ql * ld + ix<true>(y + 1)];
        *reinterpret_cast<float4 *>(S + (size_t)(kx0 + (rank * CL + ql) * w) * H + y) =
            make_float4(e0.x, e0.y, e1.x, e1.y);
    }
}

// Fallback column passes: FFTs of whole columns (one per CTA) and the group
// solves over global memory.
template <bool P2>
__global__ void __launch_bounds__(1024) prec_col_fft_kernel(PrecArgs a, int inverse) {
    extern __shared__ __align__(16) float2 psm[];
    const int k = blockIdx.y;
    if (image_idle(a, k)) return;
    const int H = a.H;
    float2 *col = a.spec + ((size_t)k * a.W + blockIdx.x) * H;
    for (int i = threadIdx.x; i < H; i += blockDim.x) psm[ix<P2>(i)] = col[i];
    __syncthreads();
    row_fft<P2>(psm, H, a.ph, a.twH, inverse != 0, threadIdx.x, blockDim.x);
    for (int i = threadIdx.x; i < H; i += blockDim.x) col[i] = psm[ix<P2>(i)];
}

template <int C>
__global__ void __launch_bounds__(256) prec_group_kernel(PrecArgs a, float scale) {
    const int k = blockIdx.y;
    if (image_idle(a, k)) return;
    const int H = a.H, W = a.W, h = H / C, w = W / C;
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= h * w) return;
    const int kx0 = gi / h, ky0 = gi - (gi / h) * h;
    float2 *S = a.spec + (size_t)k * H * W;
    auto at = [&](int p, int q) -> float2 & { return S[(size_t)(kx0 + q * w) * H + ky0 + p * h]; };
    group_solve_f<C>(at, a.bh, ky0, kx0, H, W, a.lam, scale);
}

// ---------------------------------------------------------------------------
// Row pass, inverse: transposed load, inverse row FFTs, z and r^T z.
// ---------------------------------------------------------------------------
template <bool P2>
__global__ void __launch_bounds__(1024) prec_rows_inv_kernel(PrecArgs a, RowGeom g) {
    extern __shared__ __align__(16) float2 psm[];
    __shared__ double red[2][32];
    const int k = blockIdx.y;
    if (image_idle(a, k)) return;
    const int H = a.H, W = a.W, TR = g.TR, ld = g.ld;
    const size_t HW = (size_t)H * W;
    const int y0 = blockIdx.x * TR;
    const float2 *S = a.spec + (size_t)k * HW;
    if (TR % 2 == 0) {
        // two rows per 16-byte load, four loads in flight
        const int hp = TR / 2;
#pragma unroll 4
        for (int i = threadIdx.x; i < hp * W; i += blockDim.x) {
            const int r2 = i % hp, kx = i / hp;
            const float4 v =
                *reinterpret_cast<const float4 *>(S + (size_t)kx * H + y0 + 2 * r2);
            psm[(2 * r2) * ld + ix<P2>(kx)] = make_float2(v.x, v.y);
            psm[(2 * r2 + 1) * ld + ix<P2>(kx)] = make_float2(v.z, v.w);
        }
    } else {
        for (int i = threadIdx.x; i < TR * W; i += blockDim.x) {
            const int rr = i % TR, kx = i / TR;
            psm[rr * ld + ix<P2>(kx)] = S[(size_t)kx * H + y0 + rr];
        }
    }
    __syncthreads();
    const int row = threadIdx.x / g.tpr, t = threadIdx.x - row * g.tpr;
    if (P2)
        fft_p2_range(psm + row * ld, W, 1, W, a.twW, true, t, g.tpr);
    else
        fft_row<8, float2>(psm + row * ld, a.pw, a.twW, true, t, g.tpr);
    __syncthreads();
    const size_t o0 = (size_t)(2 * k) * HW + (size_t)y0 * W;
    const bool two = 2 * k + 1 < a.N;
    float d0 = 0.f, d1 = 0.f;
    const int n4 = TR * W / 4;
    float4 *z0 = reinterpret_cast<float4 *>(a.z + o0);
    float4 *z1 = reinterpret_cast<float4 *>(a.z + o0 + HW);
    const float4 *q0 = reinterpret_cast<const float4 *>(a.r + o0);
    const float4 *q1 = reinterpret_cast<const float4 *>(a.r + o0 + HW);
#pragma unroll 2
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        const int rr = (4 * i) / W, x = 4 * i - rr * W;
        const float2 *sr = psm + rr * ld;
        const float2 e0 = sr[ix<P2>(x)], e1 = sr[ix<P2>(x + 1)], e2 = sr[ix<P2>(x + 2)],
                     e3 = sr[ix<P2>(x + 3)];
        z0[i] = make_float4(e0.x, e1.x, e2.x, e3.x);
        if (two) z1[i] = make_float4(e0.y, e1.y, e2.y, e3.y);
        if (a.bands) {
            const float4 u = __ldg(q0 + i);
            d0 = fmaf(u.x, e0.x, fmaf(u.y, e1.x, fmaf(u.z, e2.x, fmaf(u.w, e3.x, d0))));
            if (two) {
                const float4 v = __ldg(q1 + i);
                d1 = fmaf(v.x, e0.y, fmaf(v.y, e1.y, fmaf(v.z, e2.y, fmaf(v.w, e3.y, d1))));
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

int fft_threads_row(int L, int per = 8) {
    int t = (L + per - 1) / per;
    t = (t + 31) & ~31;
    return t < 32 ? 32 : t;
}

bool is_pow2(int L) { return L >= 16 && (L & (L - 1)) == 0; }

int round16(int x) { return (x + 15) & ~15; }

// Launch geometry of the three passes for one size.
struct PrecPlan {
    bool p2;            // H and W powers of two: register FFT on padded rows
    RowGeom rg;         // row passes
    size_t row_smem;
    int col_per;        // fused column pass: values per thread (generic FFT)
    int col_tpr, col_ld;
    size_t col_smem;    // 0: fallback column passes
    bool col_cluster;   // the column pass split over a cluster of two CTAs
    int fb_tpr;         // fallback column FFT
    size_t fb_smem;
};

bool make_prec_plan(int H, int W, int C, PrecPlan *pl) {
    if (C != 2 && C != 3 && C != 4 && C != 6 && C != 8) return false;
    pl->p2 = is_pow2(H) && is_pow2(W);
    // rows: TR rows per CTA, a power of two dividing H, within 1024 threads
    // and the shared-memory budget
    const int tpr = pl->p2 ? W / 16 : fft_threads_row(W);
    if (tpr > 1024) return false;
    const int row_len = pl->p2 ? prow_len(W) : W;
    int TR = 8;
    auto row_bytes = [&](int tr) { return (size_t)tr * (round16(row_len) + kRowPad) * sizeof(float2); };
    while (TR > 1 && (H % TR || TR * tpr > 1024 || row_bytes(TR) > (size_t)kPrecMaxSmem)) TR >>= 1;
    if (row_bytes(TR) > (size_t)kPrecMaxSmem) return false;
    pl->rg.TR = TR;
    pl->rg.tpr = tpr;
    pl->rg.ld = round16(row_len) + kRowPad;
    pl->row_smem = row_bytes(TR);
    // columns: the C columns of one alias-group set in one CTA when they fit,
    // else (power-of-two sides, C even) half of them in each CTA of a pair
    pl->col_smem = 0;
    pl->col_per = 0;
    pl->col_cluster = false;
    if (pl->p2) {
        const int ct = H / 16;
        const size_t bytes = (size_t)C * prow_len(H) * sizeof(float2);
        if (C * ct <= col_threads_max(C) && bytes <= (size_t)kPrecMaxSmem) {
            pl->col_tpr = ct;
            pl->col_ld = prow_len(H);
            pl->col_smem = bytes;
        } else if (C % 2 == 0 && (C / 2) * ct <= 1024 && bytes / 2 <= (size_t)kPrecMaxSmem) {
            pl->col_tpr = ct;
            pl->col_ld = prow_len(H);
            pl->col_smem = bytes / 2;
            pl->col_cluster = true;
        }
        pl->fb_tpr = H / 16;
        pl->fb_smem = (size_t)prow_len(H) * sizeof(float2);
    } else {
        // the fewest values per thread that fit one CTA: 16 and 32 values a
        // thread spill at 64 registers, 8 do not
        const size_t bytes = (size_t)C * (H + kPrecPad) * sizeof(float2);
        for (int per = 8; per <= 32 && bytes <= (size_t)kPrecMaxSmem; per *= 2)
            if (C * fft_threads_row(H, per) <= (per == 32 ? 256 : col_threads_max(C))) {
                pl->col_per = per;
                pl->col_tpr = fft_threads_row(H, per);
                pl->col_ld = H + kPrecPad;
                pl->col_smem = bytes;
                break;
            }
        pl->fb_tpr = fft_threads_row(H);
        pl->fb_smem = (size_t)H * sizeof(float2);
    }
    return pl->fb_tpr <= 1024 && pl->fb_smem <= (size_t)kPrecMaxSmem;
}

template <int C, int MAXT>
void launch_cols_shape(const PrecArgs &a, const PrecPlan &pl, dim3 grd, dim3 blk, float scale,
                       cudaStream_t st) {
    if (pl.p2)
        prec_cols_kernel<C, 16, true, MAXT><<<grd, blk, pl.col_smem, st>>>(a, pl.col_tpr,
                                                                           pl.col_ld, scale);
    else if (pl.col_per == 8)
        prec_cols_kernel<C, 8, false, MAXT><<<grd, blk, pl.col_smem, st>>>(a, pl.col_tpr,
                                                                           pl.col_ld, scale);
    else if (pl.col_per == 16 || MAXT > 256)
        prec_cols_kernel<C, 16, false, MAXT><<<grd, blk, pl.col_smem, st>>>(a, pl.col_tpr,
                                                                            pl.col_ld, scale);
    else
        prec_cols_kernel<C, 32, false, 256><<<grd, blk, pl.col_smem, st>>>(a, pl.col_tpr,
                                                                           pl.col_ld, scale);
}

template <int C>
void launch_cols(const PrecArgs &a, const PrecPlan &pl, float scale, cudaStream_t st) {
    const int w = a.W / C, nimg = (a.N + 1) / 2;
    if constexpr (C % 2 == 0) {
        if (pl.col_cluster) {
            const dim3 grd(2 * w, nimg), blk((C / 2) * pl.col_tpr);
            prec_cols_cluster_kernel<C><<<grd, blk, pl.col_smem, st>>>(a, pl.col_tpr, pl.col_ld,
                                                                     scale);
            return;
        }
    }
    if (pl.col_smem) {
        const dim3 grd(w, nimg), blk(C * pl.col_tpr);
        const int shape = col_shape(C * pl.col_tpr);
        if (shape == 256)
            launch_cols_shape<C, 256>(a, pl, grd, blk, scale, st);
        else
            launch_prec_cols_wide(C, shape, a, pl.p2, pl.col_per, pl.col_tpr, pl.col_ld,
                                  pl.col_smem, scale, st);
    } else {
        const dim3 grd(a.W, nimg);
        const int groups = (a.H / C) * w;
        if (pl.p2) {
            prec_col_fft_kernel<true><<<grd, pl.fb_tpr, pl.fb_smem, st>>>(a, 0);
            prec_group_kernel<C><<<dim3((groups + 255) / 256, nimg), 256, 0, st>>>(a, scale);
            prec_col_fft_kernel<true><<<grd, pl.fb_tpr, pl.fb_smem, st>>>(a, 1);
        } else {
            prec_col_fft_kernel<false><<<grd, pl.fb_tpr, pl.fb_smem, st>>>(a, 0);
            prec_group_kernel<C><<<dim3((groups + 255) / 256, nimg), 256, 0, st>>>(a, scale);
            prec_col_fft_kernel<false><<<grd, pl.fb_tpr, pl.fb_smem, st>>>(a, 1);
        }
    }
}

template <class F>
cudaError_t smem_attr(F *f) {
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kPrecMaxSmem);
}

template <int C, int MAXT>
cudaError_t set_attrs_cs() {
    cudaError_t e = smem_attr(prec_cols_kernel<C, 8, false, MAXT>);
    if (e == cudaSuccess) e = smem_attr(prec_cols_kernel<C, 16, false, MAXT>);
    if (MAXT == 256 && e == cudaSuccess) e = smem_attr(prec_cols_kernel<C, 32, false, 256>);
    if (e == cudaSuccess) e = smem_attr(prec_cols_kernel<C, 16, true, MAXT>);
    return e;
}

template <int C>
cudaError_t set_attrs_c() {
    return set_attrs_cs<C, 256>();
}

// Rows per CTA `tr` for the row passes, if it is a valid choice.
bool prec_rows_valid(const PrecPlan &pl, int H, int W, int tr) {
    if (tr != 1 && tr != 2 && tr != 4 && tr != 8) return false;
    if (H % tr || tr * pl.rg.tpr > 1024) return false;
    const int row_len = pl.p2 ? prow_len(W) : W;
    return (size_t)tr * (round16(row_len) + kRowPad) * sizeof(float2) <= (size_t)kPrecMaxSmem;
}

}  // namespace

#ifdef PS_PREC_WIDE
// The 512- and 1024-thread column shapes (ratios 2 and 4), built in a
// translation unit of their own.
void launch_prec_cols_wide(int C, int shape, const PrecArgs &a, bool p2, int col_per, int col_tpr,
                           int col_ld, size_t col_smem, float scale, cudaStream_t st) {
    PrecPlan pl;
    memset(&pl, 0, sizeof(pl));
    pl.p2 = p2;
    pl.col_per = col_per;
    pl.col_tpr = col_tpr;
    pl.col_ld = col_ld;
    pl.col_smem = col_smem;
    const dim3 grd(a.W / C, (a.N + 1) / 2), blk(C * col_tpr);
    if (C == 4 && shape == 512) launch_cols_shape<4, 512>(a, pl, grd, blk, scale, st);
    if (C == 4 && shape == 1024) launch_cols_shape<4, 1024>(a, pl, grd, blk, scale, st);
    if (C == 2 && shape == 512) launch_cols_shape<2, 512>(a, pl, grd, blk, scale, st);
    if (C == 2 && shape == 1024) launch_cols_shape<2, 1024>(a, pl, grd, blk, scale, st);
}

cudaError_t precond_set_attrs_wide() {
    cudaError_t e = set_attrs_cs<4, 512>();
    if (e == cudaSuccess) e = set_attrs_cs<4, 1024>();
    if (e == cudaSuccess) e = set_attrs_cs<2, 512>();
    if (e == cudaSuccess) e = set_attrs_cs<2, 1024>();
    return e;
}
#else

bool precond_rows_ok(int H, int W, int c, int tr) {
    PrecPlan pl;
    return make_prec_plan(H, W, c, &pl) && prec_rows_valid(pl, H, W, tr);
}

bool precond_supported(int H, int W, int c) {
    PrecPlan pl;
    return make_prec_plan(H, W, c, &pl);
}

// impl 3: the column pass split over two-CTA clusters even where one CTA
// would hold it (power-of-two sides, even ratio); for tests of that path
bool precond_cluster_supported(int H, int W, int c) {
    return is_pow2(H) && is_pow2(W) && c % 2 == 0 && c <= 8 && H % c == 0 && W % c == 0 &&
           (c / 2) * (H / 16) <= 1024 &&
           (size_t)(c / 2) * prow_len(H) * sizeof(float2) <= (size_t)kPrecMaxSmem;
}

void launch_precond(const PrecArgs &a, cudaStream_t st) {
    if (a.impl != 1 && a.impl != 3 && launch_precond_reg(a, st)) return;
    PrecPlan pl;
    if (!make_prec_plan(a.H, a.W, a.c, &pl)) return;  // callers check precond_supported
    if (a.impl == 3 && precond_cluster_supported(a.H, a.W, a.c) && !pl.col_cluster) {
        pl.col_tpr = a.H / 16;
        pl.col_ld = prow_len(a.H);
        pl.col_smem = (size_t)(a.c / 2) * prow_len(a.H) * sizeof(float2);
        pl.col_cluster = true;
    }
    if (a.rows && a.rows != pl.rg.TR && prec_rows_valid(pl, a.H, a.W, a.rows)) {
        const int row_len = pl.p2 ? prow_len(a.W) : a.W;
        pl.rg.TR = a.rows;
        pl.rg.ld = round16(row_len) + kRowPad;
        pl.row_smem = (size_t)a.rows * pl.rg.ld * sizeof(float2);
    }
    const int nimg = (a.N + 1) / 2;
    const float scale = 1.0f / ((float)a.H * (float)a.W);
    const dim3 rgrd(a.H / pl.rg.TR, nimg), rblk(pl.rg.TR * pl.rg.tpr);
    if (pl.p2)
        prec_rows_fwd_kernel<true><<<rgrd, rblk, pl.row_smem, st>>>(a, pl.rg);
    else
        prec_rows_fwd_kernel<false><<<rgrd, rblk, pl.row_smem, st>>>(a, pl.rg);
    switch (a.c) {
        case 2: launch_cols<2>(a, pl, scale, st); break;
        case 3: launch_cols<3>(a, pl, scale, st); break;
        case 4: launch_cols<4>(a, pl, scale, st); break;
        case 6: launch_cols<6>(a, pl, scale, st); break;
        case 8: launch_cols<8>(a, pl, scale, st); break;
        default: break;
    }
    if (pl.p2)
        prec_rows_inv_kernel<true><<<rgrd, rblk, pl.row_smem, st>>>(a, pl.rg);
    else
        prec_rows_inv_kernel<false><<<rgrd, rblk, pl.row_smem, st>>>(a, pl.rg);
}

// B^ in FP32, same [kx][ky] layout as the FP64 spectrum it is rounded from.
__global__ void spectrum_to_f32_kernel(const double2 *__restrict__ in, float2 *__restrict__ out,
                                       size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

void launch_spectrum_to_f32(const double2 *in, float2 *out, size_t n, cudaStream_t st) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    spectrum_to_f32_kernel<<<blocks, 256, 0, st>>>(in, out, n);
}

cudaError_t precond_set_attrs() {
    cudaError_t e = smem_attr(prec_rows_fwd_kernel<true>);
    if (e == cudaSuccess) e = smem_attr(prec_rows_fwd_kernel<false>);
    if (e == cudaSuccess) e = smem_attr(prec_rows_inv_kernel<true>);
    if (e == cudaSuccess) e = smem_attr(prec_rows_inv_kernel<false>);
    if (e == cudaSuccess) e = smem_attr(prec_col_fft_kernel<true>);
    if (e == cudaSuccess) e = smem_attr(prec_col_fft_kernel<false>);
    if (e == cudaSuccess) e = smem_attr(prec_cols_cluster_kernel<2>);
    if (e == cudaSuccess) e = smem_attr(prec_cols_cluster_kernel<4>);
    if (e == cudaSuccess) e = smem_attr(prec_cols_cluster_kernel<6>);
    if (e == cudaSuccess) e = smem_attr(prec_cols_cluster_kernel<8>);
    if (e == cudaSuccess) e = set_attrs_c<2>();
    if (e == cudaSuccess) e = set_attrs_c<3>();
    if (e == cudaSuccess) e = set_attrs_c<4>();
    if (e == cudaSuccess) e = set_attrs_c<6>();
    if (e == cudaSuccess) e = set_attrs_c<8>();
    if (e == cudaSuccess) e = precond_set_attrs_wide();
    if (e == cudaSuccess) e = precond_reg_set_attrs();
    return e;
}
#endif  // PS_PREC_WIDE

}  // namespace ps
