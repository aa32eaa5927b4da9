// Image-domain operators of Algorithm 2 and the CG loop kernels (sm_103a).
//
//   pan_stats_kernel  PAN window statistics (Algorithm 2 step 3)
//   db_kernel         D B(u) p on the LR grid, with the CG direction update
//                     p = r + beta p fused into its load
//   adj_kernel        B(u)^T D^T v (right-hand side of Eq. Z_ini_matting)
//   llp_kernel        fused tile kernel: the Z0 operator of Eq. Z_ini_matting
//                     (+ p^T A p), the Z-step right-hand side of
//                     Eq. Z_solution, or the guided filter alone
//   cg_*_kernel       CG vector updates, per-band scalars, loop control
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace ps {

__device__ __forceinline__ int wrapm(int i, int n) {
    int m = i % n;
    return m < 0 ? m + n : m;
}

// ----------------------------------------------------------------------------
// PAN statistics: I = L Y (5-point Laplacian of Eq. reg2), and per
// (2r+1)^2 torus window mu = mean(I), s = 1 / (var(I) + eps), var the
// population variance. The Laplacian and the window sums run in FP64 (the
// E[I^2] - mu^2 difference cancels); outputs are stored in FP32.
// ----------------------------------------------------------------------------
template <int RW>
__global__ void __launch_bounds__(256) pan_stats_kernel(
    const float *__restrict__ Y, int H, int W, float eps, float *__restrict__ I,
    float *__restrict__ mu, float *__restrict__ s, float4 *__restrict__ st4) {
    constexpr int TX = 32, TY = 8;
    constexpr int GY = TY + 2 * RW + 2, GX = TX + 2 * RW + 2;
    constexpr int IY = TY + 2 * RW, IX = TX + 2 * RW;
    __shared__ float sY[GY][GX];
    __shared__ double sI[IY][IX];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.y * TX + threadIdx.x;
    for (int k = tid; k < GY * GX; k += TX * TY) {
        const int yy = k / GX, xx = k - (k / GX) * GX;
        sY[yy][xx] = Y[(size_t)wrapm(y0 - RW - 1 + yy, H) * W + wrapm(x0 - RW - 1 + xx, W)];
    }
    __syncthreads();
    for (int k = tid; k < IY * IX; k += TX * TY) {
        const int yy = k / IX, xx = k - (k / IX) * IX;
        sI[yy][xx] = 4.0 * (double)sY[yy + 1][xx + 1] - (double)sY[yy][xx + 1] -
                     (double)sY[yy + 2][xx + 1] - (double)sY[yy + 1][xx] -
                     (double)sY[yy + 1][xx + 2];
    }
    __syncthreads();
    const int y = y0 + threadIdx.y, x = x0 + threadIdx.x;
    if (y < H && x < W) {
        double s1 = 0.0, s2 = 0.0;
#pragma unroll
        for (int dy = 0; dy <= 2 * RW; ++dy)
#pragma unroll
            for (int dx = 0; dx <= 2 * RW; ++dx) {
                const double v = sI[threadIdx.y + dy][threadIdx.x + dx];
                s1 += v;
                s2 += v * v;
            }
        constexpr double nw = (double)((2 * RW + 1) * (2 * RW + 1));
        const double m = s1 / nw;
        const double var = s2 / nw - m * m;
        const size_t o = (size_t)y * W + x;
        const float iv = (float)sI[threadIdx.y + RW][threadIdx.x + RW];
        const float mv = (float)m, sv = (float)(1.0 / (var + (double)eps));
        if (I) {
            I[o] = iv;
            mu[o] = mv;
            s[o] = sv;
        }
        if (st4) st4[o] = make_float4(iv, mv, sv, 0.0f);
    }
}

// (I, mu, s) -> one float4 per pixel, the layout the LLP kernel reads.
__global__ void pack_stats_kernel(const float *__restrict__ I, const float *__restrict__ mu,
                                  const float *__restrict__ s, size_t n, float4 *__restrict__ st4) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        st4[k] = make_float4(I[k], mu[k], s[k], 0.0f);
}

void launch_pack_stats(const float *I, const float *mu, const float *s, size_t n, float4 *st4,
                       cudaStream_t st) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    pack_stats_kernel<<<blocks, 256, 0, st>>>(I, mu, s, n, st4);
}

void launch_pan_stats(const float *Y, int H, int W, int r, float eps, float *I,
                      float *mu, float *s, float4 *st4, cudaStream_t st) {
    dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8);
    switch (r) {
        case 1: pan_stats_kernel<1><<<grd, blk, 0, st>>>(Y, H, W, eps, I, mu, s, st4); break;
        case 2: pan_stats_kernel<2><<<grd, blk, 0, st>>>(Y, H, W, eps, I, mu, s, st4); break;
        case 3: pan_stats_kernel<3><<<grd, blk, 0, st>>>(Y, H, W, eps, I, mu, s, st4); break;
        default: pan_stats_kernel<4><<<grd, blk, 0, st>>>(Y, H, W, eps, I, mu, s, st4); break;
    }
}

// ----------------------------------------------------------------------------
// v = D B(u) z on the LR grid. One thread per LR site over an 8 x 32 LR tile;
// the HR footprint (c*8 + 2R) x (c*32 + 2R) is staged in shared memory split
// by column phase (column x stored in plane x mod c at x / c), so that the
// 32 sites of a warp, c columns apart on the HR grid, read consecutive words.
// In CG mode the staged value is p_new = r + beta p_old (beta = 0: p_new = r),
// and every CTA also writes p_new for the HR block its LR sites own.
// ----------------------------------------------------------------------------
constexpr int DB_TLX = 32, DB_TLY = 8, DB_TY = 4;   // 128 threads, 2 sites each

__global__ void __launch_bounds__(128) db_kernel(
    const float *__restrict__ src, const float *__restrict__ rsrc,
    float *__restrict__ pdst, CgBand *bands, const CgGlobal *g, int cg,
    int H, int W, int c, const float *__restrict__ u, int R,
    float *__restrict__ v) {
    extern __shared__ float sm[];
    __shared__ float vred[4];
    const int b = blockIdx.z;
    float beta = 0.0f;
    bool use_old = false;
    if (cg) {
        if (g->stop || bands[b].done) return;
        const double bd = bands[b].beta;
        beta = (float)bd;
        use_old = bd != 0.0;
    }
    const int n = 2 * R + 1, nt = n * n;
    const int h = H / c, w = W / c;
    const size_t HW = (size_t)H * W;
    float *su = sm;
    float *sp = sm + ((nt + 3) & ~3);
    const int FY = c * DB_TLY + 2 * R, FX = c * DB_TLX + 2 * R;
    const int FXp = (FX + c - 1) / c, plane = FY * FXp;
    const int ky0 = blockIdx.y * DB_TLY, kx0 = blockIdx.x * DB_TLX;
    const int oy = c * ky0 - R, ox = c * kx0 - R;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * DB_TLX + tx;
    for (int k = tid; k < nt; k += 128) su[k] = u[k];
    const float *S = src + (size_t)b * HW;
    const float *Rr = cg ? rsrc + (size_t)b * HW : nullptr;
    float *P = cg ? pdst + (size_t)b * HW : nullptr;
    // column walk of this thread: xx = tx + 32 m, phase and index within it
    const int step_ph = 32 % c, step_q = 32 / c;
    for (int yy = ty; yy < FY; yy += DB_TY) {
        const size_t grow = (size_t)wrapm(oy + yy, H) * W;
        const bool own_row = cg && yy >= R && yy < R + c * DB_TLY && c * ky0 + (yy - R) < H;
        int ph = tx % c, q = tx / c;
        int gx = wrapm(ox + tx, W);
        for (int xx = tx; xx < FX; xx += 32) {
            const size_t gi = grow + gx;
            float val;
            if (cg) {
                val = use_old ? fmaf(beta, S[gi], Rr[gi]) : Rr[gi];
                if (own_row && xx >= R && xx < R + c * DB_TLX) {
                    const int hx = c * kx0 + (xx - R);
                    if (hx < W) P[(size_t)(c * ky0 + (yy - R)) * W + hx] = val;
                }
            } else {
                val = S[gi];
            }
            sp[ph * plane + yy * FXp + q] = val;
            ph += step_ph;
            q += step_q;
            if (ph >= c) {
                ph -= c;
                ++q;
            }
            gx += 32;
            while (gx >= W) gx -= W;
        }
    }
    __syncthreads();
    // sites (ty, tx) and (ty + 4, tx). Sample (c ky - i, c kx - j): footprint
    // row c ty - i + R, column c tx + t with t = R - j, i.e. plane t mod c,
    // index tx + t / c.
    float acc0 = 0.0f, acc1 = 0.0f;
    const int rstep = c * DB_TY * FXp;
    for (int i = -R; i <= R; ++i) {
        const int row = c * ty - i + R;
        const float *ur = su + (i + R) * n + 2 * R;   // tap j = R - t at ur[-t]
        for (int ph = 0; ph < c; ++ph) {
            const float *b0 = sp + ph * plane + row * FXp + tx;
            const float *b1 = b0 + rstep;
            const float *uu = ur - ph;
            const int cnt = (ph <= 2 * R) ? (2 * R - ph) / c + 1 : 0;
            for (int qq = 0; qq < cnt; ++qq) {
                const float uv = uu[-c * qq];
                acc0 = fmaf(uv, b0[qq], acc0);
                acc1 = fmaf(uv, b1[qq], acc1);
            }
        }
    }
    const int kx = kx0 + tx;
    const int ky_a = ky0 + ty, ky_b = ky0 + ty + DB_TY;
    float vv = 0.0f;
    if (kx < w) {
        if (ky_a < h) {
            v[(size_t)b * h * w + (size_t)ky_a * w + kx] = acc0;
            vv = acc0 * acc0;
        }
        if (ky_b < h) {
            v[(size_t)b * h * w + (size_t)ky_b * w + kx] = acc1;
            vv = fmaf(acc1, acc1, vv);
        }
    }
    if (cg) {
        for (int o = 16; o > 0; o >>= 1) vv += __shfl_xor_sync(0xffffffffu, vv, o);
        if (tx == 0) vred[ty] = vv;
        __syncthreads();
        if (tid == 0)
            atomicAdd(&bands[b].vv, (double)vred[0] + (double)vred[1] + (double)vred[2] +
                                        (double)vred[3]);
    }
}

size_t db_smem_bytes(int c, int R) {
    const int n = 2 * R + 1;
    const int FY = c * DB_TLY + 2 * R, FX = c * DB_TLX + 2 * R;
    const int FXp = (FX + c - 1) / c;
    return sizeof(float) * (((n * n + 3) & ~3) + (size_t)c * FY * FXp);
}

void launch_db(const float *src, const float *rsrc, float *pdst, const CgBand *bands,
               const CgGlobal *g, int cg, int N, int H, int W, int c, const float *u,
               int R, float *v, cudaStream_t st, int impl) {
    if (launch_db_fast(src, rsrc, pdst, const_cast<CgBand *>(bands), g, cg, N, H, W, c, u, R, v,
                       st, impl))
        return;
    const int h = H / c, w = W / c;
    dim3 blk(DB_TLX, DB_TY), grd((w + DB_TLX - 1) / DB_TLX, (h + DB_TLY - 1) / DB_TLY, N);
    db_kernel<<<grd, blk, db_smem_bytes(c, R), st>>>(src, rsrc, pdst, const_cast<CgBand *>(bands),
                                                     g, cg, H, W, c, u, R, v);
}

// ----------------------------------------------------------------------------
// Data term B(u)^T D^T v at HR pixel (y, x): the taps (i, j) with
// (y + i) = 0 and (x + j) = 0 (mod c) pick the LR sample ((y+i)/c, (x+j)/c).
// The taps of a pixel form a grid of step c; the first tap and its LR index
// are found once per axis, the others follow by increments.
// ----------------------------------------------------------------------------
struct AdjAxis {
    int t0;  // first tap + R
    int k0;  // LR index of the first tap
};

__device__ __forceinline__ AdjAxis adj_axis(int y, int Hs, int c, int R) {
    int m = (y - R) % c;
    if (m < 0) m += c;
    const int i0 = -R + (c - m) % c;
    int yy = y + i0;
    if (yy < 0) yy += Hs;
    else if (yy >= Hs) yy -= Hs;
    return {i0 + R, yy / c};
}

__device__ __forceinline__ float adj_sum(const float *__restrict__ vb, int h, int w, int c,
                                         int n, const float *su, AdjAxis ay, AdjAxis ax) {
    float acc = 0.0f;
    int ky = ay.k0;
    for (int ti = ay.t0; ti < n; ti += c) {
        const float *vr = vb + (size_t)ky * w;
        const float *ur = su + ti * n;
        int kx = ax.k0;
        for (int tj = ax.t0; tj < n; tj += c) {
            acc = fmaf(ur[tj], __ldg(vr + kx), acc);
            kx = (kx + 1 == w) ? 0 : kx + 1;
        }
        ky = (ky + 1 == h) ? 0 : ky + 1;
    }
    return acc;
}

// z = B^T D^T v for every band (one thread per HR pixel).
__global__ void __launch_bounds__(256) adj_kernel(const float *__restrict__ v, int H, int W,
                                                  int c, const float *__restrict__ u, int R,
                                                  float *__restrict__ z) {
    __shared__ float su[kMaxTaps];
    const int n = 2 * R + 1;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int k = tid; k < n * n; k += 256) su[k] = u[k];
    __syncthreads();
    const int b = blockIdx.z;
    const int h = H / c, w = W / c;
    const int y = blockIdx.y * 8 + threadIdx.y, x = blockIdx.x * 32 + threadIdx.x;
    if (y >= H || x >= W) return;
    z[(size_t)b * H * W + (size_t)y * W + x] =
        adj_sum(v + (size_t)b * h * w, h, w, c, n, su, adj_axis(y, H, c, R), adj_axis(x, W, c, R));
}

void launch_adj(const float *v, int N, int H, int W, int c, const float *u, int R,
                float *z, cudaStream_t st) {
    dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8, N);
    adj_kernel<<<grd, blk, 0, st>>>(v, H, W, c, u, R, z);
}

// ----------------------------------------------------------------------------
// Fused LLP kernel, register-streaming form.
//
// For the input field alpha (alpha = L p in modes APPLY / ZRHS, alpha = q in
// mode GF) every window j gets the affine fit of Eq. ac_h_compute,
//   a_j = (mean_j(I alpha) - mu_j mean_j(alpha)) s_j,  b_j = mean_j(alpha) - a_j mu_j,
// and with Sa, Sb their sums over the windows containing a pixel:
//   guided filter   GF(alpha) = (Sa I + Sb) / |w|
//   matting matrix  M alpha   = |w| alpha - Sa I - Sb = |w| (alpha - GF(alpha)).
// Modes:
//   APPLY: out = B^T D^T v + lam L M L p            (Eq. Z_ini_matting operator)
//   CGQ:   out = q = lam L M L p, the prior part of A p inside the CG loop, and
//          p^T q accumulated per band (FP64); the band's last CTA computes
//          alpha = r^T r / (||D B p||^2 + p^T q), the data part of p^T A p
//          being ||v||^2 from db_kernel. The data part of A p itself,
//          B^T D^T v, is added in cg_update_kernel.
//   ZRHS:  out = B^T D^T X + lam L GF(L z0)          (Eq. Z_solution rhs),
//          written into the packed complex FFT buffer (band 2k -> real,
//          band 2k+1 -> imaginary part of image k).
//   GF:    out = GF(q).
//
// Each warp owns a strip of 32 columns and walks down LLP_TY output rows plus
// a halo of G rows on each side. Every stage of the chain (Laplacian, row and
// column window sums, affine fit, second window sums, final Laplacian) is
// kept in registers as a short rolling buffer of rows; horizontal neighbours
// come from warp shuffles, so lanes near the strip edges only feed their
// neighbours and the 32 - 2G middle lanes produce outputs.
// ----------------------------------------------------------------------------
constexpr int LLP_WARPS = 4;
constexpr unsigned FULL = 0xffffffffu;

// Output rows per warp: for r = 1 a multiple of 3, so that the 3-deep rolling
// buffers cycle within the 3-way unrolled walk and need no register moves.
template <int RW>
struct LlpRows {
    static constexpr int TY = (RW == 1) ? 66 : 64;
    static constexpr int UNR = (RW == 1) ? 3 : 1;
};

template <int RW, int MODE>
__global__ void __launch_bounds__(128) llp_kernel(LlpArgs a) {
    constexpr int G = (MODE == LLP_GF) ? 2 * RW : 2 * RW + 2;
    constexpr int VALID = 32 - 2 * G;
    constexpr int NB = 2 * RW + 1;
    constexpr int TY = LlpRows<RW>::TY;
    constexpr float nw = (float)(NB * NB);
    constexpr float inw = 1.0f / nw;
    constexpr bool DATA = (MODE == LLP_APPLY || MODE == LLP_ZRHS);
    constexpr bool MATT = (MODE == LLP_APPLY || MODE == LLP_CGQ);
    __shared__ float su[kMaxTaps];
    __shared__ double red[LLP_WARPS];
    const int b = blockIdx.z;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (MODE == LLP_CGQ) {
        if (a.g->stop || a.bands[b].done) return;
    }
    const int H = a.H, W = a.W;
    const int HWi = H * W;
    const size_t HW = (size_t)HWi;
    const int n = 2 * a.R + 1;
    if (DATA) {
        for (int k = tid; k < n * n; k += blockDim.x) su[k] = a.u[k];
        __syncthreads();
    }
    const int x0 = blockIdx.x * VALID;
    const int y0 = (blockIdx.y * LLP_WARPS + warp) * TY;
    const int xl = x0 - G + lane;
    const int gx = wrapm(xl, W);
    const bool out_lane = lane >= G && lane < 32 - G && xl < W;
    const float *in = a.in + (size_t)b * HW;
    const float4 *st4 = a.st4;
    const int c = a.c;
    const int h = H / c, w = W / c;
    float part = 0.0f;

    if (y0 < H) {
        const AdjAxis ax = DATA ? adj_axis(gx, W, c, a.R) : AdjAxis{0, 0};
        const float *lrb = DATA ? a.lr + (size_t)b * h * w : nullptr;
        // row offsets (row * W) of the input row, the alpha row and the output row
        int rowIn = wrapm(y0 - G, H) * W;
        int rowA = ((MODE == LLP_GF) ? wrapm(y0 - G, H) : wrapm(y0 - G - 1, H)) * W;
        int gyD = wrapm(y0, H);
        int rowD = gyD * W;
        float pm2 = 0.f, pm1 = 0.f, p0 = 0.f;
        float hA[NB], hIA[NB], ab[NB], ib[NB], ha[NB], hb[NB], mub[RW + 1], sb[RW + 1];
#pragma unroll
        for (int d = 0; d < NB; ++d) hA[d] = hIA[d] = ab[d] = ib[d] = ha[d] = hb[d] = 0.f;
#pragma unroll
        for (int d = 0; d <= RW; ++d) mub[d] = sb[d] = 0.f;
        float mm2 = 0.f, mm1 = 0.f, m0 = 0.f;
        // Loads run PF rows ahead of their use (a small register queue), so
        // that each warp keeps several rows of global loads in flight.
        constexpr int PF = 3;
        float qp[PF];
        float4 qs[PF];
        // history of the input, to multiply the output row by its p (CG mode)
        constexpr int PH = ((G + 1 + 2) / 3) * 3;
        float ph[PH];
#pragma unroll
        for (int d = 0; d < PH; ++d) ph[d] = 0.f;
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            qp[k] = in[rowIn + gx];
            qs[k] = st4[rowA + gx];
            rowIn += W;
            if (rowIn == HWi) rowIn = 0;
            rowA += W;
            if (rowA == HWi) rowA = 0;
        }

        // one row of the chain; returns the chain output for the row G behind
        // the input row (valid once the buffers are full)
        auto advance = [&]() -> float {
            const float pin = qp[0];
            const float4 stv = qs[0];
#pragma unroll
            for (int k = 0; k < PF - 1; ++k) {
                qp[k] = qp[k + 1];
                qs[k] = qs[k + 1];
            }
            qp[PF - 1] = in[rowIn + gx];
            qs[PF - 1] = st4[rowA + gx];
            rowIn += W;
            if (rowIn == HWi) rowIn = 0;
            rowA += W;
            if (rowA == HWi) rowA = 0;
#pragma unroll
            for (int d = 0; d < PH - 1; ++d) ph[d] = ph[d + 1];
            ph[PH - 1] = pin;
            float al;
            if (MODE == LLP_GF) {
                al = pin;
            } else {
                pm2 = pm1;
                pm1 = p0;
                p0 = pin;
                al = 4.0f * pm1 - pm2 - p0 - __shfl_up_sync(FULL, pm1, 1) -
                     __shfl_down_sync(FULL, pm1, 1);
            }
            const float iv = stv.x;
            const float ia = iv * al;
            float h1 = al, h2 = ia;
#pragma unroll
            for (int d = 1; d <= RW; ++d) {
                h1 += __shfl_up_sync(FULL, al, d) + __shfl_down_sync(FULL, al, d);
                h2 += __shfl_up_sync(FULL, ia, d) + __shfl_down_sync(FULL, ia, d);
            }
#pragma unroll
            for (int d = 0; d < NB - 1; ++d) {
                hA[d] = hA[d + 1];
                hIA[d] = hIA[d + 1];
                ab[d] = ab[d + 1];
                ib[d] = ib[d + 1];
            }
            hA[NB - 1] = h1;
            hIA[NB - 1] = h2;
            ab[NB - 1] = al;
            ib[NB - 1] = iv;
#pragma unroll
            for (int d = 0; d < RW; ++d) {
                mub[d] = mub[d + 1];
                sb[d] = sb[d + 1];
            }
            mub[RW] = stv.y;
            sb[RW] = stv.z;
            float s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int d = 0; d < NB; ++d) {
                s1 += hA[d];
                s2 += hIA[d];
            }
            const float mu = mub[0], sv = sb[0];
            const float ma = s1 * inw, mia = s2 * inw;
            const float av = (mia - mu * ma) * sv;
            const float bv = ma - av * mu;
            float g1 = av, g2 = bv;
#pragma unroll
            for (int d = 1; d <= RW; ++d) {
                g1 += __shfl_up_sync(FULL, av, d) + __shfl_down_sync(FULL, av, d);
                g2 += __shfl_up_sync(FULL, bv, d) + __shfl_down_sync(FULL, bv, d);
            }
#pragma unroll
            for (int d = 0; d < NB - 1; ++d) {
                ha[d] = ha[d + 1];
                hb[d] = hb[d + 1];
            }
            ha[NB - 1] = g1;
            hb[NB - 1] = g2;
            float sa = 0.f, sbb = 0.f;
#pragma unroll
            for (int d = 0; d < NB; ++d) {
                sa += ha[d];
                sbb += hb[d];
            }
            // alpha and I of the row whose window sums are complete: ab[0], ib[0]
            if (MODE == LLP_GF) return (sa * ib[0] + sbb) * inw;
            const float mv = MATT ? nw * ab[0] - sa * ib[0] - sbb : (sa * ib[0] + sbb) * inw;
            mm2 = mm1;
            mm1 = m0;
            m0 = mv;
            return 4.0f * mm1 - mm2 - m0 - __shfl_up_sync(FULL, mm1, 1) -
                   __shfl_down_sync(FULL, mm1, 1);
        };

        for (int step = 0; step < 2 * G; ++step) (void)advance();
#pragma unroll LlpRows<RW>::UNR
        for (int yy = 0; yy < TY; ++yy) {
            float val = advance();
            if (out_lane && y0 + yy < H) {
                const int o = rowD + gx;
                if (DATA) {
                    const float dat = adj_sum(lrb, h, w, c, n, su, adj_axis(gyD, H, c, a.R), ax);
                    val = fmaf(a.lam, val, dat);
                } else if (MODE == LLP_CGQ) {
                    val *= a.lam;
                }
                if (MODE == LLP_ZRHS && a.cout) {
                    double2 *cimg = a.cout + (size_t)(b >> 1) * HW + o;
                    if (b & 1)
                        reinterpret_cast<double *>(cimg)[1] = (double)val;
                    else if (b == a.N - 1)
                        *cimg = make_double2((double)val, 0.0);
                    else
                        reinterpret_cast<double *>(cimg)[0] = (double)val;
                } else {
                    a.out[(size_t)b * HW + o] = val;
                }
                // the output row is the input row of G steps ago
                if (MODE == LLP_CGQ) part = fmaf(ph[PH - 1 - G], val, part);
            }
            rowD += W;
            if (rowD == HWi) rowD = 0;
            if (DATA) gyD = (gyD + 1 == H) ? 0 : gyD + 1;
        }
    }
    if (MODE == LLP_CGQ) {
        double pd = (double)part;
        for (int o = 16; o > 0; o >>= 1) pd += __shfl_xor_sync(FULL, pd, o);
        if (lane == 0) red[warp] = pd;
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            for (int k = 0; k < LLP_WARPS; ++k) tot += red[k];
            CgBand *bd = a.bands + b;
            atomicAdd(&bd->pAp, tot);
            __threadfence();
            const unsigned int nblk = gridDim.x * gridDim.y;
            const unsigned int t = atomicAdd(&bd->cnt_apply, 1u);
            if (t == nblk - 1) {
                __threadfence();
                // p^T A p = ||D B p||^2 + p^T (lam L^T M L) p
                const double pAp = atomicAdd(&bd->pAp, 0.0) + bd->vv;
                const double rr = bd->rho;
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
                    bd->alpha = rr / pAp;  // rho / p^T A p
                }
            }
        }
    }
}

size_t llp_smem_bytes(int) { return 0; }

template <int RW>
static void launch_llp_r(const LlpArgs &a, int mode, int N, cudaStream_t st) {
    const int G = (mode == LLP_GF) ? 2 * RW : 2 * RW + 2;
    const int valid = 32 - 2 * G;
    const int rows = LlpRows<RW>::TY * LLP_WARPS;
    dim3 grd((a.W + valid - 1) / valid, (a.H + rows - 1) / rows, N);
    switch (mode) {
        case LLP_APPLY: llp_kernel<RW, LLP_APPLY><<<grd, 32 * LLP_WARPS, 0, st>>>(a); break;
        case LLP_ZRHS: llp_kernel<RW, LLP_ZRHS><<<grd, 32 * LLP_WARPS, 0, st>>>(a); break;
        case LLP_CGQ: llp_kernel<RW, LLP_CGQ><<<grd, 32 * LLP_WARPS, 0, st>>>(a); break;
        default: llp_kernel<RW, LLP_GF><<<grd, 32 * LLP_WARPS, 0, st>>>(a); break;
    }
}

cudaError_t operators_set_attrs() {
    cudaError_t e = cudaFuncSetAttribute(db_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)db_smem_bytes(8, kMaxR));
    if (e != cudaSuccess) return e;
    return cg_fast_set_attrs();
}

void launch_llp(const LlpArgs &a, int mode, int r, int N, cudaStream_t st) {
    switch (r) {
        case 1: launch_llp_r<1>(a, mode, N, st); break;
        case 2: launch_llp_r<2>(a, mode, N, st); break;
        case 3: launch_llp_r<3>(a, mode, N, st); break;
        default: launch_llp_r<4>(a, mode, N, st); break;
    }
}

// ----------------------------------------------------------------------------
// CG bookkeeping. Every per-band decision is taken by the last CTA of that
// band to arrive (atomic counter, no waiting); the loop condition is taken by
// a one-warp control kernel that always runs, so the device loop ends after
// at most max_iter iterations whatever the band states.
// ----------------------------------------------------------------------------
__global__ void cg_reset_kernel(CgBand *bands, CgGlobal *g, int N, double tol, int max_iter,
                                int precond, int rule) {
    const int t = threadIdx.x;
    const unsigned long long now = global_ns();
    for (int b = t; b < N; b += blockDim.x) {
        CgBand z = {};
        z.t_start = now;
        bands[b] = z;
    }
    // every loop-control record of the solve (one per branch loop), alike
    if (t < kMaxSplit) {
        CgGlobal *gk = g + t;
        gk->cnt_bands = 0u;
        gk->active = N;
        gk->max_iters = 0;
        gk->stop = 0;
        gk->iter = 0;
        gk->max_iter = max_iter;
        gk->tol = tol;
        gk->precond = precond;
        gk->rule = rule;
    }
}

// r = b - (Ax0 if warm) ; x = x0 or 0; r^T r and b^T b per band.
__global__ void __launch_bounds__(256) cg_init_kernel(const float4 *__restrict__ bvec,
                                                      const float4 *__restrict__ ax0,
                                                      const float4 *__restrict__ x0,
                                                      float4 *__restrict__ x,
                                                      float4 *__restrict__ r, size_t n4,
                                                      CgBand *bands, CgGlobal *g) {
    __shared__ double red[8];
    const int b = blockIdx.y;
    const size_t off = (size_t)b * n4;
    double rr = 0.0, bb = 0.0;
    for (size_t i = blockIdx.x * 256 + threadIdx.x; i < n4; i += (size_t)gridDim.x * 256) {
        const float4 bv = bvec[off + i];
        float4 rv = bv;
        if (ax0) {
            const float4 a = ax0[off + i];
            rv.x -= a.x; rv.y -= a.y; rv.z -= a.z; rv.w -= a.w;
            x[off + i] = x0[off + i];
        } else {
            x[off + i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        r[off + i] = rv;
        rr += (double)(rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w);
        bb += (double)(bv.x * bv.x + bv.y * bv.y + bv.z * bv.z + bv.w * bv.w);
    }
    const double trr = block_sum_d(rr, red);
    const double tbb = block_sum_d(bb, red);
    if (threadIdx.x == 0) {
        CgBand *bd = bands + b;
        atomicAdd(&bd->rr_new, trr);
        atomicAdd(&bd->pAp, tbb);
        __threadfence();
        const unsigned int t = atomicAdd(&bd->cnt_init, 1u);
        if (t == gridDim.x - 1) {
            __threadfence();
            const double r2 = atomicAdd(&bd->rr_new, 0.0);
            const double b2 = atomicAdd(&bd->pAp, 0.0);
            bd->rr = r2;
            bd->rho = r2;  // replaced by r^T z when a preconditioner follows
            bd->bb = b2;
            bd->rr_new = 0.0;
            bd->pAp = 0.0;
            bd->vv = 0.0;
            bd->beta = 0.0;
            bd->alpha = 0.0;
            bd->iters = 0;
            bd->cnt_init = 0u;
            if (!isfinite(r2) || !isfinite(b2)) {
                bd->status = PS_ERR_NONFINITE;
                bd->done = 1;
            } else if (b2 == 0.0 || r2 == 0.0 || (g->rule == 0 && sqrt(r2 / b2) <= g->tol)) {
                // the relative-change rule needs a step: only an exact start ends here
                bd->done = 1;
            }
        }
    }
}

// x += alpha p; r -= alpha (B^T D^T v + q); the next r^T r. The data part of
// A p is formed here from the LR samples v = D B p (held in L2) rather than in
// the stencil kernel, where it would cost issue slots that this kernel, bound
// by HBM, has to spare. One CTA covers 128 float4 of one row; the band's last
// CTA takes beta, the convergence test and the iteration cap.
__global__ void __launch_bounds__(128) cg_update_kernel(float4 *__restrict__ x,
                                                        float4 *__restrict__ r,
                                                        const float4 *__restrict__ p,
                                                        const float4 *__restrict__ q,
                                                        const float *__restrict__ v,
                                                        const float *__restrict__ u, int R,
                                                        int c, int H, int W, CgBand *bands,
                                                        const CgGlobal *g) {
    __shared__ float su[kMaxTaps];
    __shared__ double red[3][4];
    const int b = blockIdx.z, y = blockIdx.y;
    if (g->stop || bands[b].done) return;
    const int n = 2 * R + 1;
    for (int k = threadIdx.x; k < n * n; k += 128) su[k] = u[k];
    __syncthreads();
    const float al = (float)bands[b].alpha;
    const int W4 = W >> 2, h = H / c, w = W / c;
    const int x4 = blockIdx.x * 128 + threadIdx.x;
    float rrf = 0.0f, xxf = 0.0f, ppf = 0.0f;
    if (x4 < W4) {
        const size_t o = ((size_t)b * H + y) * W4 + x4;
        const AdjAxis ay = adj_axis(y, H, c, R);
        const float *vb = v + (size_t)b * h * w;
        const int x0 = 4 * x4;
        const float d0 = adj_sum(vb, h, w, c, n, su, ay, adj_axis(x0, W, c, R));
        const float d1 = adj_sum(vb, h, w, c, n, su, ay, adj_axis(x0 + 1, W, c, R));
        const float d2 = adj_sum(vb, h, w, c, n, su, ay, adj_axis(x0 + 2, W, c, R));
        const float d3 = adj_sum(vb, h, w, c, n, su, ay, adj_axis(x0 + 3, W, c, R));
        float4 xv = x[o], rv = r[o];
        const float4 pv = p[o], qv = q[o];
        xv.x = fmaf(al, pv.x, xv.x); xv.y = fmaf(al, pv.y, xv.y);
        xv.z = fmaf(al, pv.z, xv.z); xv.w = fmaf(al, pv.w, xv.w);
        rv.x = fmaf(-al, d0 + qv.x, rv.x); rv.y = fmaf(-al, d1 + qv.y, rv.y);
        rv.z = fmaf(-al, d2 + qv.z, rv.z); rv.w = fmaf(-al, d3 + qv.w, rv.w);
        x[o] = xv;
        r[o] = rv;
        rrf = rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
        xxf = xv.x * xv.x + xv.y * xv.y + xv.z * xv.z + xv.w * xv.w;
        ppf = pv.x * pv.x + pv.y * pv.y + pv.z * pv.z + pv.w * pv.w;
    }
    const bool rel = g->rule == 1;
    double rr = (double)rrf, xx = (double)xxf, pp = (double)ppf;
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
        if (rel) {
            xx += __shfl_xor_sync(0xffffffffu, xx, o);
            pp += __shfl_xor_sync(0xffffffffu, pp, o);
        }
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = rr;
        red[1][threadIdx.x >> 5] = xx;
        red[2][threadIdx.x >> 5] = pp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double t = red[0][0] + red[0][1] + red[0][2] + red[0][3];
        CgBand *bd = bands + b;
        atomicAdd(&bd->rr_new, t);
        if (rel) {
            atomicAdd(&bd->xx_new, red[1][0] + red[1][1] + red[1][2] + red[1][3]);
            atomicAdd(&bd->pp_new, red[2][0] + red[2][1] + red[2][2] + red[2][3]);
        }
        __threadfence();
        const unsigned int k = atomicAdd(&bd->cnt_update, 1u);
        if (k == gridDim.x * gridDim.y - 1) {
            __threadfence();
            const double rn = atomicAdd(&bd->rr_new, 0.0);
            const double xn = atomicAdd(&bd->xx_new, 0.0), pn = atomicAdd(&bd->pp_new, 0.0);
            const double ro = bd->rho;
            bd->cnt_update = 0u;
            bd->rr_new = 0.0;
            bd->xx_new = 0.0;
            bd->pp_new = 0.0;
            bd->pAp = 0.0;
            bd->vv = 0.0;
            bd->iters += 1;
            if (!isfinite(rn)) {
                bd->status = PS_ERR_NONFINITE;
                bd->done = 1;
                bd->beta = 0.0;
            } else {
                if (!g->precond) {
                    bd->beta = rn / ro;
                    bd->rho = rn;
                }
                bd->rr = rn;
                if (cg_converged(g, bd, rn, xn, pn)) {
                    bd->done = 1;
                } else if (bd->iters >= g->max_iter) {
                    bd->status = PS_ERR_NOT_CONVERGED;
                    bd->done = 1;
                }
            }
        }
    }
}

__global__ void cg_control_kernel(CgBand *bands, CgGlobal *g, int N, int use_cond,
                                  cudaGraphConditionalHandle handle) {
    const int lane = threadIdx.x;
    int active = 0, mx = 0;
    for (int b = lane; b < N; b += 32) {
        active += bands[b].done ? 0 : 1;
        mx = max(mx, bands[b].iters);
    }
    for (int o = 16; o > 0; o >>= 1) {
        active += __shfl_xor_sync(0xffffffffu, active, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    // lane 0 decides; every lane then stamps its bands' stop time (a band
    // that stopped in this iteration, or every band when the loop ends here)
    int ending = 0;
    if (lane == 0) {
        unsigned int cond = 1u;
        if (g->stop) {
            cond = 0u;
        } else {
            g->iter += 1;
            g->active = active;
            g->max_iters = mx;
            if (active == 0 || g->iter >= g->max_iter) {
                g->stop = 1;
                cond = 0u;
                ending = 1;
            }
        }
        if (use_cond) cudaGraphSetConditional(handle, cond);
    }
    ending = __shfl_sync(0xffffffffu, ending, 0);
    const unsigned long long now = global_ns();
    for (int b = lane; b < N; b += 32)
        if (bands[b].t_done == 0ull && (bands[b].done || ending)) bands[b].t_done = now;
}

void launch_cg_reset(CgBand *bands, CgGlobal *g, int N, double tol, int max_iter, int precond,
                     int rule, cudaStream_t st) {
    cg_reset_kernel<<<1, 64, 0, st>>>(bands, g, N, tol, max_iter, precond, rule);
}

static int vec_blocks(size_t n4) {
    size_t bl = (n4 + 256 * 4 - 1) / (256 * 4);
    if (bl < 1) bl = 1;
    if (bl > 4096) bl = 4096;
    return (int)bl;
}

void launch_cg_init(const float *bvec, const float *ax0, const float *x0, float *x, float *r,
                    int N, size_t HW, CgBand *bands, CgGlobal *g, cudaStream_t st) {
    const size_t n4 = HW / 4;
    dim3 grd(vec_blocks(n4), N);
    cg_init_kernel<<<grd, 256, 0, st>>>(
        reinterpret_cast<const float4 *>(bvec), reinterpret_cast<const float4 *>(ax0),
        reinterpret_cast<const float4 *>(x0), reinterpret_cast<float4 *>(x),
        reinterpret_cast<float4 *>(r), n4, bands, g);
}

void launch_cg_update(float *x, float *r, const float *p, const float *q, const float *v,
                      const float *u, int R, int c, int N, int H, int W, CgBand *bands,
                      const CgGlobal *g, cudaStream_t st) {
    if (launch_cg_update_fast(x, r, p, q, v, u, R, c, N, H, W, bands, g, st)) return;
    dim3 grd((W / 4 + 127) / 128, H, N);
    cg_update_kernel<<<grd, 128, 0, st>>>(
        reinterpret_cast<float4 *>(x), reinterpret_cast<float4 *>(r),
        reinterpret_cast<const float4 *>(p), reinterpret_cast<const float4 *>(q), v, u, R, c, H,
        W, bands, g);
}

void launch_cg_control(CgBand *bands, CgGlobal *g, int N, int use_cond,
                       cudaGraphConditionalHandle handle, cudaStream_t st) {
    cg_control_kernel<<<1, 32, 0, st>>>(bands, g, N, use_cond, handle);
}

// The device's global nanosecond timer, written by one thread: marks where
// a scene of a batched call starts and ends inside the one graph launch.
__global__ void stamp_kernel(unsigned long long *t) {
    unsigned long long v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    *t = v;
}

void launch_stamp(unsigned long long *t, cudaStream_t st) { stamp_kernel<<<1, 1, 0, st>>>(t); }

}  // namespace ps
