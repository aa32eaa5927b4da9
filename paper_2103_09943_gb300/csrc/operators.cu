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
    float *__restrict__ mu, float *__restrict__ s) {
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
        I[o] = (float)sI[threadIdx.y + RW][threadIdx.x + RW];
        mu[o] = (float)m;
        s[o] = (float)(1.0 / (var + (double)eps));
    }
}

void launch_pan_stats(const float *Y, int H, int W, int r, float eps, float *I,
                      float *mu, float *s, cudaStream_t st) {
    dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8);
    switch (r) {
        case 1: pan_stats_kernel<1><<<grd, blk, 0, st>>>(Y, H, W, eps, I, mu, s); break;
        case 2: pan_stats_kernel<2><<<grd, blk, 0, st>>>(Y, H, W, eps, I, mu, s); break;
        case 3: pan_stats_kernel<3><<<grd, blk, 0, st>>>(Y, H, W, eps, I, mu, s); break;
        default: pan_stats_kernel<4><<<grd, blk, 0, st>>>(Y, H, W, eps, I, mu, s); break;
    }
}

// ----------------------------------------------------------------------------
// v = D B(u) z on the LR grid. One thread per LR site over an 8 x 32 LR tile;
// the HR footprint (c*8 + 2R) x (c*32 + 2R) is staged in shared memory.
// In CG mode the staged value is p_new = r + beta p_old (beta = 0: p_new = r),
// and every CTA also writes p_new for the HR block its LR sites own.
// ----------------------------------------------------------------------------
constexpr int DB_TLX = 32, DB_TLY = 8;

__global__ void __launch_bounds__(256) db_kernel(
    const float *__restrict__ src, const float *__restrict__ rsrc,
    float *__restrict__ pdst, const CgBand *bands, const CgGlobal *g, int cg,
    int H, int W, int c, const float *__restrict__ u, int R,
    float *__restrict__ v) {
    extern __shared__ float sm[];
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
    const int ky0 = blockIdx.y * DB_TLY, kx0 = blockIdx.x * DB_TLX;
    const int oy = c * ky0 - R, ox = c * kx0 - R;
    const int tid = threadIdx.y * DB_TLX + threadIdx.x;
    for (int k = tid; k < nt; k += 256) su[k] = u[k];
    const float *S = src + (size_t)b * HW;
    const float *Rr = cg ? rsrc + (size_t)b * HW : nullptr;
    float *P = cg ? pdst + (size_t)b * HW : nullptr;
    for (int k = tid; k < FY * FX; k += 256) {
        const int yy = k / FX, xx = k - (k / FX) * FX;
        const size_t gi = (size_t)wrapm(oy + yy, H) * W + wrapm(ox + xx, W);
        float val;
        if (cg) {
            val = use_old ? fmaf(beta, S[gi], Rr[gi]) : Rr[gi];
            if (yy >= R && yy < R + c * DB_TLY && xx >= R && xx < R + c * DB_TLX) {
                const int hy = c * ky0 + (yy - R), hx = c * kx0 + (xx - R);
                if (hy < H && hx < W) P[(size_t)hy * W + hx] = val;
            }
        } else {
            val = S[gi];
        }
        sp[k] = val;
    }
    __syncthreads();
    const int ly = threadIdx.y, lx = threadIdx.x;
    const int ky = ky0 + ly, kx = kx0 + lx;
    if (ky < h && kx < w) {
        float acc = 0.0f;
        for (int i = -R; i <= R; ++i) {
            const float *row = sp + (c * ly - i + R) * FX + c * lx + R;
            const float *ur = su + (i + R) * n + R;
            for (int j = -R; j <= R; ++j) acc = fmaf(ur[j], row[-j], acc);
        }
        v[(size_t)b * h * w + (size_t)ky * w + kx] = acc;
    }
}

size_t db_smem_bytes(int c, int R) {
    const int n = 2 * R + 1;
    return sizeof(float) * (((n * n + 3) & ~3) +
                            (size_t)(c * DB_TLY + 2 * R) * (c * DB_TLX + 2 * R));
}

void launch_db(const float *src, const float *rsrc, float *pdst, const CgBand *bands,
               const CgGlobal *g, int cg, int N, int H, int W, int c, const float *u,
               int R, float *v, cudaStream_t st) {
    const int h = H / c, w = W / c;
    dim3 blk(DB_TLX, DB_TLY), grd((w + DB_TLX - 1) / DB_TLX, (h + DB_TLY - 1) / DB_TLY, N);
    db_kernel<<<grd, blk, db_smem_bytes(c, R), st>>>(src, rsrc, pdst, bands, g, cg, H, W,
                                                     c, u, R, v);
}

// ----------------------------------------------------------------------------
// Data term B(u)^T D^T v at one HR pixel: the taps (i, j) with
// (y + i) = 0 and (x + j) = 0 (mod c) pick the LR sample ((y+i)/c, (x+j)/c).
// ----------------------------------------------------------------------------
__device__ __forceinline__ float adj_at(const float *__restrict__ vb, int h, int w, int H,
                                        int W, int c, const float *su, int n, int R,
                                        int y, int x) {
    const int my = ((y - R) % c + c) % c;
    const int mx = ((x - R) % c + c) % c;
    const int i0 = -R + (c - my) % c;
    const int j0 = -R + (c - mx) % c;
    float acc = 0.0f;
    for (int i = i0; i <= R; i += c) {
        const int ky = wrapm(y + i, H) / c;
        const float *vr = vb + (size_t)ky * w;
        const float *ur = su + (i + R) * n + R;
        for (int j = j0; j <= R; j += c) {
            const int kx = wrapm(x + j, W) / c;
            acc = fmaf(ur[j], __ldg(vr + kx), acc);
        }
    }
    (void)h;
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
        adj_at(v + (size_t)b * h * w, h, w, H, W, c, su, n, R, y, x);
}

void launch_adj(const float *v, int N, int H, int W, int c, const float *u, int R,
                float *z, cudaStream_t st) {
    dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8, N);
    adj_kernel<<<grd, blk, 0, st>>>(v, H, W, c, u, R, z);
}

// ----------------------------------------------------------------------------
// Fused LLP tile kernel. Output tile 32 x 32, 256 threads.
//
// For the input field alpha (alpha = L p in modes APPLY / ZRHS, alpha = q in
// mode GF) every window j gets the affine fit of Eq. ac_h_compute,
//   a_j = (mean_j(I alpha) - mu_j mean_j(alpha)) s_j,  b_j = mean_j(alpha) - a_j mu_j,
// and with Sa, Sb their sums over the windows containing a pixel:
//   guided filter   GF(alpha) = (Sa I + Sb) / |w|
//   matting matrix  M alpha   = |w| alpha - Sa I - Sb = |w| (alpha - GF(alpha)).
// Modes:
//   APPLY: out = B^T D^T v + lam L M L p            (Eq. Z_ini_matting operator)
//          and, in CG, p^T out accumulated per band (FP64) with the last CTA
//          of the band computing alpha = r^T r / p^T A p.
//   ZRHS:  out = B^T D^T X + lam L GF(L z0)          (Eq. Z_solution rhs),
//          written into the packed complex FFT buffer (band 2k -> real,
//          band 2k+1 -> imaginary part of image k).
//   GF:    out = GF(q).
// Shared-memory regions (relative to the tile origin, G = 2r+2):
//   P   = input on T+G          A, I, IA = alpha, I, I*alpha on T+(2r+1)
//   HS  = row sums on rows T+(2r+1), cols T+(r+1)
//   AB  = a, b on T+(r+1)      HAB = row sums of a, b on rows T+(r+1), cols T+1
//   MM  = M alpha or GF(alpha) on T+1
// ----------------------------------------------------------------------------
constexpr int LT = 32;

template <int RW>
struct LlpDims {
    static constexpr int G = 2 * RW + 2;
    static constexpr int AO = 2 * RW + 1, BO = RW + 1;
    static constexpr int PY = LT + 2 * G, PX = PY;
    static constexpr int AY = LT + 2 * AO, AX = AY;
    static constexpr int BY = LT + 2 * BO, BX = BY;
    static constexpr int CY = LT + 2, CX = CY;
    static constexpr int szP = PY * PX, szA = AY * AX, szHS = AY * BX, szB = BY * BX,
                         szHB = BY * CX, szC = CY * CX;
    static constexpr int total = szP + 3 * szA + 2 * szHS + 2 * szB + 2 * szHB + szC;
};

template <int RW>
size_t llp_smem_bytes_t() {
    return sizeof(float) * (LlpDims<RW>::total + ((kMaxTaps + 3) & ~3)) + 64 * sizeof(double);
}

size_t llp_smem_bytes(int r) {
    switch (r) {
        case 1: return llp_smem_bytes_t<1>();
        case 2: return llp_smem_bytes_t<2>();
        case 3: return llp_smem_bytes_t<3>();
        default: return llp_smem_bytes_t<4>();
    }
}

template <int RW, int MODE>
__global__ void __launch_bounds__(256) llp_kernel(LlpArgs a) {
    using D = LlpDims<RW>;
    extern __shared__ float sm[];
    const int b = blockIdx.z;
    if (MODE == LLP_APPLY && a.cg) {
        if (a.g->stop || a.bands[b].done) return;
    }
    float *sP = sm;
    float *sA = sP + D::szP;
    float *sI = sA + D::szA;
    float *sIA = sI + D::szA;
    float *hS1 = sIA + D::szA;
    float *hS2 = hS1 + D::szHS;
    float *sa = hS2 + D::szHS;
    float *sb = sa + D::szB;
    float *ha = sb + D::szB;
    float *hb = ha + D::szHB;
    float *sM = hb + D::szHB;
    float *su = sM + D::szC;
    double *red = reinterpret_cast<double *>(su + ((kMaxTaps + 3) & ~3));

    const int H = a.H, W = a.W;
    const size_t HW = (size_t)H * W;
    const int y0 = blockIdx.y * LT, x0 = blockIdx.x * LT;
    const int tid = threadIdx.x;
    const float *in = a.in + (size_t)b * HW;
    constexpr float nw = (float)((2 * RW + 1) * (2 * RW + 1));
    const int n = 2 * a.R + 1;

    if (MODE != LLP_GF)
        for (int k = tid; k < n * n; k += 256) su[k] = a.u[k];

    // Phase 0/1: alpha, I, I*alpha on T + (2r+1).
    if (MODE == LLP_GF) {
        for (int k = tid; k < D::szA; k += 256) {
            const int yy = k / D::AX, xx = k - (k / D::AX) * D::AX;
            const size_t gi = (size_t)wrapm(y0 - D::AO + yy, H) * W + wrapm(x0 - D::AO + xx, W);
            const float al = in[gi], iv = a.I[gi];
            sA[k] = al;
            sI[k] = iv;
            sIA[k] = iv * al;
        }
    } else {
        for (int k = tid; k < D::szP; k += 256) {
            const int yy = k / D::PX, xx = k - (k / D::PX) * D::PX;
            sP[k] = in[(size_t)wrapm(y0 - D::G + yy, H) * W + wrapm(x0 - D::G + xx, W)];
        }
        __syncthreads();
        for (int k = tid; k < D::szA; k += 256) {
            const int yy = k / D::AX, xx = k - (k / D::AX) * D::AX;
            const float *pc = sP + (yy + 1) * D::PX + (xx + 1);
            const float al = 4.0f * pc[0] - pc[-D::PX] - pc[D::PX] - pc[-1] - pc[1];
            const float iv =
                a.I[(size_t)wrapm(y0 - D::AO + yy, H) * W + wrapm(x0 - D::AO + xx, W)];
            sA[k] = al;
            sI[k] = iv;
            sIA[k] = iv * al;
        }
    }
    __syncthreads();
    // Phase 2: row sums over 2r+1 columns.
    for (int k = tid; k < D::szHS; k += 256) {
        const int yy = k / D::BX, xx = k - (k / D::BX) * D::BX;
        const float *r1 = sA + yy * D::AX + xx;
        const float *r2 = sIA + yy * D::AX + xx;
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int d = 0; d <= 2 * RW; ++d) {
            s1 += r1[d];
            s2 += r2[d];
        }
        hS1[k] = s1;
        hS2[k] = s2;
    }
    __syncthreads();
    // Phase 3: column sums -> window means -> affine fit (a, b) on T + (r+1).
    for (int k = tid; k < D::szB; k += 256) {
        const int yy = k / D::BX, xx = k - (k / D::BX) * D::BX;
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int d = 0; d <= 2 * RW; ++d) {
            s1 += hS1[(yy + d) * D::BX + xx];
            s2 += hS2[(yy + d) * D::BX + xx];
        }
        const size_t gi = (size_t)wrapm(y0 - D::BO + yy, H) * W + wrapm(x0 - D::BO + xx, W);
        const float m = a.mu[gi], sv = a.s[gi];
        const float ma = s1 * (1.0f / nw), mia = s2 * (1.0f / nw);
        const float av = (mia - m * ma) * sv;
        sa[k] = av;
        sb[k] = ma - av * m;
    }
    __syncthreads();
    // Phase 4: row sums of a, b.
    for (int k = tid; k < D::szHB; k += 256) {
        const int yy = k / D::CX, xx = k - (k / D::CX) * D::CX;
        const float *r1 = sa + yy * D::BX + xx;
        const float *r2 = sb + yy * D::BX + xx;
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int d = 0; d <= 2 * RW; ++d) {
            s1 += r1[d];
            s2 += r2[d];
        }
        ha[k] = s1;
        hb[k] = s2;
    }
    __syncthreads();
    // Phase 5: column sums -> M alpha (APPLY) or GF(alpha) (ZRHS, GF) on T + 1.
    for (int k = tid; k < D::szC; k += 256) {
        const int yy = k / D::CX, xx = k - (k / D::CX) * D::CX;
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int d = 0; d <= 2 * RW; ++d) {
            s1 += ha[(yy + d) * D::CX + xx];
            s2 += hb[(yy + d) * D::CX + xx];
        }
        const int ai = (yy + 2 * RW) * D::AX + (xx + 2 * RW);
        const float iv = sI[ai];
        if (MODE == LLP_APPLY)
            sM[k] = nw * sA[ai] - s1 * iv - s2;
        else
            sM[k] = (s1 * iv + s2) * (1.0f / nw);
    }
    __syncthreads();
    // Phase 6: outputs.
    const int h = H / a.c, w = W / a.c;
    float part = 0.0f;
    for (int k = tid; k < LT * LT; k += 256) {
        const int ty = k >> 5, tx = k & 31;
        const int y = y0 + ty, x = x0 + tx;
        if (y >= H || x >= W) continue;
        const float *mc = sM + (ty + 1) * D::CX + (tx + 1);
        float val;
        if (MODE == LLP_GF) {
            val = mc[0];
        } else {
            const float lm = 4.0f * mc[0] - mc[-D::CX] - mc[D::CX] - mc[-1] - mc[1];
            const float dat = adj_at(a.lr + (size_t)b * h * w, h, w, H, W, a.c, su, n, a.R, y, x);
            val = fmaf(a.lam, lm, dat);
        }
        const size_t o = (size_t)y * W + x;
        if (MODE == LLP_ZRHS) {
            float2 *cimg = a.cout + (size_t)(b >> 1) * HW + o;
            if (b & 1)
                reinterpret_cast<float *>(cimg)[1] = val;
            else if (b == a.N - 1)
                *cimg = make_float2(val, 0.0f);
            else
                reinterpret_cast<float *>(cimg)[0] = val;
        } else {
            a.out[(size_t)b * HW + o] = val;
        }
        if (MODE == LLP_APPLY && a.cg) part = fmaf(sP[(ty + D::G) * D::PX + (tx + D::G)], val, part);
    }
    if (MODE == LLP_APPLY && a.cg) {
        const double tot = block_sum_d((double)part, red);
        if (tid == 0) {
            CgBand *bd = a.bands + b;
            atomicAdd(&bd->pAp, tot);
            __threadfence();
            const unsigned int nblk = gridDim.x * gridDim.y;
            const unsigned int t = atomicAdd(&bd->cnt_apply, 1u);
            if (t == nblk - 1) {
                __threadfence();
                const double pAp = atomicAdd(&bd->pAp, 0.0);
                const double rr = bd->rr;
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
                    bd->alpha = rr / pAp;
                }
            }
        }
    }
}

template <int RW>
static void launch_llp_r(const LlpArgs &a, int mode, dim3 grd, cudaStream_t st) {
    const size_t sm = llp_smem_bytes_t<RW>();
    switch (mode) {
        case LLP_APPLY: llp_kernel<RW, LLP_APPLY><<<grd, 256, sm, st>>>(a); break;
        case LLP_ZRHS: llp_kernel<RW, LLP_ZRHS><<<grd, 256, sm, st>>>(a); break;
        default: llp_kernel<RW, LLP_GF><<<grd, 256, sm, st>>>(a); break;
    }
}

template <int RW>
static cudaError_t llp_set_attrs_r() {
    const int sm = (int)llp_smem_bytes_t<RW>();
    cudaError_t e;
    e = cudaFuncSetAttribute(llp_kernel<RW, LLP_APPLY>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(llp_kernel<RW, LLP_ZRHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(llp_kernel<RW, LLP_GF>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

cudaError_t operators_set_attrs() {
    cudaError_t e;
    if ((e = llp_set_attrs_r<1>()) != cudaSuccess) return e;
    if ((e = llp_set_attrs_r<2>()) != cudaSuccess) return e;
    if ((e = llp_set_attrs_r<3>()) != cudaSuccess) return e;
    if ((e = llp_set_attrs_r<4>()) != cudaSuccess) return e;
    return cudaFuncSetAttribute(db_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)db_smem_bytes(8, kMaxR));
}

void launch_llp(const LlpArgs &a, int mode, int r, int N, cudaStream_t st) {
    dim3 grd((a.W + LT - 1) / LT, (a.H + LT - 1) / LT, N);
    switch (r) {
        case 1: launch_llp_r<1>(a, mode, grd, st); break;
        case 2: launch_llp_r<2>(a, mode, grd, st); break;
        case 3: launch_llp_r<3>(a, mode, grd, st); break;
        default: launch_llp_r<4>(a, mode, grd, st); break;
    }
}

// ----------------------------------------------------------------------------
// CG bookkeeping. Every per-band decision is taken by the last CTA of that
// band to arrive (atomic counter, no waiting); the loop condition is taken by
// a one-warp control kernel that always runs, so the device loop ends after
// at most max_iter iterations whatever the band states.
// ----------------------------------------------------------------------------
__global__ void cg_reset_kernel(CgBand *bands, CgGlobal *g, int N, double tol, int max_iter) {
    const int t = threadIdx.x;
    for (int b = t; b < N; b += blockDim.x) {
        CgBand z = {};
        bands[b] = z;
    }
    if (t == 0) {
        g->cnt_bands = 0u;
        g->active = N;
        g->max_iters = 0;
        g->stop = 0;
        g->iter = 0;
        g->max_iter = max_iter;
        g->tol = tol;
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
            bd->bb = b2;
            bd->rr_new = 0.0;
            bd->pAp = 0.0;
            bd->beta = 0.0;
            bd->alpha = 0.0;
            bd->iters = 0;
            bd->cnt_init = 0u;
            if (!isfinite(r2) || !isfinite(b2)) {
                bd->status = PS_ERR_NONFINITE;
                bd->done = 1;
            } else if (b2 == 0.0 || sqrt(r2 / b2) <= g->tol) {
                bd->done = 1;
            }
        }
    }
}

// x += alpha p; r -= alpha Ap; the next r^T r; the band's last CTA takes
// beta, the convergence test and the iteration cap.
__global__ void __launch_bounds__(256) cg_update_kernel(float4 *__restrict__ x,
                                                        float4 *__restrict__ r,
                                                        const float4 *__restrict__ p,
                                                        const float4 *__restrict__ ap,
                                                        size_t n4, CgBand *bands,
                                                        const CgGlobal *g) {
    __shared__ double red[8];
    const int b = blockIdx.y;
    if (g->stop || bands[b].done) return;
    const float al = (float)bands[b].alpha;
    const size_t off = (size_t)b * n4;
    double rr = 0.0;
    for (size_t i = blockIdx.x * 256 + threadIdx.x; i < n4; i += (size_t)gridDim.x * 256) {
        float4 xv = x[off + i], rv = r[off + i];
        const float4 pv = p[off + i], av = ap[off + i];
        xv.x = fmaf(al, pv.x, xv.x); xv.y = fmaf(al, pv.y, xv.y);
        xv.z = fmaf(al, pv.z, xv.z); xv.w = fmaf(al, pv.w, xv.w);
        rv.x = fmaf(-al, av.x, rv.x); rv.y = fmaf(-al, av.y, rv.y);
        rv.z = fmaf(-al, av.z, rv.z); rv.w = fmaf(-al, av.w, rv.w);
        x[off + i] = xv;
        r[off + i] = rv;
        rr += (double)(rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w);
    }
    const double t = block_sum_d(rr, red);
    if (threadIdx.x == 0) {
        CgBand *bd = bands + b;
        atomicAdd(&bd->rr_new, t);
        __threadfence();
        const unsigned int k = atomicAdd(&bd->cnt_update, 1u);
        if (k == gridDim.x - 1) {
            __threadfence();
            const double rn = atomicAdd(&bd->rr_new, 0.0);
            const double ro = bd->rr;
            bd->cnt_update = 0u;
            bd->rr_new = 0.0;
            bd->pAp = 0.0;
            bd->iters += 1;
            if (!isfinite(rn)) {
                bd->status = PS_ERR_NONFINITE;
                bd->done = 1;
                bd->beta = 0.0;
            } else {
                bd->beta = rn / ro;
                bd->rr = rn;
                if (sqrt(rn / bd->bb) <= g->tol) {
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
            }
        }
        if (use_cond) cudaGraphSetConditional(handle, cond);
    }
}

void launch_cg_reset(CgBand *bands, CgGlobal *g, int N, double tol, int max_iter,
                     cudaStream_t st) {
    cg_reset_kernel<<<1, 64, 0, st>>>(bands, g, N, tol, max_iter);
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

void launch_cg_update(float *x, float *r, const float *p, const float *ap, int N, size_t HW,
                      CgBand *bands, const CgGlobal *g, cudaStream_t st) {
    const size_t n4 = HW / 4;
    dim3 grd(vec_blocks(n4), N);
    cg_update_kernel<<<grd, 256, 0, st>>>(
        reinterpret_cast<float4 *>(x), reinterpret_cast<float4 *>(r),
        reinterpret_cast<const float4 *>(p), reinterpret_cast<const float4 *>(ap), n4, bands,
        g);
}

void launch_cg_control(CgBand *bands, CgGlobal *g, int N, int use_cond,
                       cudaGraphConditionalHandle handle, cudaStream_t st) {
    cg_control_kernel<<<1, 32, 0, st>>>(bands, g, N, use_cond, handle);
}

}  // namespace ps
