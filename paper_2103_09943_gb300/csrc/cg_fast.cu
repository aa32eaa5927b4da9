// CG-loop kernels specialised for a compile-time resolution ratio C and
// kernel radius R (sm_103a). With both known, the tap loops unroll completely,
// every register and shared-memory index becomes a constant, and a tap costs
// one broadcast shared load of u and one FMA per output it feeds.
//
//   db_site_kernel<C,R>        v = D B(u) p_new for 8 x 32 LR sites per CTA,
//                              with p_new = r + beta p_old fused into the load
//                              and ||v||^2 accumulated per band
//   cg_update_site_kernel<C,R> one thread per LR site: B^T D^T v for its C x C
//                              block of HR pixels (from a register window of
//                              v), then x += alpha p, r -= alpha (B^T D^T v + q)
//                              and the next r^T r
//
// Instantiated for C in {2, 4} and R in [1, 8]; compiled a second time with
// PS_SITE_WIDE (cg_fast_wide.cu, a translation unit of its own so that the two
// build in parallel) for C = 4 and R in {12, 14, 16}, the paper's 29 x 29
// support among them. Other sizes use the generic kernels of operators.cu.
#include "common.cuh"
#include "kernels.cuh"

#ifdef PS_SITE_WIDE
#define PS_SITE_FN(name) name##_wide
#else
#define PS_SITE_FN(name) name
#endif

namespace ps {

namespace {

__device__ __forceinline__ int wrap_mod(int i, int n) {
    int m = i % n;
    return m < 0 ? m + n : m;
}

constexpr int SITE_TX = 32, SITE_TYT = 4, SITE_K = 2, SITE_TY = SITE_TYT * SITE_K;

template <int C, int R>
struct SiteDims {
    static constexpr int n = 2 * R + 1;
    static constexpr int FY = C * SITE_TY + 2 * R;
    static constexpr int FX = C * SITE_TX + 2 * R;
    static constexpr int FXp = (FX + C - 1) / C;
    // plane stride padded so that the C planes start on different banks
    static constexpr int plane0 = FY * FXp;
    static constexpr int plane = plane0 + ((40 - plane0 % 32) % 32);
    static constexpr int smem_floats = ((n * n + 3) & ~3) + C * plane;
};

template <int C, int R>
__global__ void __launch_bounds__(128) db_site_kernel(const float *__restrict__ src,
                                                      const float *__restrict__ rsrc,
                                                      float *__restrict__ pdst, CgBand *bands,
                                                      const CgGlobal *g, int cg, int H, int W,
                                                      const float *__restrict__ u,
                                                      float *__restrict__ v) {
    using D = SiteDims<C, R>;
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
    const int h = H / C, w = W / C;
    const size_t HW = (size_t)H * W;
    float *su = sm;
    float *sp = sm + ((D::n * D::n + 3) & ~3);
    const int ky0 = blockIdx.y * SITE_TY, kx0 = blockIdx.x * SITE_TX;
    const int oy = C * ky0 - R, ox = C * kx0 - R;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * SITE_TX + tx;
    for (int k = tid; k < D::n * D::n; k += 128) su[k] = u[k];
    const float *S = src + (size_t)b * HW;
    const float *Rr = cg ? rsrc + (size_t)b * HW : nullptr;
    float *P = cg ? pdst + (size_t)b * HW : nullptr;
    // Fill: every footprint row's loads are issued before any is used, so a
    // thread keeps 2 * ceil(FX / 32) loads in flight.
    constexpr int NXW = (D::FX + 31) / 32;
    const int gx0 = wrap_mod(ox + tx, W);
#pragma unroll 2
    for (int yy = ty; yy < D::FY; yy += SITE_TYT) {
        const size_t grow = (size_t)wrap_mod(oy + yy, H) * W;
        const bool own_row = cg && yy >= R && yy < R + C * SITE_TY && C * ky0 + (yy - R) < H;
        float rv[NXW], pv[NXW];
        int gx = gx0;
#pragma unroll
        for (int m = 0; m < NXW; ++m) {
            if (tx + 32 * m < D::FX) {
                const size_t gi = grow + gx;
                if (cg) {
                    rv[m] = Rr[gi];
                    pv[m] = use_old ? S[gi] : 0.0f;
                } else {
                    rv[m] = S[gi];
                    pv[m] = 0.0f;
                }
            }
            gx += 32;
            while (gx >= W) gx -= W;
        }
#pragma unroll
        for (int m = 0; m < NXW; ++m) {
            const int xx = tx + 32 * m;
            if (xx < D::FX) {
                const float val = (cg && use_old) ? fmaf(beta, pv[m], rv[m]) : rv[m];
                if (own_row && xx >= R && xx < R + C * SITE_TX) {
                    const int hx = C * kx0 + (xx - R);
                    if (hx < W) P[(size_t)(C * ky0 + (yy - R)) * W + hx] = val;
                }
                sp[(xx % C) * D::plane + yy * D::FXp + xx / C] = val;
            }
        }
    }
    __syncthreads();
    // sites (ty + 4 k, tx), k < SITE_K; sample (C ky - i, C kx - j) lives at
    // footprint row C ty - i + R, column C tx + t with t = R - j. Each tap's
    // weight is one broadcast load shared by the thread's SITE_K sites.
    float acc[SITE_K];
#pragma unroll
    for (int k = 0; k < SITE_K; ++k) acc[k] = 0.0f;
    const float *base = sp + (C * ty + R) * D::FXp + tx;
    constexpr int rstep = C * SITE_TYT * D::FXp;
#pragma unroll
    for (int i = -R; i <= R; ++i) {
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t) {
            const float uv = su[(i + R) * D::n + (2 * R - t)];
            const float *bp = base + (t % C) * D::plane - i * D::FXp + t / C;
#pragma unroll
            for (int k = 0; k < SITE_K; ++k) acc[k] = fmaf(uv, bp[k * rstep], acc[k]);
        }
    }
    const int kx = kx0 + tx;
    float vv = 0.0f;
    if (kx < w) {
#pragma unroll
        for (int k = 0; k < SITE_K; ++k) {
            const int ky = ky0 + ty + k * SITE_TYT;
            if (ky < h) {
                v[(size_t)b * h * w + (size_t)ky * w + kx] = acc[k];
                vv = fmaf(acc[k], acc[k], vv);
            }
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

// ---------------------------------------------------------------------------
// v = D B(u) p_new, register-blocked (the autotuner's db_impl = 2; measured
// 5-10 % faster than db_site_kernel at 1024^2 with R = 6..8, slower at 512^2
// and 2048^2): a CTA of 128 threads covers 16 x 32 LR
// sites; thread (g, kyl) takes the four sites kx0 + 4 g + s (s < 4) of row
// ky0 + kyl. The footprint is stored as C phase planes (HR column x in plane
// x mod C at entry x div C), so for a tap row i the samples of the four
// sites and of every tap column lie in C short runs of consecutive entries:
// per tap row the thread loads NCH aligned float4 of each plane into
// registers and feeds its four accumulators from them, one broadcast load of
// the weight per tap (about a quarter of the shared loads of one load per
// sample and site).
// ---------------------------------------------------------------------------
constexpr int S4_GX = 8, S4_TY = 16, S4_TX = 4 * S4_GX;

template <int C, int R>
struct Site4Dims {
    static constexpr int n = 2 * R + 1;
    static constexpr int FY = C * S4_TY + 2 * R;
    static constexpr int FX = C * S4_TX + 2 * R;
    static constexpr int MMAX = (n + C - 1) / C;       // taps per plane, at most
    static constexpr int NCH = (3 + MMAX + 3) / 4;     // float4 runs per plane and tap row
    static constexpr int FXc = (FX + C - 1) / C;
    static constexpr int FXr = 4 * (S4_GX - 1) + 4 * NCH;
    static constexpr int FXp = (((FXc > FXr) ? FXc : FXr) + 3) & ~3;
    static constexpr int plane = FY * FXp;             // a multiple of 4
    static constexpr int uoff = (n * n + 3) & ~3;
    static constexpr int smem_floats = uoff + C * plane;
};

template <int C, int R>
__global__ void __launch_bounds__(128) db_site4_kernel(const float *__restrict__ src,
                                                       const float *__restrict__ rsrc,
                                                       float *__restrict__ pdst, CgBand *bands,
                                                       const CgGlobal *g, int cg, int H, int W,
                                                       const float *__restrict__ u,
                                                       float *__restrict__ v) {
    using D = Site4Dims<C, R>;
    extern __shared__ __align__(16) float sm4[];
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
    const int h = H / C, w = W / C;
    const size_t HW = (size_t)H * W;
    float *su = sm4;
    float *sp = sm4 + D::uoff;
    const int ky0 = blockIdx.y * S4_TY, kx0 = blockIdx.x * S4_TX;
    const int oy = C * ky0 - R, ox = C * kx0 - R;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    for (int k = tid; k < D::n * D::n; k += 128) su[k] = u[k];
    const float *S = src + (size_t)b * HW;
    const float *Rr = cg ? rsrc + (size_t)b * HW : nullptr;
    float *P = cg ? pdst + (size_t)b * HW : nullptr;
    // fill (p_new = r + beta p_old fused into the load; own pixels stored)
    constexpr int NXW = (D::FX + 31) / 32;
    const int gx0 = wrap_mod(ox + tx, W);
#pragma unroll 2
    for (int yy = ty; yy < D::FY; yy += 4) {
        const size_t grow = (size_t)wrap_mod(oy + yy, H) * W;
        const bool own_row = cg && yy >= R && yy < R + C * S4_TY && C * ky0 + (yy - R) < H;
        float rv[NXW], pv[NXW];
        int gx = gx0;
#pragma unroll
        for (int m = 0; m < NXW; ++m) {
            if (tx + 32 * m < D::FX) {
                const size_t gi = grow + gx;
                if (cg) {
                    rv[m] = Rr[gi];
                    pv[m] = use_old ? S[gi] : 0.0f;
                } else {
                    rv[m] = S[gi];
                    pv[m] = 0.0f;
                }
            }
            gx += 32;
            while (gx >= W) gx -= W;
        }
#pragma unroll
        for (int m = 0; m < NXW; ++m) {
            const int xx = tx + 32 * m;
            if (xx < D::FX) {
                const float val = (cg && use_old) ? fmaf(beta, pv[m], rv[m]) : rv[m];
                if (own_row && xx >= R && xx < R + C * S4_TX) {
                    const int hx = C * kx0 + (xx - R);
                    if (hx < W) P[(size_t)(C * ky0 + (yy - R)) * W + hx] = val;
                }
                sp[(xx % C) * D::plane + yy * D::FXp + xx / C] = val;
            }
        }
    }
    __syncthreads();
    // site (kyl, 4 g + s); tap (i, j = R - jj) reads footprint row
    // C kyl + R - i, plane jj mod C, entry 4 g + s + jj div C
    const int gq = tid & (S4_GX - 1), kyl = tid >> 3;
    const float *rowbase = sp + (C * kyl + R) * D::FXp + 4 * gq;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = -R; i <= R; ++i) {
        const float *rp = rowbase - i * D::FXp;
        float vals[C][4 * D::NCH];
#pragma unroll
        for (int p = 0; p < C; ++p)
#pragma unroll
            for (int c = 0; c < D::NCH; ++c) {
                const float4 q = *reinterpret_cast<const float4 *>(rp + p * D::plane + 4 * c);
                vals[p][4 * c] = q.x;
                vals[p][4 * c + 1] = q.y;
                vals[p][4 * c + 2] = q.z;
                vals[p][4 * c + 3] = q.w;
            }
#pragma unroll
        for (int jj = 0; jj <= 2 * R; ++jj) {
            const float wv = su[(i + R) * D::n + (2 * R - jj)];
#pragma unroll
            for (int s2 = 0; s2 < 4; ++s2)
                acc[s2] = fmaf(wv, vals[jj % C][jj / C + s2], acc[s2]);
        }
    }
    const int ky = ky0 + kyl;
    float vv = 0.0f;
    if (ky < h) {
        float *vrow = v + (size_t)b * h * w + (size_t)ky * w;
#pragma unroll
        for (int s2 = 0; s2 < 4; ++s2) {
            const int kx = kx0 + 4 * gq + s2;
            if (kx < w) {
                vrow[kx] = acc[s2];
                vv = fmaf(acc[s2], acc[s2], vv);
            }
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

template <int C>
struct VecT;
template <>
struct VecT<2> {
    using T = float2;
};
template <>
struct VecT<4> {
    using T = float4;
};

__device__ __forceinline__ void vupd(float2 &x, float2 &r, float2 p, float2 q, const float *d,
                                     float al, float &rr) {
    x.x = fmaf(al, p.x, x.x);
    x.y = fmaf(al, p.y, x.y);
    r.x = fmaf(-al, d[0] + q.x, r.x);
    r.y = fmaf(-al, d[1] + q.y, r.y);
    rr = fmaf(r.x, r.x, fmaf(r.y, r.y, rr));
}

__device__ __forceinline__ void vupd(float4 &x, float4 &r, float4 p, float4 q, const float *d,
                                     float al, float &rr) {
    x.x = fmaf(al, p.x, x.x);
    x.y = fmaf(al, p.y, x.y);
    x.z = fmaf(al, p.z, x.z);
    x.w = fmaf(al, p.w, x.w);
    r.x = fmaf(-al, d[0] + q.x, r.x);
    r.y = fmaf(-al, d[1] + q.y, r.y);
    r.z = fmaf(-al, d[2] + q.z, r.z);
    r.w = fmaf(-al, d[3] + q.w, r.w);
    rr = fmaf(r.x, r.x, fmaf(r.y, r.y, fmaf(r.z, r.z, fmaf(r.w, r.w, rr))));
}

__device__ __forceinline__ float vsq(float2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float vsq(float4 a) {
    return a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
}

// B^T D^T v on the C x C block of LR site (ky, kx): pixel (C ky + a, C kx + b)
// takes tap (i, j) exactly when i = -a and j = -b (mod C), with the sample
// v(ky + (a + i)/C, kx + (b + j)/C).
template <int C, int R>
__global__ void __launch_bounds__(128) cg_update_site_kernel(
    float *__restrict__ x, float *__restrict__ r, const float *__restrict__ p,
    const float *__restrict__ q, const float *__restrict__ v, const float *__restrict__ u,
    int H, int W, CgBand *bands, const CgGlobal *g) {
    constexpr int n = 2 * R + 1;
    constexpr int K0 = -(R / C);
    constexpr int K1 = (C - 1 + R) / C;
    constexpr int KN = K1 - K0 + 1;
    using V = typename VecT<C>::T;
    __shared__ float su[n * n];
    __shared__ double red[3][4];
    const int b = blockIdx.z, ky = blockIdx.y;
    if (g->stop || bands[b].done) return;
    for (int k = threadIdx.x; k < n * n; k += 128) su[k] = u[k];
    __syncthreads();
    const int h = H / C, w = W / C;
    const int kx = blockIdx.x * 128 + threadIdx.x;
    float rrf = 0.0f, xxf = 0.0f, ppf = 0.0f;
    const bool rel = g->rule == 1;
    if (kx < w) {
        const float *vb = v + (size_t)b * h * w;
        float vw[KN][KN];
#pragma unroll
        for (int dy = 0; dy < KN; ++dy) {
            const float *vr = vb + (size_t)wrap_mod(ky + K0 + dy, h) * w;
#pragma unroll
            for (int dx = 0; dx < KN; ++dx) vw[dy][dx] = __ldg(vr + wrap_mod(kx + K0 + dx, w));
        }
        float acc[C][C];
#pragma unroll
        for (int a = 0; a < C; ++a)
#pragma unroll
            for (int bb = 0; bb < C; ++bb) acc[a][bb] = 0.0f;
#pragma unroll
        for (int i = -R; i <= R; ++i) {
            const int a = ((-i) % C + C) % C;
            const int dy = (a + i) / C - K0;
#pragma unroll
            for (int j = -R; j <= R; ++j) {
                const int bb = ((-j) % C + C) % C;
                const int dx = (bb + j) / C - K0;
                acc[a][bb] = fmaf(su[(i + R) * n + (j + R)], vw[dy][dx], acc[a][bb]);
            }
        }
        const float al = (float)bands[b].alpha;
#pragma unroll
        for (int a = 0; a < C; ++a) {
            const size_t o = ((size_t)b * H + (size_t)(C * ky + a)) * W + (size_t)C * kx;
            V xv = *reinterpret_cast<const V *>(x + o);
            V rv = *reinterpret_cast<const V *>(r + o);
            const V pv = __ldg(reinterpret_cast<const V *>(p + o));
            const V qv = __ldg(reinterpret_cast<const V *>(q + o));
            vupd(xv, rv, pv, qv, acc[a], al, rrf);
            if (rel) {
                xxf += vsq(xv);
                ppf += vsq(pv);
            }
            *reinterpret_cast<V *>(x + o) = xv;
            *reinterpret_cast<V *>(r + o) = rv;
        }
    }
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

template <int C, int R>
bool launch_pair(int which, const float *a0, const float *a1, float *a2, CgBand *bands,
                 const CgGlobal *g, int cg, int N, int H, int W, const float *u, float *v,
                 float *x, float *r, const float *q, cudaStream_t st, int impl) {
    const int h = H / C, w = W / C;
    if (which == 0 && impl != 2) {
        using D = SiteDims<C, R>;
        dim3 blk(SITE_TX, SITE_TYT), grd((w + SITE_TX - 1) / SITE_TX, (h + SITE_TY - 1) / SITE_TY, N);
        db_site_kernel<C, R><<<grd, blk, D::smem_floats * sizeof(float), st>>>(
            a0, a1, a2, bands, g, cg, H, W, u, v);
    } else if (which == 0) {
        using D = Site4Dims<C, R>;
        dim3 grd((w + S4_TX - 1) / S4_TX, (h + S4_TY - 1) / S4_TY, N);
        db_site4_kernel<C, R><<<grd, 128, D::smem_floats * sizeof(float), st>>>(
            a0, a1, a2, bands, g, cg, H, W, u, v);
    } else {
        dim3 grd((w + 127) / 128, h, N);
        cg_update_site_kernel<C, R><<<grd, 128, 0, st>>>(x, r, a0, q, v, u, H, W, bands, g);
    }
    return true;
}

template <int C>
bool dispatch_r(int R, int which, const float *a0, const float *a1, float *a2, CgBand *bands,
                const CgGlobal *g, int cg, int N, int H, int W, const float *u, float *v,
                float *x, float *r, const float *q, cudaStream_t st, int impl) {
    switch (R) {
#define PS_CASE(RR)                                                                          \
    case RR:                                                                                 \
        return launch_pair<C, RR>(which, a0, a1, a2, bands, g, cg, N, H, W, u, v, x, r, q, \
                                  st, impl);
#ifdef PS_SITE_WIDE
        PS_CASE(12) PS_CASE(14) PS_CASE(16)
#else
        PS_CASE(1) PS_CASE(2) PS_CASE(3) PS_CASE(4) PS_CASE(5) PS_CASE(6) PS_CASE(7) PS_CASE(8)
#endif
#undef PS_CASE
        default: return false;
    }
}

bool dispatch(int C, int R, int which, const float *a0, const float *a1, float *a2,
              CgBand *bands, const CgGlobal *g, int cg, int N, int H, int W, const float *u,
              float *v, float *x, float *r, const float *q, cudaStream_t st, int impl = 0) {
    if (C == 4)
        return dispatch_r<4>(R, which, a0, a1, a2, bands, g, cg, N, H, W, u, v, x, r, q, st, impl);
#ifndef PS_SITE_WIDE
    if (C == 2)
        return dispatch_r<2>(R, which, a0, a1, a2, bands, g, cg, N, H, W, u, v, x, r, q, st, impl);
#endif
    return false;
}

template <int C, int R>
cudaError_t set_attr_one() {
    cudaError_t e = cudaFuncSetAttribute(db_site_kernel<C, R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(SiteDims<C, R>::smem_floats * sizeof(float)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(db_site4_kernel<C, R>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(Site4Dims<C, R>::smem_floats * sizeof(float)));
    return e;
}

template <int C>
cudaError_t set_attrs_c() {
    cudaError_t e = cudaSuccess;
#define PS_ATTR(RR) \
    if (e == cudaSuccess) e = set_attr_one<C, RR>();
#ifdef PS_SITE_WIDE
    PS_ATTR(12) PS_ATTR(14) PS_ATTR(16)
#else
    PS_ATTR(1) PS_ATTR(2) PS_ATTR(3) PS_ATTR(4) PS_ATTR(5) PS_ATTR(6) PS_ATTR(7) PS_ATTR(8)
#endif
#undef PS_ATTR
    return e;
}

}  // namespace

bool PS_SITE_FN(launch_db_fast)(const float *src, const float *rsrc, float *pdst,
                                CgBand *bands, const CgGlobal *g, int cg, int N, int H, int W,
                                int c, const float *u, int R, float *v, cudaStream_t st,
                                int impl) {
#ifndef PS_SITE_WIDE
    if (R > 8)
        return launch_db_fast_wide(src, rsrc, pdst, bands, g, cg, N, H, W, c, u, R, v, st, impl);
#endif
    return dispatch(c, R, 0, src, rsrc, pdst, bands, g, cg, N, H, W, u, v, nullptr, nullptr,
                    nullptr, st, impl);
}

bool PS_SITE_FN(launch_cg_update_fast)(float *x, float *r, const float *p, const float *q,
                                       const float *v, const float *u, int R, int c, int N,
                                       int H, int W, CgBand *bands, const CgGlobal *g,
                                       cudaStream_t st) {
#ifndef PS_SITE_WIDE
    if (R > 8)
        return launch_cg_update_fast_wide(x, r, p, q, v, u, R, c, N, H, W, bands, g, st);
#endif
    return dispatch(c, R, 1, p, nullptr, nullptr, bands, g, 1, N, H, W, u,
                    const_cast<float *>(v), x, r, q, st);
}

cudaError_t PS_SITE_FN(cg_fast_set_attrs)() {
    cudaError_t e = set_attrs_c<4>();
#ifndef PS_SITE_WIDE
    if (e == cudaSuccess) e = set_attrs_c<2>();
    if (e == cudaSuccess) e = cg_fast_set_attrs_wide();
#endif
    return e;
}

}  // namespace ps
