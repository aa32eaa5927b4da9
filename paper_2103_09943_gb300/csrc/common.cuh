// Shared device helpers of the F-BMP CUDA path (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ps.h"

namespace ps {

constexpr int kMaxR = 16;          // kernel radius: n = 2R + 1 <= 33
constexpr int kMaxTaps = (2 * kMaxR + 1) * (2 * kMaxR + 1);
constexpr int kMaxWinR = 4;        // LLP window radius r <= 4
constexpr int kMaxBands = 64;
constexpr int kMaxFFT = 8192;      // H, W <= 8192
constexpr int kMaxRatio = 8;
constexpr int kMaxSplit = 4;       // parallel branches (own loops) of the CG iteration

// Wrap an index that lies in [-n, 2n) onto [0, n).
__host__ __device__ __forceinline__ int wrapi(int i, int n) {
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

// Per-band CG scalars. FP64: the inner products of the solver are, with the
// PAN statistics and the kernel normal equations, where double precision is
// spent.
struct CgBand {
    double rr;       // r^T r of the current residual
    double bb;       // b^T b
    double pAp;      // accumulator of p^T (lam L^T M L) p (zeroed after use)
    double vv;       // accumulator of ||D B p||^2 = p^T B^T D^T D B p (zeroed after use)
    double rr_new;   // accumulator of the next r^T r (zeroed after use)
    double rho;      // numerator of alpha: r^T r (plain CG) or r^T z (preconditioned)
    double rz_new;   // accumulator of the next r^T z (zeroed after use)
    double xx_new;   // accumulators of ||x_new||^2 and ||p||^2 for the relative-
    double pp_new;   // change stop rule (zeroed after use)
    double alpha;
    double beta;
    int iters;
    int status;      // ps_status
    int done;
    unsigned int cnt_apply;   // CTA arrival counters (last-block pattern)
    unsigned int cnt_update;
    unsigned int cnt_init;
    unsigned int cnt_prec;    // CTAs of the preconditioner's last kernel (per band pair)
    unsigned long long t_start;  // device global timer (ns) when the solve was reset
    unsigned long long t_done;   // ... when the control kernel first saw the band stopped
};

// The device's global nanosecond timer.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    return v;
}

struct CgGlobal {
    double tol;               // relative residual target
    unsigned int cnt_bands;
    int active;               // bands not yet done
    int max_iters;            // max over bands of iters
    int stop;                 // set once the loop must end
    int iter;                 // loop iterations run
    int max_iter;             // hard cap
    int precond;              // 1: z = P^{-1} r feeds p and beta (preconditioned CG)
    int rule;                 // stop rule: 0 ||r|| / ||b|| <= tol; 1 ||x_new - x|| / ||x_new|| < tol
};

// The stop test of a band after an update with step alpha: the relative
// residual, or the relative change ||alpha p|| / ||x_new|| of the iterate
// in the Frobenius norm (the rule the paper states for the Z0 CG, Sec. IV-F).
__device__ __forceinline__ bool cg_converged(const CgGlobal *g, const CgBand *bd, double rn,
                                             double xx, double pp) {
    if (g->rule == 1) return bd->alpha * bd->alpha * pp < g->tol * g->tol * xx;
    return sqrt(rn / bd->bb) <= g->tol;
}

// Block-wide sum of a double over a 1-D block; the result is valid in
// thread 0. `red` holds blockDim.x / 32 doubles of shared memory.
__device__ __forceinline__ double block_sum_d(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int tid = threadIdx.x;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid < 32) {
        s = (tid < nw) ? red[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

}  // namespace ps
