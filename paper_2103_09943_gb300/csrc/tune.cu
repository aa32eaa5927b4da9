// Table of launch choices picked by the autotuner (ps_autotune in api.cu):
// per device and problem size, the rows per CTA of the preconditioner's row
// passes and the rows per warp of the CG-loop LLP kernel. Launchers read it;
// sizes never tuned get the static defaults.
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace ps {

namespace {

struct Entry {
    int dev, N, H, W, c, r;
    Tuning t;
};
std::mutex g_tune_mu;
std::vector<Entry> g_tune;

}  // namespace

Tuning tuning_get(int dev, int N, int H, int W, int c, int r) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const Entry &e : g_tune)
        if (e.dev == dev && e.N == N && e.H == H && e.W == W && e.c == c && e.r == r) return e.t;
    return Tuning{0, 0, 0, 0, 0, 0, 0, 0};
}

void tuning_set(int dev, int N, int H, int W, int c, int r, const Tuning &t) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (Entry &e : g_tune)
        if (e.dev == dev && e.N == N && e.H == H && e.W == W && e.c == c && e.r == r) {
            e.t = t;
            return;
        }
    g_tune.push_back(Entry{dev, N, H, W, c, r, t});
}

}  // namespace ps

namespace ps {

namespace {
__global__ void fill_kernel(float *p, size_t n, float v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        p[i] = v;
}
}  // namespace

void launch_fill(float *p, size_t n, float v, cudaStream_t st) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    fill_kernel<<<blocks, 256, 0, st>>>(p, n, v);
}

}  // namespace ps
