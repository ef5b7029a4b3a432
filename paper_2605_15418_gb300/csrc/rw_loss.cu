// A8: normalised least-squares loss of Eq. 3,
//   L = || alpha I - T ||^2,  alpha = <I, T> / <I, I>  (the optimal scale),
// and its gradient dL/dI = 2 alpha (alpha I - T) (alpha held at its optimum,
// where dL/dalpha = 0).  Sums are accumulated in double.
#include "rw_kernels.cuh"

__global__ void k_loss_sums(const float* __restrict__ I, const float* __restrict__ T, long long n,
                            double* __restrict__ acc) {
    double s_it = 0.0, s_ii = 0.0, s_tt = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double a = I[i], b = T[i];
        s_it += a * b; s_ii += a * a; s_tt += b * b;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s_it += __shfl_xor_sync(0xffffffffu, s_it, o);
        s_ii += __shfl_xor_sync(0xffffffffu, s_ii, o);
        s_tt += __shfl_xor_sync(0xffffffffu, s_tt, o);
    }
    __shared__ double red[3][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { red[0][w] = s_it; red[1][w] = s_ii; red[2][w] = s_tt; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a += red[0][k]; b += red[1][k]; c += red[2][k]; }
        atomicAdd(acc + 0, a); atomicAdd(acc + 1, b); atomicAdd(acc + 2, c);
    }
}

__global__ void k_loss_grad(const float* __restrict__ I, const float* __restrict__ T, long long n,
                            const double* __restrict__ acc, double* __restrict__ out,
                            float* __restrict__ g) {
    const double it = acc[0], ii = acc[1], tt = acc[2];
    const double alpha = ii > 0.0 ? it / ii : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && out) {
        out[0] = ii > 0.0 ? tt - it * it / ii : tt;
        out[1] = alpha;
        out[2] = ii;
    }
    if (!g) return;
    const float af = (float)alpha;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        g[i] = 2.f * af * (af * I[i] - T[i]);
}

cudaError_t launch_loss_eq3(const LaunchCtx& L, const float* I, const float* T, long long n,
                            double* acc, double* out, float* g) {
    cudaError_t e = cudaMemsetAsync(acc, 0, 3 * sizeof(double), L.stream);
    if (e != cudaSuccess) return e;
    long long grid = (n + 255) / 256;
    long long cap = (long long)L.num_sms * 4;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    RW_MARK(L, "k_loss_sums");
    k_loss_sums<<<(unsigned)grid, 256, 0, L.stream>>>(I, T, n, acc);
    RW_MARK(L, nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    RW_MARK(L, "k_loss_grad");
    k_loss_grad<<<(unsigned)grid, 256, 0, L.stream>>>(I, T, n, acc, out, g);
    RW_MARK(L, nullptr);
    return cudaGetLastError();
}

// Reduction-throughput probe (the RED ceiling of the adjoint's map scatter):
// `nwin` windows of win x win pixels at pseudo-random offsets of an H x W
// float map, one atomic add per pixel with the result unused, a warp's lanes
// on adjacent pixels of a row -- the access pattern of the patch scatter.
__global__ void k_probe_red(float* __restrict__ map, int H, int W, int win, long long nwin) {
    for (long long wdx = blockIdx.x; wdx < nwin; wdx += gridDim.x) {
        // splitmix-style hash of the window index (integer only)
        unsigned long long z = (unsigned long long)wdx * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const int r0 = (int)((z & 0xffffffffull) % (unsigned long long)(H - win + 1));
        const int c0 = (int)((z >> 32) % (unsigned long long)(W - win + 1));
        for (int f = threadIdx.x; f < win * win; f += blockDim.x) {
            const int b = f / win, a = f - (f / win) * win;
            atomicAdd(map + (long long)(r0 + b) * W + (c0 + a), 1e-3f);
        }
    }
}

cudaError_t launch_probe_red(const LaunchCtx& L, float* map, int H, int W, int win,
                             long long nwin) {
    long long grid = (long long)L.num_sms * 8;
    if (grid > nwin) grid = nwin;
    if (grid < 1) grid = 1;
    RW_MARK(L, "k_probe_red");
    k_probe_red<<<(unsigned)grid, 256, 0, L.stream>>>(map, H, W, win, nwin);
    RW_MARK(L, nullptr);
    return cudaGetLastError();
}
