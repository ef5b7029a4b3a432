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
