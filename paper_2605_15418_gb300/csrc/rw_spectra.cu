// A3 + A4 on their own: the angular spectrum U~ of every incident ray's
// patch, written to HBM.  Two implementations with identical output:
//
//   k_spectra_fft<M>  FP32 mixed-radix Stockham FFT in shared memory (the
//                     per-ray CUDA-core form used inside the fused kernels),
//                     any supported padded size M = P D;
//   k_spectra_tc      the dense contraction U = F X F^T on the tensor cores
//                     (tcgen05, D = 64 without padding), BF16x3 split with
//                     FP32 accumulation in tensor memory.
//
// Tensor-core form.  A complex product C = A B is one real product
//   [C_re; C_im] = [[A_re, -A_im], [A_im, A_re]] [B_re; B_im],
// so with F[m][k] = exp(-2 pi i m k / D) each stage is one M = K = 2D = 128
// GEMM against a constant 128 x 128 operand:
//   stage 1: Y = F_v X        (A = F_big, B rows n = a, K = (re/im, b))
//   stage 2: Z^T = F_u Y^T    (A = F_big, B rows n = m_v, K = (re/im, a))
// Each real operand v is split v = hi + lo in bf16 and every product is
// A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped lo*lo term is ~2^-16
// relative), accumulated in FP32 in tensor memory.  Stage 1's accumulator
// is read back (tcgen05.ld), re-split and stored transposed as stage 2's B
// operand; stage 2's accumulator is staged through shared memory so the
// spectrum is written coalesced, with the phase factors that refer it to
// the hit point and the normalisation (1/D^2 without padding) applied on the
// way out.
#include <cstring>

#include "rw_kernels.cuh"
#include "rw_tc.cuh"

// ------------------------------------------------------------------ FFT form
template <int M>
__global__ void __launch_bounds__(RW_THREADS, M <= 64 ? 2 : 1)
k_spectra_fft(const DSys sys, const DJob* __restrict__ jobs, const long long* __restrict__ prefix,
              int njob, long long total, RaysIn rays, const float2* __restrict__ Tmaps,
              float2* __restrict__ out, unsigned* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    float2* X = reinterpret_cast<float2*>(smem);
    float2* tw = X + Patch<M>::ELEMS;
    float2* phu = tw + M;
    float2* phv = phu + M;
    RayAtDoe* info = reinterpret_cast<RayAtDoe*>(phv + M);
    fft_twiddles<M>(tw);
    const float norm = sys.norm;
    const long long npix_map = (long long)sys.H * sys.W;
    const long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        if (threadIdx.x < RW_TILE)
            incident_to_doe(sys, jobs, prefix, njob, total, rays, tile * RW_TILE + threadIdx.x,
                            info[threadIdx.x], status);
        __syncthreads();
        for (int r = 0; r < RW_TILE; ++r) {
            const long long g = tile * RW_TILE + r;
            if (g >= total) break;
            const RayAtDoe& R = info[r];
            float2* o = out + g * (long long)(M * M);
            if (!R.alive) {
                for (int f = threadIdx.x; f < M * M; f += RW_THREADS) o[f] = make_float2(0.f, 0.f);
                continue;
            }
            gather_patch<M>(sys, R, Tmaps + (long long)jobs[R.job].slot * npix_map, X, phu, phv);
            __syncthreads();
            fft2d<M, false>(X, tw);
            for (int f = threadIdx.x; f < M * M; f += RW_THREADS) {
                const int jvi = f / M, jui = f - (f / M) * M;
                o[f] = spectrum_at<M>(X, phu, phv, jui, jvi, norm);
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------ tensor-core form
#define RW_TC_WAIT (1ll << 26)   // polls of an mbarrier before the kernel gives up

namespace tcdft {
constexpr int D = 64, M = 2 * D, K = 2 * D, N = D;
constexpr uint32_t TILE_A = M * K * 2;          // 32 KB per bf16 plane
constexpr uint32_t TILE_B = N * K * 2;          // 16 KB per bf16 plane
constexpr uint32_t OFF_AHI = 0, OFF_ALO = TILE_A, OFF_B = 2 * TILE_A;
constexpr uint32_t OFF_BHI = OFF_B, OFF_BLO = OFF_B + TILE_B;   // staging S aliases [OFF_B, +32 KB)
constexpr uint32_t OFF_PH = OFF_B + 2 * TILE_B;
constexpr uint32_t OFF_INFO = OFF_PH + 2 * D * sizeof(float2);
constexpr uint32_t OFF_BAR = OFF_INFO + RW_TILE * sizeof(RayAtDoe);
constexpr uint32_t SMEM = OFF_BAR + 64;
constexpr uint32_t TMEM_COLS = 2 * N;           // stage-1 and stage-2 accumulators
constexpr uint32_t IDESC = tc_idesc_bf16(M, N);
static_assert(D * D * sizeof(float2) <= 2 * TILE_B, "staging must fit the B region");
}  // namespace tcdft

// Issue one stage: D[tmem] = A_hi B_hi + A_hi B_lo + A_lo B_hi over K, with
// A hi / lo at a, a + TILE_A and B hi / lo at b, b + TILE_B.
__device__ __forceinline__ void tc_issue_stage_at(const unsigned char* a, const unsigned char* b,
                                                  uint32_t d_tmem) {
    using namespace tcdft;
    const uint32_t a_hi = smem_addr(a), a_lo = smem_addr(a + TILE_A);
    const uint32_t b_hi = smem_addr(b), b_lo = smem_addr(b + TILE_B);
    const uint32_t sbo = 16 * K;
#pragma unroll
    for (int s = 0; s < K / 16; ++s) {
        const uint32_t ks = 256u * s;                 // two core matrices along K
        tc_mma_bf16(d_tmem, tc_smem_desc(a_hi + ks, 128, sbo), tc_smem_desc(b_hi + ks, 128, sbo),
                    IDESC, s > 0);
        tc_mma_bf16(d_tmem, tc_smem_desc(a_hi + ks, 128, sbo), tc_smem_desc(b_lo + ks, 128, sbo),
                    IDESC, 1);
        tc_mma_bf16(d_tmem, tc_smem_desc(a_lo + ks, 128, sbo), tc_smem_desc(b_hi + ks, 128, sbo),
                    IDESC, 1);
    }
}

__device__ __forceinline__ void tc_issue_stage(unsigned char* smem, uint32_t d_tmem) {
    tc_issue_stage_at(smem + tcdft::OFF_AHI, smem + tcdft::OFF_BHI, d_tmem);
}

__device__ __forceinline__ void put_bf16(unsigned char* base, uint32_t off, __nv_bfloat16 v) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = v;
}

__global__ void __launch_bounds__(RW_THREADS, 2)
k_spectra_tc(const DSys sys, const DJob* __restrict__ jobs, const long long* __restrict__ prefix,
             int njob, long long total, RaysIn rays, const float2* __restrict__ Tmaps,
             float2* __restrict__ out, unsigned* status) {
    using namespace tcdft;
    extern __shared__ __align__(1024) unsigned char smem[];
    float2* S = reinterpret_cast<float2*>(smem + OFF_B);
    float2* phu = reinterpret_cast<float2*>(smem + OFF_PH);
    float2* phv = phu + D;
    RayAtDoe* info = reinterpret_cast<RayAtDoe*>(smem + OFF_INFO);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + OFF_BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + OFF_BAR + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // ---- constant operand: F_big = [[F_re, -F_im], [F_im, F_re]], split in bf16
    for (int i = tid; i < M * K; i += RW_THREADS) {
        const int r = i / K, k = i - (i / K) * K;
        const int po = r / D, m = r - po * D, pi = k / D, kk = k - pi * D;
        float s, c;
        sincospif(2.f * (float)((m * kk) % D) / (float)D, &s, &c);   // F = c - i s
        const float v = (po == pi) ? c : (po == 0 ? s : -s);
        __nv_bfloat16 hi, lo;
        bf16_split(v, hi, lo);
        const uint32_t off = kmajor_off(r, k, K);
        put_bf16(smem + OFF_AHI, off, hi);
        put_bf16(smem + OFF_ALO, off, lo);
    }
    if (tid == 0) mbar_init(bar, 1);
    if (warp == 0) tmem_alloc(tslot, TMEM_COLS);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t d1 = tmem, d2 = tmem + N;
    const int q = warp & 3;                      // TMEM lane quarter of this warp
    const int row = q * 32 + lane;               // accumulator row = TMEM lane
    const int cbase = (warp >> 2) * (N / 2);     // this warp's half of the columns
    const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
    uint32_t parity = 0;
    bool failed = false;
    const long long npix_map = (long long)sys.H * sys.W;
    const long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    for (long long tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
        __syncthreads();
        if (tid < RW_TILE)
            incident_to_doe(sys, jobs, prefix, njob, total, rays, tile * RW_TILE + tid, info[tid],
                            status);
        __syncthreads();
        for (int r = 0; r < RW_TILE; ++r) {
            const long long g = tile * RW_TILE + r;
            if (g >= total) break;
            const RayAtDoe& R = info[r];
            float2* o = out + g * (long long)(D * D);
            if (!R.alive) {
                for (int f = tid; f < D * D; f += RW_THREADS) o[f] = make_float2(0.f, 0.f);
                continue;
            }
            // ---- A3: patch -> B (rows n = a, K = (re/im, b)), complex split to bf16 hi/lo
            const float2* T = Tmaps + (long long)jobs[R.job].slot * npix_map;
            for (int f = tid; f < D * D; f += RW_THREADS) {
                const int b = f / D, a = f - (f / D) * D;
                float2 t;
                if (sys.gather == RW_GATHER_NEAREST) {
                    t = tmap(T, sys.H, sys.W, R.r0 + b, R.c0 + a);
                } else {
                    const float oa = (float)(a - D / 2), ob = (float)(b - D / 2);
                    const float fu = R.s0 + oa * R.u[0] + ob * R.v[0];
                    const float fv = R.t0 + oa * R.u[1] + ob * R.v[1];
                    const float iuf = floorf(fu), ivf = floorf(fv);
                    const float wu = fu - iuf, wv = fv - ivf;
                    const int i0 = R.c0 + (int)iuf, j0 = R.r0 + (int)ivf;
                    const float2 t00 = tmap(T, sys.H, sys.W, j0, i0), t10 = tmap(T, sys.H, sys.W, j0, i0 + 1);
                    const float2 t01 = tmap(T, sys.H, sys.W, j0 + 1, i0), t11 = tmap(T, sys.H, sys.W, j0 + 1, i0 + 1);
                    const float w00 = (1.f - wu) * (1.f - wv), w10 = wu * (1.f - wv);
                    const float w01 = (1.f - wu) * wv, w11 = wu * wv;
                    t = make_float2(w00 * t00.x + w10 * t10.x + w01 * t01.x + w11 * t11.x,
                                    w00 * t00.y + w10 * t10.y + w01 * t01.y + w11 * t11.y);
                }
                __nv_bfloat16 hi, lo;
                bf16_split(t.x, hi, lo);
                put_bf16(smem + OFF_BHI, kmajor_off(a, b, K), hi);
                put_bf16(smem + OFF_BLO, kmajor_off(a, b, K), lo);
                bf16_split(t.y, hi, lo);
                put_bf16(smem + OFF_BHI, kmajor_off(a, D + b, K), hi);
                put_bf16(smem + OFF_BLO, kmajor_off(a, D + b, K), lo);
            }
            if (tid < D) {
                const float j = (float)(tid - D / 2);
                float s, c;
                if (sys.gather == RW_GATHER_NEAREST) {
                    sincospif(-2.f * j * R.s0, &s, &c);
                    phu[tid] = make_float2(c, s);
                    sincospif(-2.f * j * R.t0, &s, &c);
                    phv[tid] = make_float2(c, s);
                } else {
                    const float sg = (((tid - D / 2) & 1) ? -1.f : 1.f);
                    phu[tid] = make_float2(sg, 0.f);
                    phv[tid] = make_float2(sg, 0.f);
                }
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            // ---- stage 1: Y = F X
            if (tid == 0) {
                tc_issue_stage(smem, d1);
                tc_commit(bar);
            }
            bool ok = mbar_wait_bounded(bar, parity, RW_TC_WAIT);
            parity ^= 1u;
            if (__syncthreads_or(!ok)) { failed = true; break; }
            tc_fence_after();
            // ---- Y (TMEM rows (re/im, m_v), columns a) -> B rows n = m_v, K = (re/im, a)
            {
                const int p = row / D, mv = row - (row / D) * D;
#pragma unroll
                for (int cc = 0; cc < N / 2; cc += 16) {
                    float v[16];
                    tmem_ld16(d1 + lane_addr + (uint32_t)(cbase + cc), v);
#pragma unroll
                    for (int j = 0; j < 16; j += 8) {
                        __align__(16) __nv_bfloat16 hi8[8], lo8[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) bf16_split(v[j + e], hi8[e], lo8[e]);
                        const uint32_t off = kmajor_off(mv, p * D + cbase + cc + j, K);
                        *reinterpret_cast<uint4*>(smem + OFF_BHI + off) = *reinterpret_cast<uint4*>(hi8);
                        *reinterpret_cast<uint4*>(smem + OFF_BLO + off) = *reinterpret_cast<uint4*>(lo8);
                    }
                }
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            // ---- stage 2: Z^T = F Y^T
            if (tid == 0) {
                tc_issue_stage(smem, d2);
                tc_commit(bar);
            }
            ok = mbar_wait_bounded(bar, parity, RW_TC_WAIT);
            parity ^= 1u;
            if (__syncthreads_or(!ok)) { failed = true; break; }
            tc_fence_after();
            // ---- Z^T (rows (re/im, m_u), columns m_v) -> S[m_v][m_u]
            {
                const int p = row / D, mu = row - (row / D) * D;
                float* Sf = reinterpret_cast<float*>(S);
#pragma unroll
                for (int cc = 0; cc < N / 2; cc += 16) {
                    float v[16];
                    tmem_ld16(d2 + lane_addr + (uint32_t)(cbase + cc), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) Sf[2 * ((cbase + cc + j) * D + mu) + p] = v[j];
                }
            }
            tc_fence_before();
            __syncthreads();
            // ---- U~ = Z (natural order) * phases / D^2, coalesced
            for (int f = tid; f < D * D; f += RW_THREADS) {
                const int jvi = f / D, jui = f - (f / D) * D;
                o[f] = spectrum_at<D, D>(S, phu, phv, jui, jvi, sys.norm);
            }
            __syncthreads();
        }
    }
    if (failed) {
        if (tid == 0) atomicOr(status, RW_ST_TIMEOUT);
        // let any MMA still in flight finish before the tensor memory is released
        mbar_wait_bounded(bar, parity ^ 1u, RW_TC_WAIT);   // the phase that timed out
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// ------------------------------------------------------------------ launchers
template <int M>
static cudaError_t launch_spectra_fft_d(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                                        const long long* prefix, int njob, long long total,
                                        const RaysIn& rays, const float2* T, float2* out,
                                        unsigned* status) {
    const size_t smem = forward_smem_bytes(M);
    auto kern = k_spectra_fft<M>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RW_THREADS, smem);
    if (e != cudaSuccess) return e;
    long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    long long grid = (long long)L.num_sms * (per_sm > 0 ? per_sm : 1);
    grid = pick_grid(L, RW_K_SPECTRA, grid);
    if (grid > ntiles) grid = ntiles;
    RW_MARK(L, "k_spectra_fft");
    kern<<<(unsigned)grid, RW_THREADS, smem, L.stream>>>(sys, jobs, prefix, njob, total, rays, T,
                                                          out, status);
    RW_MARK(L, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_spectra(const LaunchCtx& L, const DSys& sys, int tc, const DJob* jobs,
                           const long long* prefix, int njob, long long total, const RaysIn& rays,
                           const float2* T, float2* out, unsigned* status) {
    if (tc) {
        if (sys.D != tcdft::D || sys.M != tcdft::D) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(k_spectra_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)tcdft::SMEM);
        if (e != cudaSuccess) return e;
        long long ntiles = (total + RW_TILE - 1) / RW_TILE;
        long long grid = (long long)L.num_sms * 2;
        grid = pick_grid(L, RW_K_SPECTRA, grid);
        if (grid > ntiles) grid = ntiles;
        RW_MARK(L, "k_spectra_tc");
        k_spectra_tc<<<(unsigned)grid, RW_THREADS, tcdft::SMEM, L.stream>>>(
            sys, jobs, prefix, njob, total, rays, T, out, status);
        RW_MARK(L, nullptr);
        return cudaGetLastError();
    }
    switch (sys.M) {
        case 16: return launch_spectra_fft_d<16>(L, sys, jobs, prefix, njob, total, rays, T, out, status);
        case 32: return launch_spectra_fft_d<32>(L, sys, jobs, prefix, njob, total, rays, T, out, status);
        case 64: return launch_spectra_fft_d<64>(L, sys, jobs, prefix, njob, total, rays, T, out, status);
        case 96: return launch_spectra_fft_d<96>(L, sys, jobs, prefix, njob, total, rays, T, out, status);
        case 128: return launch_spectra_fft_d<128>(L, sys, jobs, prefix, njob, total, rays, T, out, status);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ fused forward, tensor cores
// The incoherent exhaustive forward of rw_forward / rw_forward_vis with the
// patch transform on the tensor cores (D = 64, no padding): per incident ray
// the patch is gathered straight into the bf16 hi/lo B operand, the two
// stages of k_spectra_tc run, and stage 2's accumulator is read back from
// tensor memory into the shared spectrum buffer X in the layout the FFT path
// leaves (row stride 65, FFT order), so that block culling, emission, the
// sensor splat, the visibility mask and the adjoint's tape are the FFT path's
// own.  One CTA per SM (the constant operand takes 64 KB of shared memory).
namespace tcfwd {
using namespace tcdft;
// Two groups of RW_THREADS threads per CTA share the constant operand and the
// tensor core; each group runs its own tiles of rays with its own operand,
// spectrum and scratch, so that one group's gather, conversions and
// emission overlap the other's MMAs and memory latency.
constexpr int NGRP = 2;
constexpr uint32_t X_BYTES = (uint32_t)(Patch<D>::ELEMS * sizeof(float2));
constexpr uint32_t G_B = 0;                                   // B hi, then B lo
constexpr uint32_t G_X = 2 * TILE_B;
constexpr uint32_t G_PH = G_X + X_BYTES;
constexpr uint32_t G_INFO = G_PH + 2 * D * sizeof(float2);
constexpr uint32_t G_VW = (uint32_t)((G_INFO + RW_TILE * sizeof(RayAtDoe) + 15) & ~15u);
constexpr uint32_t G_KEEP = (uint32_t)(G_VW + cull_scratch_bytes(D));
constexpr uint32_t G_BAR = G_KEEP + RW_TILE * 2 * sizeof(unsigned);
constexpr uint32_t G_BYTES = (G_BAR + 16 + 1023) & ~1023u;
constexpr uint32_t OFF_G = 2 * TILE_A;                        // after A hi, A lo
constexpr uint32_t OFF_SLOT = OFF_G + NGRP * G_BYTES;
constexpr uint32_t SMEM = OFF_SLOT + 16;
constexpr uint32_t COLS = NGRP * 2 * N;                       // two accumulators per group
static_assert(SMEM <= 227 * 1024, "shared memory of the two-group tensor-core forward");
}  // namespace tcfwd

// A3 for the tensor-core forward: patch sample (a, b) of ray R (nearest or
// bilinear, as gather_patch) for rows b0 .. b0+7 of column a, split into
// bf16 hi / lo and stored as the 16-byte K runs of the stage-1 operand
// (row n = a, K = (re/im, b)).
__device__ __forceinline__ void tc_gather8(const DSys& sys, const RayAtDoe& R,
                                           const float2* __restrict__ T, int a, int b0,
                                           unsigned char* B) {
    using namespace tcdft;
    __align__(16) __nv_bfloat16 hr[8], lr[8], hi_[8], li[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int b = b0 + j;
        float2 t;
        if (sys.gather == RW_GATHER_NEAREST) {
            t = tmap(T, sys.H, sys.W, R.r0 + b, R.c0 + a);
        } else {
            const float oa = (float)(a - D / 2), ob = (float)(b - D / 2);
            const float fu = R.s0 + oa * R.u[0] + ob * R.v[0];
            const float fv = R.t0 + oa * R.u[1] + ob * R.v[1];
            const float iuf = floorf(fu), ivf = floorf(fv);
            const float wu = fu - iuf, wv = fv - ivf;
            const int i0 = R.c0 + (int)iuf, j0 = R.r0 + (int)ivf;
            const float2 t00 = tmap(T, sys.H, sys.W, j0, i0), t10 = tmap(T, sys.H, sys.W, j0, i0 + 1);
            const float2 t01 = tmap(T, sys.H, sys.W, j0 + 1, i0), t11 = tmap(T, sys.H, sys.W, j0 + 1, i0 + 1);
            const float w00 = (1.f - wu) * (1.f - wv), w10 = wu * (1.f - wv);
            const float w01 = (1.f - wu) * wv, w11 = wu * wv;
            t = make_float2(w00 * t00.x + w10 * t10.x + w01 * t01.x + w11 * t11.x,
                            w00 * t00.y + w10 * t10.y + w01 * t01.y + w11 * t11.y);
        }
        bf16_split(t.x, hr[j], lr[j]);
        bf16_split(t.y, hi_[j], li[j]);
    }
    const uint32_t ore = kmajor_off(a, b0, K), oim = kmajor_off(a, D + b0, K);
    *reinterpret_cast<uint4*>(B + ore) = *reinterpret_cast<const uint4*>(hr);
    *reinterpret_cast<uint4*>(B + TILE_B + ore) = *reinterpret_cast<const uint4*>(lr);
    *reinterpret_cast<uint4*>(B + oim) = *reinterpret_cast<const uint4*>(hi_);
    *reinterpret_cast<uint4*>(B + TILE_B + oim) = *reinterpret_cast<const uint4*>(li);
}

// The fused forward with the tensor-core patch transform (D = 64, no
// padding, exhaustive emission, incoherent sensor): per incident ray the
// patch is gathered into the stage-1 operand, U = F X F^T is formed on the
// tensor cores (BF16x3, FP32 accumulation in tensor memory), the spectrum
// lands in shared memory in the FFT's layout, and the FFT path's emission
// (culled blocks, mask, tape) runs on it unchanged.  Every wait on the
// tensor core is bounded: on a timeout the status word gets RW_ST_TIMEOUT
// and the group stops.
template <int NS>
__global__ void __launch_bounds__(tcfwd::NGRP * RW_THREADS, 1)
k_forward_tc(const DSys sys, const DJob* __restrict__ jobs, const long long* __restrict__ prefix,
             int njob, long long total, RaysIn rays, const float2* __restrict__ Tmaps,
             double* __restrict__ psf, unsigned* status, unsigned* __restrict__ vis,
             const unsigned* __restrict__ keep, SplitBufs tape) {
    using namespace tcfwd;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int grp = threadIdx.x / RW_THREADS, lt = ltid(), lwarp = lt >> 5, lane = lt & 31;
    unsigned char* gb = smem + OFF_G + grp * G_BYTES;
    unsigned char* B = gb + G_B;
    float2* X = reinterpret_cast<float2*>(gb + G_X);
    float2* phu = reinterpret_cast<float2*>(gb + G_PH);
    float2* phv = phu + D;
    RayAtDoe* info = reinterpret_cast<RayAtDoe*>(gb + G_INFO);
    unsigned* vw = reinterpret_cast<unsigned*>(gb + G_VW);
    unsigned* skeep = reinterpret_cast<unsigned*>(gb + G_KEEP);
    uint64_t* bar = reinterpret_cast<uint64_t*>(gb + G_BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + OFF_SLOT);
    if (tape.epoch && blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long e = atomicAdd(tape.epoch, 1ull) + 1ull;
        if (tape.iray) tape.epoch[1] = e;
    }
    if (vis)
        for (int i = lt; i < D * D / 32; i += RW_THREADS) vw[i] = 0u;
    // ---- constant operand: F_big = [[F_re, -F_im], [F_im, F_re]], split in bf16
    for (int i = threadIdx.x; i < M * K; i += NGRP * RW_THREADS) {
        const int r = i / K, k = i - (i / K) * K;
        const int po = r / D, m = r - po * D, pi = k / D, kk = k - pi * D;
        float sn, cs;
        sincospif(2.f * (float)((m * kk) % D) / (float)D, &sn, &cs);   // F = c - i s
        const float v = (po == pi) ? cs : (po == 0 ? sn : -sn);
        __nv_bfloat16 hi, lo;
        bf16_split(v, hi, lo);
        const uint32_t off = kmajor_off(r, k, K);
        put_bf16(smem + OFF_AHI, off, hi);
        put_bf16(smem + OFF_ALO, off, lo);
    }
    if (lt == 0) mbar_init(bar, 1);
    if (threadIdx.x < 32) tmem_alloc(tslot, COLS);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t d1 = tmem + (uint32_t)(grp * 2 * N), d2 = d1 + N;
    const int q = lwarp & 3;                     // TMEM lane quarter of this warp
    const int row = q * 32 + lane;               // accumulator row = TMEM lane
    const int cbase = (lwarp >> 2) * (N / 2);    // this warp's half of the columns
    const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
    uint32_t parity = 0;
    bool failed = false;
    const long long npix_map = (long long)sys.H * sys.W;
    const long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    for (long long tile = (long long)blockIdx.x * NGRP + grp; tile < ntiles && !failed;
         tile += (long long)gridDim.x * NGRP) {
        main_sync();
        if (lt < RW_TILE) {
            const long long g = tile * RW_TILE + lt;
            incident_to_doe(sys, jobs, prefix, njob, total, rays, g, info[lt], status);
            if (tape.rinfo && g < total) tape.rinfo[g] = info[lt];
        }
        if (keep) {
            constexpr int KW = cull_keep_words(D);
            const long long w0 = tile * RW_TILE * KW;
            if (lt < RW_TILE * KW && KW <= 2)
                skeep[lt] = (w0 + lt < total * KW) ? __ldg(keep + w0 + lt) : 0u;
        }
        main_sync();
        for (int r = 0; r < RW_TILE; ++r) {
            const long long g = tile * RW_TILE + r;
            const RayAtDoe& R = info[r];
            if (!R.alive) {
                if (vis && g < total)
                    for (int f = lt; f < D * D / 32; f += RW_THREADS)
                        vis[g * (long long)(D * D / 32) + f] = 0u;
                continue;
            }
            const DJob& J = jobs[R.job];
            const float2* T = Tmaps + (long long)J.slot * npix_map;
            // ---- A3: patch -> stage-1 operand, eight rows of one column per item
            for (int it = lt; it < D * (D / 8); it += RW_THREADS)
                tc_gather8(sys, R, T, it & (D - 1), 8 * (it / D), B);
            phase_factors<D>(sys, R, phu, phv);
            fence_async_smem();
            tc_fence_before();
            main_sync();
            tc_fence_after();
            // ---- A4 stage 1: Y = F X
            if (lt == 0) {
                tc_issue_stage_at(smem + OFF_AHI, B, d1);
                tc_commit(bar);
            }
            bool ok = mbar_wait_bounded(bar, parity, RW_TC_WAIT);
            parity ^= 1u;
            if (group_or(!ok)) { failed = true; break; }
            tc_fence_after();
            // ---- Y (TMEM rows (re/im, m_v), columns a) -> B rows n = m_v, K = (re/im, a)
            {
                const int p = row / D, mv = row - (row / D) * D;
#pragma unroll
                for (int cc = 0; cc < N / 2; cc += 16) {
                    float v[16];
                    tmem_ld16(d1 + lane_addr + (uint32_t)(cbase + cc), v);
#pragma unroll
                    for (int j = 0; j < 16; j += 8) {
                        __align__(16) __nv_bfloat16 hi8[8], lo8[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) bf16_split(v[j + e], hi8[e], lo8[e]);
                        const uint32_t off = kmajor_off(mv, p * D + cbase + cc + j, K);
                        *reinterpret_cast<uint4*>(B + off) = *reinterpret_cast<uint4*>(hi8);
                        *reinterpret_cast<uint4*>(B + TILE_B + off) = *reinterpret_cast<uint4*>(lo8);
                    }
                }
            }
            fence_async_smem();
            tc_fence_before();
            main_sync();
            tc_fence_after();
            // ---- stage 2: Z^T = F Y^T
            if (lt == 0) {
                tc_issue_stage_at(smem + OFF_AHI, B, d2);
                tc_commit(bar);
            }
            ok = mbar_wait_bounded(bar, parity, RW_TC_WAIT);
            parity ^= 1u;
            if (group_or(!ok)) { failed = true; break; }
            tc_fence_after();
            // ---- Z^T (rows (re/im, m_u), columns m_v) -> X[m_v][m_u], row stride D + 1
            {
                const int p = row / D, mu = row - (row / D) * D;
                float* Xf = reinterpret_cast<float*>(X);
#pragma unroll
                for (int cc = 0; cc < N / 2; cc += 16) {
                    float v[16];
                    tmem_ld16(d2 + lane_addr + (uint32_t)(cbase + cc), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        Xf[2 * ((cbase + cc + j) * Patch<D>::S + mu) + p] = v[j];
                }
            }
            tc_fence_before();
            main_sync();
            // ---- A5..A7: the FFT path's emission on the same spectrum
            emit_exhaustive<D, MODE_SPLAT, NS>(sys, J, R, X, phu, phv, psf, nullptr, EmitOut{},
                                               g, status, vis,
                                               keep ? skeep + r * cull_keep_words(D) : nullptr,
                                               vw, tape);
            main_sync();
        }
    }
    if (failed) {
        if (lt == 0) atomicOr(status, RW_ST_TIMEOUT);
        // let the group's MMA still in flight finish before the tensor memory is released
        mbar_wait_bounded(bar, parity ^ 1u, RW_TC_WAIT);   // the phase that timed out
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(tmem, COLS);
}

template <int NS>
static cudaError_t launch_forward_tc_d(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                                       const long long* prefix, int njob, long long total,
                                       const RaysIn& rays, const float2* T, double* psf,
                                       unsigned* status, unsigned* vis, unsigned* keep,
                                       const SplitBufs* tapep) {
    SplitBufs tape;
    std::memset(&tape, 0, sizeof(tape));
    if (keep) {
        cudaError_t e = launch_cull(L, sys, jobs, prefix, njob, total, rays, keep, status);
        if (e != cudaSuccess) return e;
        if (tapep && vis) tape = *tapep;
    } else if (tapep && vis) {
        tape = *tapep;
        tape.iray = nullptr;                    // only the culled path tapes
    }
    auto kern = k_forward_tc<NS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tcfwd::SMEM);
    if (e != cudaSuccess) return e;
    const long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    const long long units = (ntiles + tcfwd::NGRP - 1) / tcfwd::NGRP;   // tiles per CTA step
    long long grid = pick_grid(L, RW_K_FORWARD, (long long)L.num_sms);
    if (grid > units) grid = units;
    if (grid < 1) grid = 1;
    RW_MARK(L, "k_forward_tc");
    kern<<<(unsigned)grid, tcfwd::NGRP * RW_THREADS, tcfwd::SMEM, L.stream>>>(
        sys, jobs, prefix, njob, total, rays, T, psf, status, vis, keep, tape);
    RW_MARK(L, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_forward_tc(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                              const long long* prefix, int njob, long long total,
                              const RaysIn& rays, const float2* T, double* psf, unsigned* status,
                              unsigned* vis, unsigned* keep, const SplitBufs* tape) {
    if (sys.M != tcdft::D || sys.D != tcdft::D) return cudaErrorInvalidValue;
    if (sys.fast_ok) {
        switch (sys.n_post) {
            case 0: return launch_forward_tc_d<0>(L, sys, jobs, prefix, njob, total, rays, T, psf, status, vis, keep, tape);
            case 2: return launch_forward_tc_d<2>(L, sys, jobs, prefix, njob, total, rays, T, psf, status, vis, keep, tape);
            case 4: return launch_forward_tc_d<4>(L, sys, jobs, prefix, njob, total, rays, T, psf, status, vis, keep, tape);
            case 6: return launch_forward_tc_d<6>(L, sys, jobs, prefix, njob, total, rays, T, psf, status, vis, keep, tape);
            default: break;
        }
    }
    return launch_forward_tc_d<-1>(L, sys, jobs, prefix, njob, total, rays, T, psf, status, vis,
                                   nullptr, tape);
}
