// Forward kernels of the ray-wave path: transmission maps (A3 input), ray
// generation (A0), and the fused per-incident-ray pipeline
//   incident trace (A1) -> DOE hit + frame (A2) -> patch gather (A3)
//   -> FP32 2D FFT in shared memory (A4) -> secondary rays (A5)
//   -> downstream trace (A6) -> sensor splat (A7) or HBM write (emit).
//
// One CTA of 256 threads owns one incident ray at a time: warp 0 first
// traces a tile of 32 incident rays to the DOE, then the CTA walks the tile,
// each thread handling M^2/256 spectral bins of the current ray (M = P D,
// the zero-padded transform size; the template parameter).
#include <cstring>

#include "rw_kernels.cuh"

// ------------------------------------------------------------- A3 input
// T_slot[r][c] = A[r][c] exp(i phi[r][c] scale_slot): one complex map per
// wavelength, so the per-patch gather is a plain 8-byte load.
__global__ void k_prep_maps(const float* __restrict__ phi, const float* __restrict__ phi2,
                            const float* __restrict__ amp, int64_t npix,
                            const float* __restrict__ scales, int nslot,
                            float2* __restrict__ T) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix * nslot;
         i += (int64_t)gridDim.x * blockDim.x) {
        int slot = (int)(i / npix);
        int64_t p = i - (int64_t)slot * npix;
        float ph = phi[p] * scales[slot];
        float s, c;
        sincosf(ph, &s, &c);
        if (phi2) {
            // two superposed phase profiles: exp(i phi) + exp(i phi2)
            float s2, c2;
            sincosf(phi2[p] * scales[slot], &s2, &c2);
            c += c2;
            s += s2;
        }
        float A = amp ? amp[p] : 1.f;
        T[i] = make_float2(A * c, A * s);
    }
}

// ------------------------------------------------------------- A0
// Collimated grid per job.  Positions in double without FMA contraction,
// rounded once to float, so they equal the host-side definition exactly.
__global__ void k_generate_rays(const GenJob* __restrict__ jobs, const long long* __restrict__ prefix,
                                int njob, long long total, double z_start, double n_object,
                                RaysOut out) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        int j = find_job(prefix, njob, g);
        const GenJob J = jobs[j];
        long long l = g - prefix[j];
        long long ix = l % J.n, iy = l / J.n;
        double half = __dmul_rn((double)(J.n - 1), 0.5);
        double x = __dadd_rn(J.x0, __dmul_rn(__dadd_rn((double)ix, -half), J.spacing));
        double y = __dadd_rn(J.y0, __dmul_rn(__dadd_rn((double)iy, -half), J.spacing));
        float xf = (float)x, yf = (float)y, zf = (float)z_start;
        long long r = J.off + l;
        out.ox[r] = xf; out.oy[r] = yf; out.oz[r] = zf;
        out.dx[r] = J.dx; out.dy[r] = J.dy; out.dz[r] = J.dz;
        out.are[r] = 1.f; out.aim[r] = 0.f;
        double dot = __dadd_rn(__dadd_rn(__dmul_rn((double)J.dx, (double)xf),
                                         __dmul_rn((double)J.dy, (double)yf)),
                               __dmul_rn((double)J.dz, (double)zf));
        out.opl[r] = __dmul_rn(n_object, dot);
    }
}

// ------------------------------------------------------------- fused forward
// Resident CTAs per SM the register allocation is sized for (M >= 96 needs
// more registers for its FFT stages and more shared memory per CTA).
template <int M>
struct FwdOcc { static constexpr int value = M <= 64 ? 4 : 1; };

// Helper warps of the sampled forward: threads RW_THREADS.. of the block.
// They walk the same tiles and rays as the main threads, meet them at the
// CTA barriers (tile start, and around the draws of every live ray) and make
// their share of the draws -- the (draw, bin) Philox screening that is
// nearly all of the sampled forward's work; the rest stays with the main
// threads.
template <int M>
__device__ __noinline__ void sampled_draw_helpers(const DSys& sys, long long total,
                                                  const RayAtDoe* info, unsigned char* scratch) {
    const float* p = reinterpret_cast<const float*>(scratch);
    const uint4* thr4 = reinterpret_cast<const uint4*>(p + M * M);
    int* sel = reinterpret_cast<int*>(scratch + 8 * (size_t)M * M);
    unsigned char* qmem = scratch + sampled_queue_offset(M, sys.n_ssr);
    const uint32_t k0 = (uint32_t)(sys.seed & 0xffffffffull), k1 = (uint32_t)(sys.seed >> 32);
    const long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();                     // CTA: tile start
        __syncthreads();                     // CTA: the tile's rays are at the DOE
        for (int r = 0; r < RW_TILE; ++r) {
            if (!info[r].alive) continue;
            __syncthreads();                 // CTA: p_j and the thresholds ready
            gumbel_draws<M, RW_GQ_HELPED>(p, thr4, sel, 0, sys.n_ssr, (uint32_t)info[r].rid,
                                          (uint32_t)sys.rng_offset, k0, k1, qmem);
            __syncthreads();                 // CTA: draws done
        }
    }
}

// HW helper warps (sampled emission into the incoherent image only, see
// sampled_draw_helpers); HW = 0 is the plain kernel.
template <int M, int MODE, int NS, int HW = 0>
__global__ void __launch_bounds__(RW_THREADS + 32 * HW, FwdOcc<M>::value)
k_forward(const DSys sys, const DJob* __restrict__ jobs, const long long* __restrict__ prefix,
          int njob, long long total, RaysIn rays, const float2* __restrict__ Tmaps,
          double* __restrict__ psf, float2* __restrict__ field, EmitOut eo, unsigned* status,
          unsigned* __restrict__ vis, const unsigned* __restrict__ keep, SplitBufs tape) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2* X = reinterpret_cast<float2*>(smem);
    float2* tw = X + Patch<M>::ELEMS;
    float2* phu = tw + M;
    float2* phv = phu + M;
    RayAtDoe* info = reinterpret_cast<RayAtDoe*>(phv + M);
    if constexpr (HW > 0) {
        if (threadIdx.x >= RW_THREADS) {
            sampled_draw_helpers<M>(sys, total, info, smem + sampled_scratch_offset(M));
            return;
        }
    }
    // exhaustive emission with block culling: visibility words of the ray
    unsigned* vw = reinterpret_cast<unsigned*>(smem + sampled_scratch_offset(M));
    if (tape.epoch && blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long e = atomicAdd(tape.epoch, 1ull) + 1ull;
        if (tape.iray) tape.epoch[1] = e;
    }
    __shared__ unsigned skeep[RW_TILE * 2];        // the tile's kept-block words (M <= 64)
    if (vis)
        for (int i = threadIdx.x; i < M * M / 32; i += RW_THREADS) vw[i] = 0u;
    __shared__ __align__(8) uint64_t bulk_bar;     // completion of the patch row copies
    uint32_t bulk_phase = 0;
    if (M == 64 && threadIdx.x == 0) mbar_init(&bulk_bar, 1);
    fft_twiddles<M>(tw);
    const long long npix_map = (long long)sys.H * sys.W;
    const long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    // work unit = (tile, slice of each ray's bins); one slice outside coherent launches
    const int nslice = (MODE == MODE_COHERENT && sys.nslice > 1) ? sys.nslice : 1;
    // a slice is a range of bins (exhaustive) or of draws (sampled), in chunks of RW_THREADS
    const int nwork = (MODE == MODE_COHERENT && sys.emit != RW_EMIT_EXHAUSTIVE) ? sys.n_ssr : M * M;
    const int CH = (nwork + RW_THREADS - 1) / RW_THREADS;
    const int per = (MODE == MODE_COHERENT) ? ((CH + nslice - 1) / nslice) * RW_THREADS : M * M;
    for (long long unit = blockIdx.x; unit < ntiles * nslice; unit += gridDim.x) {
        const long long tile = (MODE == MODE_COHERENT) ? unit / nslice : unit;
        const int f0 = (MODE == MODE_COHERENT) ? (int)(unit - tile * nslice) * per : 0;
        const int f1 = (MODE == MODE_COHERENT) ? min(nwork, f0 + per) : M * M;
        __syncthreads();                                           // CTA
        if (threadIdx.x < RW_TILE) {
            const long long g = tile * RW_TILE + threadIdx.x;
            incident_to_doe(sys, jobs, prefix, njob, total, rays, g, info[threadIdx.x], status);
            if (tape.rinfo && g < total) tape.rinfo[g] = info[threadIdx.x];
        }
        if (keep) {
            constexpr int KW = cull_keep_words(M);
            const long long w0 = tile * RW_TILE * KW;
            if (threadIdx.x < RW_TILE * KW && KW <= 2)
                skeep[threadIdx.x] = (w0 + threadIdx.x < total * KW) ? __ldg(keep + w0 + threadIdx.x) : 0u;
        }
        __syncthreads();                                           // CTA
        for (int r = 0; r < RW_TILE; ++r) {
            const RayAtDoe& R = info[r];
            if (!R.alive) {
                if (MODE == MODE_EMIT) emit_dead<M>(sys, tile * RW_TILE + r, total, eo);
                if (MODE == MODE_SPLAT && vis && tile * RW_TILE + r < total)
                    for (int f = threadIdx.x; f < M * M / 32; f += RW_THREADS)
                        vis[(tile * RW_TILE + r) * (long long)(M * M / 32) + f] = 0u;
                continue;
            }
            const DJob& J = jobs[R.job];
            const float2* Tj = Tmaps + (long long)J.slot * npix_map;
            bool staged = false;
            if constexpr (M == 64) {
                if (bulk_patch_ok<M>(sys, R)) {
                    if (threadIdx.x < 32) bulk_patch_issue<M>(sys, R, Tj, X, &bulk_bar);
                    phase_factors<M>(sys, R, phu, phv);
                    if (!mbar_wait_bounded(&bulk_bar, bulk_phase, RW_BULK_WAIT) && threadIdx.x == 0)
                        atomicOr(status, RW_ST_TIMEOUT);
                    bulk_phase ^= 1u;
                    fft2d_staged<M, false>(X, tw, R.c0 & 1);
                    staged = true;
                }
            }
            if (!staged) {
                gather_patch<M>(sys, R, Tj, X, phu, phv);
                main_sync();
                fft2d<M, false>(X, tw);
            }
            if (sys.emit == RW_EMIT_EXHAUSTIVE) {
                emit_exhaustive<M, MODE, NS>(sys, J, R, X, phu, phv, psf, field, eo,
                                             tile * RW_TILE + r, status, vis,
                                             keep ? skeep + r * cull_keep_words(M) : nullptr,
                                             vw, tape, f0, f1);
            } else {
                emit_sampled<M, MODE, NS, HW ? RW_GQ_HELPED : RW_GQ>(sys, J, R, X, phu, phv, psf,
                                                                     field, eo,
                                          tile * RW_TILE + r, status,
                                          smem + sampled_scratch_offset(M),
                                          MODE == MODE_COHERENT ? f0 : 0,
                                          MODE == MODE_COHERENT ? f1 : -1);
            }
            // the next patch's bulk copies write X through the async proxy
            if (M == 64) fence_async_smem();
            main_sync();
        }
    }
}

// ------------------------------------------------------------- block culling
// keep[g * KW + w] bit b: 8 x 8 bin block 32 w + b of incident ray g may reach
// the sensor (its affine enclosure does not miss the sensor window).  With a
// planar DOE, the rays of a tile are tested in groups of 8 of one job: one
// test per (group, block) spans the group's DOE hit points and incident
// tangential wavevectors, and a kept block is kept for every ray of the
// group.  Other groups (mixed jobs, conformal DOE) are tested ray by ray.
// Rays that miss the DOE keep nothing.
template <int M, int NS>
__global__ void __launch_bounds__(RW_THREADS, 2)
k_cull(const DSys sys, const DJob* __restrict__ jobs, const long long* __restrict__ prefix,
       int njob, long long total, RaysIn rays, unsigned* __restrict__ keep, unsigned* status) {
    constexpr int B8 = M / 8, NB = B8 * B8, KW = cull_keep_words(M);
    constexpr int G = 8, NG = RW_TILE / G;
    __shared__ RayAtDoe info[RW_TILE];
    __shared__ unsigned kw[RW_TILE * KW];
    __shared__ float gbox[NG][8];     // x, y, k_u, k_v ranges of the group's rays
    __shared__ int grep[NG];          // group's first live ray; -1: ray by ray; -2: none
    const long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    const float ks = sys.kstep;
    const int lane = threadIdx.x & 31;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        if (threadIdx.x < RW_TILE)
            incident_to_doe<false>(sys, jobs, prefix, njob, total, rays,
                                   tile * RW_TILE + threadIdx.x, info[threadIdx.x], status);
        for (int i = threadIdx.x; i < RW_TILE * KW; i += RW_THREADS) kw[i] = 0u;
        __syncthreads();
        if (threadIdx.x < RW_TILE) {
            const RayAtDoe& R = info[lane];
            const bool live = R.alive == 1;
            // minima of (x, -x, y, -y, k_u, -k_u, k_v, -k_v) over each group of 8 lanes
            float v[8] = {live ? R.px : INFINITY, live ? -R.px : INFINITY,
                          live ? R.py : INFINITY, live ? -R.py : INFINITY,
                          live ? R.kin_u : INFINITY, live ? -R.kin_u : INFINITY,
                          live ? R.kin_v : INFINITY, live ? -R.kin_v : INFINITY};
            int jlo = live ? R.job : 0x7fffffff, jhi = live ? R.job : -1;
            int first = live ? lane : 0x7fffffff;
            for (int o = 1; o < G; o <<= 1) {
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] = fminf(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
                jlo = min(jlo, __shfl_xor_sync(0xffffffffu, jlo, o));
                jhi = max(jhi, __shfl_xor_sync(0xffffffffu, jhi, o));
                first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
            }
            if ((lane & (G - 1)) == 0) {
                const int g = lane / G;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    gbox[g][2 * k] = v[2 * k];
                    gbox[g][2 * k + 1] = -v[2 * k + 1];
                }
                grep[g] = (jhi < 0) ? -2 : ((jlo == jhi && !sys.conformal) ? first : -1);
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < NG * NB; t += RW_THREADS) {
            const int g = t / NB, bi = t - g * NB;
            const int rep = grep[g];
            if (rep < 0) continue;
            const float* b = gbox[g];
            const float ju_c = (float)((bi % B8) * 8 - M / 2) + 3.5f;
            const float jv_c = (float)((bi / B8) * 8 - M / 2) + 3.5f;
            // centre and half-width of each range, widened by a relative 1e-6
            const float hu = (3.5f * ks + 0.5f * (b[5] - b[4])) * (1.f + 1e-6f);
            const float hv = (3.5f * ks + 0.5f * (b[7] - b[6])) * (1.f + 1e-6f);
            const float hx = 0.5f * (b[1] - b[0]) * (1.f + 1e-6f);
            const float hy = 0.5f * (b[3] - b[2]) * (1.f + 1e-6f);
            if (!af_block_misses_sensor<NS>(sys, info[rep], fmaf(ks, ju_c, 0.5f * (b[4] + b[5])),
                                            hu, fmaf(ks, jv_c, 0.5f * (b[6] + b[7])), hv,
                                            0.5f * (b[0] + b[1]), hx, 0.5f * (b[2] + b[3]), hy)) {
                for (int i = 0; i < G; ++i)
                    if (info[g * G + i].alive == 1)
                        atomicOr(&kw[(g * G + i) * KW + (bi >> 5)], 1u << (bi & 31));
            }
        }
        for (int t = threadIdx.x; t < RW_TILE * NB; t += RW_THREADS) {
            const int r = t / NB, bi = t - r * NB;
            if (grep[r / G] != -1) continue;
            const RayAtDoe& R = info[r];
            if (R.alive != 1) continue;
            const float ju_c = (float)((bi % B8) * 8 - M / 2) + 3.5f;
            const float jv_c = (float)((bi / B8) * 8 - M / 2) + 3.5f;
            if (!af_block_misses_sensor<NS>(sys, R, fmaf(ks, ju_c, R.kin_u), 3.5f * ks,
                                            fmaf(ks, jv_c, R.kin_v), 3.5f * ks, R.px, 0.f, R.py,
                                            0.f))
                atomicOr(&kw[r * KW + (bi >> 5)], 1u << (bi & 31));
        }
        // rays the FP32 run could not place: every block kept
        for (int t = threadIdx.x; t < RW_TILE * KW; t += RW_THREADS) {
            const int r = t / KW, w = t - (t / KW) * KW;
            if (info[r].alive == 2) {
                const int nb = NB - 32 * w;
                kw[t] = nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u);
            }
        }
        __syncthreads();
        const long long g0 = tile * RW_TILE;
        for (int i = threadIdx.x; i < RW_TILE * KW; i += RW_THREADS)
            if (g0 + i / KW < total) keep[g0 * KW + i] = kw[i];
    }
}

// float PSF from the double accumulator.
__global__ void k_psf_finalize(const double* __restrict__ acc, float* __restrict__ psf,
                               long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        psf[i] = (float)acc[i];
}

// |U|^2 of the coherent field.
__global__ void k_coherent_finalize(const float2* __restrict__ field, float* __restrict__ psf,
                                    long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float2 f = field[i];
        psf[i] = f.x * f.x + f.y * f.y;
    }
}

// dL/dU = 2 (dL/dI) U for I = |U|^2 (real and imaginary part), in place.
__global__ void k_coherent_grad(float2* __restrict__ field, const float* __restrict__ g,
                                long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 f = field[i];
        const float s = 2.f * g[i];
        field[i] = make_float2(s * f.x, s * f.y);
    }
}

// ------------------------------------------------------------- launchers
template <int M, int NS>
static cudaError_t launch_cull_d(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                                const long long* prefix, int njob, long long total,
                                const RaysIn& rays, unsigned* keep, unsigned* status) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cull<M, NS>,
                                                                  RW_THREADS, 0);
    if (e != cudaSuccess) return e;
    long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    long long grid = pick_grid(L, RW_K_CULL, (long long)L.num_sms * (per_sm > 0 ? per_sm : 1));
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    RW_MARK(L, "k_cull");
    k_cull<M, NS><<<(unsigned)grid, RW_THREADS, 0, L.stream>>>(sys, jobs, prefix, njob, total,
                                                              rays, keep, status);
    RW_MARK(L, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_cull(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                        const long long* prefix, int njob, long long total, const RaysIn& rays,
                        unsigned* keep, unsigned* status) {
#define RW_CULL_NS(DD)                                                                          \
    switch (sys.n_post) {                                                                       \
        case 0: return launch_cull_d<DD, 0>(L, sys, jobs, prefix, njob, total, rays, keep, status); \
        case 2: return launch_cull_d<DD, 2>(L, sys, jobs, prefix, njob, total, rays, keep, status); \
        case 4: return launch_cull_d<DD, 4>(L, sys, jobs, prefix, njob, total, rays, keep, status); \
        case 6: return launch_cull_d<DD, 6>(L, sys, jobs, prefix, njob, total, rays, keep, status); \
        default: return cudaErrorInvalidValue;                                                  \
    }
    switch (sys.M) {
        case 16: RW_CULL_NS(16)
        case 32: RW_CULL_NS(32)
        case 64: RW_CULL_NS(64)
        default: return cudaErrorInvalidValue;
    }
#undef RW_CULL_NS
}

// Helper warps of the sampled forward at M = 96 (one CTA per SM): 8 more
// warps, so 16 per SM, when their queues still fit in shared memory.
#define RW_FWD_HELPERS 8

template <int M, int MODE, int NS, int HW = 0>
static cudaError_t launch_forward_d(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                                    const long long* prefix, int njob, long long total,
                                    const RaysIn& rays, const float2* T, double* psf,
                                    float2* field, const EmitOut& eo, unsigned* status,
                                    unsigned* vis, unsigned* keep, const SplitBufs* tapep) {
    if constexpr (HW == 0 && M == 96 && MODE == MODE_SPLAT) {
        int dev = 0, optin = 0;
        if (sys.emit == RW_EMIT_SAMPLED && cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) ==
                cudaSuccess &&
            forward_smem_bytes(M, sys.emit, sys.n_ssr, RW_FWD_HELPERS) <= (size_t)optin)
            return launch_forward_d<M, MODE, NS, RW_FWD_HELPERS>(L, sys, jobs, prefix, njob,
                                                                 total, rays, T, psf, field, eo,
                                                                 status, vis, keep, tapep);
    }
    constexpr int NT = RW_THREADS + 32 * HW;
    SplitBufs tape;
    std::memset(&tape, 0, sizeof(tape));
    if constexpr (MODE == MODE_SPLAT && NS >= 0 && M <= 64) {
        if (keep) {
            // block culling: kept-block bits for every incident ray first
            cudaError_t e = launch_cull_d<M, NS>(L, sys, jobs, prefix, njob, total, rays, keep,
                                                 status);
            if (e != cudaSuccess) return e;
        }
        if (tapep && vis) {
            tape = *tapep;
            if (!keep) tape.iray = nullptr;     // only the culled path tapes
        }
    } else {
        keep = nullptr;
    }
    size_t smem = forward_smem_bytes(M, sys.emit, sys.n_ssr, HW);
    auto kern = k_forward<M, MODE, NS, HW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    long long grid = pick_grid(L, RW_K_FORWARD, (long long)L.num_sms * per_sm);
    // Coherent exhaustive emission: each ray's wavelet sums outweigh its patch
    // FFT by orders of magnitude, so when the tiles alone cannot fill the GPU
    // every ray's bins are split into slices (the FFT is redone per slice).
    DSys s = sys;
    s.nslice = 1;
    if (MODE == MODE_COHERENT && ntiles < grid) {
        const long long want = (grid + ntiles - 1) / ntiles;
        const long long most = sys.emit == RW_EMIT_EXHAUSTIVE
                                   ? (long long)M * M / RW_THREADS
                                   : ((long long)sys.n_ssr + RW_THREADS - 1) / RW_THREADS;
        s.nslice = (int)(want < most ? want : most);
    }
    const long long units = ntiles * s.nslice;
    if (grid > units) grid = units;
    if (grid < 1) grid = 1;
    RW_MARK(L, "k_forward");
    kern<<<(unsigned)grid, NT, smem, L.stream>>>(s, jobs, prefix, njob, total, rays, T, psf,
                                                  field, eo, status, vis, keep, tape);
    RW_MARK(L, nullptr);
    return cudaGetLastError();
}

// Post-DOE surface counts with a specialised (unrolled plane/sphere) trace.
template <int M>
static cudaError_t launch_splat(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                                const long long* prefix, int njob, long long total,
                                const RaysIn& rays, const float2* T, double* psf,
                                const EmitOut& eo, unsigned* status, unsigned* vis,
                                unsigned* keep, const SplitBufs* tape) {
#define RW_SPLAT(NN) \
    launch_forward_d<M, MODE_SPLAT, NN>(L, sys, jobs, prefix, njob, total, rays, T, psf, nullptr, eo, status, vis, keep, tape)
    if (sys.fast_ok) {
        switch (sys.n_post) {
            case 0: return RW_SPLAT(0);
            case 2: return RW_SPLAT(2);
            case 4: return RW_SPLAT(4);
            case 6: return RW_SPLAT(6);
            default: break;
        }
    }
    return RW_SPLAT(-1);
#undef RW_SPLAT
}

bool forward_culls(const DSys& sys) {
    return sys.cull && sys.emit == RW_EMIT_EXHAUSTIVE && !sys.coherent && sys.fast_ok &&
           sys.M <= 64 &&
           (sys.n_post == 0 || sys.n_post == 2 || sys.n_post == 4 || sys.n_post == 6);
}

cudaError_t launch_forward(const LaunchCtx& L, int mode, const DSys& sys, const DJob* jobs,
                           const long long* prefix, int njob, long long total,
                           const RaysIn& rays, const float2* T, double* psf, float2* field,
                           const EmitOut& eo, unsigned* status, unsigned* vis, unsigned* keep,
                           const SplitBufs* tape) {
#define RW_FWD_CASE(DD)                                                                       \
    case DD:                                                                                  \
        if (mode == MODE_SPLAT)                                                               \
            return launch_splat<DD>(L, sys, jobs, prefix, njob, total, rays, T, psf, eo,      \
                                    status, vis, forward_culls(sys) ? keep : nullptr, tape);  \
        if (mode == MODE_COHERENT)                                                            \
            return launch_forward_d<DD, MODE_COHERENT, -1>(L, sys, jobs, prefix, njob, total, \
                                                           rays, T, psf, field, eo, status,   \
                                                           nullptr, nullptr, nullptr);        \
        return launch_forward_d<DD, MODE_EMIT, -1>(L, sys, jobs, prefix, njob, total, rays, T,\
                                                   psf, field, eo, status, nullptr, nullptr,  \
                                                   nullptr);
    switch (sys.M) {
        RW_FWD_CASE(16)
        RW_FWD_CASE(32)
        RW_FWD_CASE(64)
        RW_FWD_CASE(96)
        RW_FWD_CASE(128)
        default: return cudaErrorInvalidValue;
    }
#undef RW_FWD_CASE
}

cudaError_t launch_prep_maps(const LaunchCtx& L, const float* phi, const float* phi2,
                             const float* amp, int64_t npix, const float* scales_dev, int nslot,
                             float2* T) {
    long long n = npix * nslot;
    long long grid = (n + 255) / 256;
    long long cap = (long long)L.num_sms * 8;
    if (grid > cap) grid = cap;
    RW_MARK(L, "k_prep_maps");
    k_prep_maps<<<(unsigned)grid, 256, 0, L.stream>>>(phi, phi2, amp, npix, scales_dev, nslot,
                                                      T);
    RW_MARK(L, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_generate_rays(const LaunchCtx& L, const GenJob* jobs, const long long* prefix,
                                 int njob, long long total, double z_start, double n_object,
                                 const RaysOut& out) {
    long long grid = (total + 255) / 256;
    long long cap = (long long)L.num_sms * 16;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    RW_MARK(L, "k_generate_rays");
    k_generate_rays<<<(unsigned)grid, 256, 0, L.stream>>>(jobs, prefix, njob, total, z_start,
                                                          n_object, out);
    RW_MARK(L, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_coherent_finalize(const LaunchCtx& L, const float2* field, float* psf,
                                     long long n) {
    long long grid = (n + 255) / 256;
    long long cap = (long long)L.num_sms * 8;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    RW_MARK(L, "k_coherent_finalize");
    k_coherent_finalize<<<(unsigned)grid, 256, 0, L.stream>>>(field, psf, n);
    RW_MARK(L, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_coherent_grad(const LaunchCtx& L, float2* field, const float* g, long long n) {
    long long grid = (n + 255) / 256;
    long long cap = (long long)L.num_sms * 8;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    RW_MARK(L, "k_coherent_grad");
    k_coherent_grad<<<(unsigned)grid, 256, 0, L.stream>>>(field, g, n);
    RW_MARK(L, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_psf_finalize(const LaunchCtx& L, const double* acc, float* psf, long long n) {
    long long grid = (n + 255) / 256;
    long long cap = (long long)L.num_sms * 8;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    RW_MARK(L, "k_psf_finalize");
    k_psf_finalize<<<(unsigned)grid, 256, 0, L.stream>>>(acc, psf, n);
    RW_MARK(L, nullptr);
    return cudaGetLastError();
}
