// A9 (exhaustive emission, with the forward's visibility mask), split by
// resource needs into three kernels:
//
//   k_bs_spectra   per incident ray: DOE hit and frame, patch, FFT, and a
//                  compaction of the bins whose secondary ray reached the
//                  sensor into a flat work list (ray, bin, U~) -- shared
//                  memory and barriers, few registers, high occupancy;
//   k_bs_trace     one thread per visible secondary ray: re-trace, reverse of
//                  sensor plane / surfaces / emission, dL/dU~ -- registers, no
//                  barriers, every lane busy; per-ray geometric sums with a
//                  segmented warp reduction, surface sums per CTA;
//   k_bs_scatter   per incident ray: sparse dL/dU~ -> dL/dX, conjugate FFT,
//                  map scatter, and the incident-side reverse (DOE hit,
//                  pre-DOE surfaces) from the per-ray sums.
//
// The arithmetic per secondary ray is exactly that of the fused adjoint
// (rw_backward.cu); only the schedule differs.
#include "rw_bwd_common.cuh"

// ------------------------------------------------------------------ count
__global__ void k_bs_count(const unsigned* __restrict__ vis, long long nwords,
                           unsigned long long* __restrict__ total) {
    unsigned long long c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nwords;
         i += (long long)gridDim.x * blockDim.x)
        c += __popc(__ldg(vis + i));
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(total, c);
}

// ------------------------------------------------------------------ 1: spectra + list
template <int M>
__global__ void __launch_bounds__(RW_THREADS, M <= 64 ? 4 : 1)
k_bs_spectra(const DSys sys, const DJob* __restrict__ jobs, const long long* __restrict__ prefix,
             int njob, long long total, RaysIn rays, const float2* __restrict__ Tmaps,
             const unsigned* __restrict__ vis, SplitBufs B, unsigned* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2* X = reinterpret_cast<float2*>(smem);
    float2* tw = X + Patch<M>::ELEMS;
    float2* phu = tw + M;
    float2* phv = phu + M;
    RayAtDoe* info = reinterpret_cast<RayAtDoe*>(phv + M);
    int* wsum = reinterpret_cast<int*>(smem + sampled_scratch_offset(M));   // [8 warps + 3]
    fft_twiddles<M>(tw);
    constexpr int NW = M * M / 32;                               // visibility words per ray
    constexpr int KW = (NW + RW_THREADS - 1) / RW_THREADS;       // words per thread
    const float norm = sys.norm;
    const long long npix_map = (long long)sys.H * sys.W;
    const long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        if (threadIdx.x < RW_TILE) {
            const long long g = tile * RW_TILE + threadIdx.x;
            incident_to_doe(sys, jobs, prefix, njob, total, rays, g, info[threadIdx.x], status);
            if (g < total) B.rinfo[g] = info[threadIdx.x];
        }
        __syncthreads();
        for (int r = 0; r < RW_TILE; ++r) {
            const long long g = tile * RW_TILE + r;
            if (g >= total) break;
            const RayAtDoe& R = info[r];
            // visible bins of this ray: thread t owns words t KW .. t KW + KW - 1
            // (word w holds bins 32w .. 32w + 31), so items come out in bin order
            unsigned word[KW];
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < KW; ++k) {
                const int wi = threadIdx.x * KW + k;
                word[k] = (R.alive && wi < NW) ? __ldg(vis + g * (long long)NW + wi) : 0u;
                cnt += __popc(word[k]);
            }
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            if (threadIdx.x == 0) {
                int t = 0;
                for (int w = 0; w < RW_THREADS / 32; ++w) { const int v = wsum[w]; wsum[w] = t; t += v; }
                long long base = 0;
                if (t > 0) base = (long long)atomicAdd(B.counter, (unsigned long long)t);
                if (base + t > B.cap) { atomicOr(status, RW_ST_CAPACITY); t = 0; base = 0; }
                B.voff[g] = base;
                B.vcnt[g] = t;
                wsum[RW_THREADS / 32] = (int)(base & 0x7fffffff);
                wsum[RW_THREADS / 32 + 1] = (int)(base >> 31);
                wsum[RW_THREADS / 32 + 2] = t;
            }
            __syncthreads();
            const int ntot = wsum[RW_THREADS / 32 + 2];
            if (ntot == 0) continue;
            const long long base = (long long)wsum[RW_THREADS / 32] +
                                   ((long long)wsum[RW_THREADS / 32 + 1] << 31);
            gather_patch<M>(sys, R, Tmaps + (long long)jobs[R.job].slot * npix_map, X, phu, phv);
            __syncthreads();
            fft2d<M, false>(X, tw);
            long long pos = base + wsum[warp] + (incl - cnt);
#pragma unroll
            for (int k = 0; k < KW; ++k) {
                unsigned wk = word[k];
                while (wk) {
                    const int b = __ffs(wk) - 1;
                    wk &= wk - 1u;
                    const int f = (threadIdx.x * KW + k) * 32 + b;
                    const int jvi = f / M, jui = f - (f / M) * M;
                    B.iray[pos] = (int)g;
                    B.ibin[pos] = f;
                    B.iU[pos] = spectrum_at<M>(X, phu, phv, jui, jvi, norm);
                    ++pos;
                }
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------ 2: trace + reverse
template <int M, int NS>
__global__ void __launch_bounds__(RW_THREADS, NS >= 6 ? 2 : 3)
k_bs_trace(const DSys sys, const float* __restrict__ gpsf, SplitBufs B, long long nitems,
           double* __restrict__ dsurf, unsigned* status) {
    __shared__ double dred[RW_MAXS * RW_NGRAD * (RW_THREADS / 32)];
    SurfGrads<NS> SG;
    SG.zero();
    float gs[RW_MAXS * RW_NGRAD];
#pragma unroll
    for (int i = 0; i < RW_MAXS * RW_NGRAD; ++i) gs[i] = 0.f;
    const long long npx = (long long)sys.nx * sys.ny;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // rounds are warp-uniform so the segmented reductions see whole warps
    const long long nround = (nitems + stride - 1) / stride;
    for (long long rd = 0; rd < nround; ++rd) {
        const long long t = rd * stride + blockIdx.x * (long long)blockDim.x + threadIdx.x;
        float acc[RW_RS];
#pragma unroll
        for (int k = 0; k < RW_RS; ++k) acc[k] = 0.f;
        int g = -1;
        if (t < nitems) {
            g = __ldg(B.iray + t);
            const int f = __ldg(B.ibin + t);
            const float2 U = B.iU[t];
            // the split adjoint runs only in single-launch calls (no wavelength
            // groups), where a job's image index is its index in the job table
            const RayAtDoe& R = B.rinfo[g];
            const int jvi = f / M, jui = f - (f / M) * M;
            float2 gU = make_float2(0.f, 0.f);
            float dx, dy, dz;
            const float2 ain = make_float2(R.a_re, R.a_im);
            if (bin_direction<(NS >= 0)>(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz)) {
                const float2 a = cmul(ain, U);
                const float w = a.x * a.x + a.y * a.y;
                float gw, gx, gy, gz, gdx, gdy, gdz;
                if (secondary_adjoint<NS>(sys, R, gpsf + (long long)R.job * npx, dx, dy, dz, w,
                                          gw, gx, gy, gz, gdx, gdy, gdz, SG, gs, status)) {
                    emission_adjoint(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz, gx, gy, gz,
                                     gdx, gdy, gdz, acc);
                    const float2 ga = make_float2(2.f * a.x * gw, 2.f * a.y * gw);
                    gU = cmulc(ga, ain);
                }
            }
            B.igU[t] = gU;
        }
        // segmented warp sum of acc over lanes with the same ray (runs are contiguous)
        const int gprev = __shfl_up_sync(0xffffffffu, g, 1);
        const bool head = (lane == 0) || (gprev != g);
        const unsigned heads = __ballot_sync(0xffffffffu, head);
        // lane of the head of my run: highest set bit of heads at or below lane
        const unsigned mine = heads & (0xffffffffu >> (31 - lane));
        const int my_head = 31 - __clz(mine);
        // end of my run: next head above me (or 32)
        const unsigned above = heads & ~(0xffffffffu >> (31 - lane));
        const int run_end = above ? (__ffs(above) - 1) : 32;
        // planar: dL/dP, dL/dkappa, dL/dK; conformal also the frame sums
        const int nk = sys.conformal ? RW_RS_GATHER : 6;
#pragma unroll
        for (int k = 0; k < RW_RS_GATHER; ++k) {
            if (k >= nk) continue;
            float v = acc[k];
            for (int o = 1; o < 32; o <<= 1) {
                const float n = __shfl_down_sync(0xffffffffu, v, o);
                if (lane + o < run_end) v += n;
            }
            acc[k] = v;   // the head lane now holds its run's sum
        }
        if (lane == my_head && g >= 0) {
            bool any = false;
#pragma unroll
            for (int k = 0; k < RW_RS_GATHER; ++k) any |= (k < nk) && acc[k] != 0.f;
            if (any)
                for (int k = 0; k < nk; ++k)
                    atomicAdd(B.rsum + (long long)g * sys.nrs + k, acc[k]);
        }
    }
    // ---- surface sums: registers -> CTA -> global
    if (!dsurf) return;
    if constexpr (NS >= 0) {
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const int si = sys.doe_index + 1 + i;
            gs[si * RW_NGRAD + 0] += SG.fz[i];
            gs[si * RW_NGRAD + 1] += SG.fc[i];
            gs[si * RW_NGRAD + 7] += SG.fn[i];
        }
        gs[sys.doe_index * RW_NGRAD + 7] += SG.f_doe_n;
    }
    for (int s = 0; s < sys.nsurf; ++s)
        for (int k = 0; k < RW_NGRAD; ++k) {
            float v = gs[s * RW_NGRAD + k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) dred[(s * RW_NGRAD + k) * (RW_THREADS / 32) + warp] = (double)v;
        }
    __syncthreads();
    for (int i = threadIdx.x; i < sys.nsurf * RW_NGRAD; i += RW_THREADS) {
        double v = 0.0;
        for (int w = 0; w < RW_THREADS / 32; ++w) v += dred[i * (RW_THREADS / 32) + w];
        if (v != 0.0) atomicAdd(dsurf + i, v);
    }
}

// ------------------------------------------------------------------ 3: conjugate FFT + scatter
template <int M>
__global__ void __launch_bounds__(RW_THREADS, M <= 64 ? 4 : 1)
k_bs_scatter(const DSys sys, const DJob* __restrict__ jobs, const long long* __restrict__ prefix,
             int njob, long long total, RaysIn rays, const float2* __restrict__ Tmaps,
             const float* __restrict__ amp, SplitBufs B, float* __restrict__ dphi,
             float* __restrict__ damp, double* __restrict__ dsurf, unsigned* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2* G = reinterpret_cast<float2*>(smem);
    float2* tw = G + Patch<M>::ELEMS;
    float2* phu = tw + M;
    float2* phv = phu + M;
    RayAtDoe* info = reinterpret_cast<RayAtDoe*>(phv + M);
    fft_twiddles<M>(tw);
    const float norm = sys.norm;
    float gs[RW_MAXS * RW_NGRAD];
    for (int i = 0; i < RW_MAXS * RW_NGRAD; ++i) gs[i] = 0.f;
    const long long npix_map = (long long)sys.H * sys.W;
    const long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        if (threadIdx.x < RW_TILE) {
            const long long g = tile * RW_TILE + threadIdx.x;
            if (g < total) info[threadIdx.x] = B.rinfo[g]; else info[threadIdx.x].alive = 0;
        }
        __syncthreads();
        for (int r = 0; r < RW_TILE; ++r) {
            const long long g = tile * RW_TILE + r;
            if (g >= total) break;
            const RayAtDoe& R = info[r];
            const int n = R.alive ? B.vcnt[g] : 0;
            if (n == 0) continue;
            const long long off = B.voff[g];
            for (int f = threadIdx.x; f < Patch<M>::ELEMS; f += RW_THREADS)
                G[f] = make_float2(0.f, 0.f);
            phase_factors<M>(sys, R, phu, phv);
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += RW_THREADS) {
                const int f = __ldg(B.ibin + off + i);
                const float2 gU = B.igU[off + i];
                const int jvi = f / M, jui = f - (f / M) * M;
                int mu = jui + M / 2; if (mu >= M) mu -= M;
                int mv = jvi + M / 2; if (mv >= M) mv -= M;
                const float2 ph = cmul(phu[jui], phv[jvi]);
                G[mv * Patch<M>::S + mu] = cscale(cmulc(gU, ph), norm);
            }
            __syncthreads();
            fft2d<M, true>(G, tw);
            float gq[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            map_scatter<M>(sys, R, Tmaps + (long long)jobs[R.job].slot * npix_map, amp, G,
                           jobs[R.job].phase_scale, dphi, damp, sys.conformal ? gq : nullptr);
            if (sys.conformal) {
                // patch-position sums of this ray: block reduction into its per-ray sums
                float* red = reinterpret_cast<float*>(info + RW_TILE);
#pragma unroll
                for (int k = 0; k < 6; ++k)
                    for (int o = 16; o > 0; o >>= 1) gq[k] += __shfl_xor_sync(0xffffffffu, gq[k], o);
                __syncthreads();
                if ((threadIdx.x & 31) == 0)
#pragma unroll
                    for (int k = 0; k < 6; ++k) red[(threadIdx.x >> 5) * 6 + k] = gq[k];
                __syncthreads();
                if (threadIdx.x < 6) {
                    float v = 0.f;
                    for (int w = 0; w < RW_THREADS / 32; ++w) v += red[w * 6 + threadIdx.x];
                    B.rsum[g * sys.nrs + RW_RS_GATHER + threadIdx.x] = v;
                }
            }
            __syncthreads();
        }
        // incident side from the per-ray sums
        if (threadIdx.x < RW_TILE && info[threadIdx.x].alive) {
            const RayAtDoe& R = info[threadIdx.x];
            const long long g = tile * RW_TILE + threadIdx.x;
            float s[RW_RS];
#pragma unroll
            for (int k = 0; k < RW_RS; ++k) s[k] = k < sys.nrs ? B.rsum[g * sys.nrs + k] : 0.f;
            incident_adjoint(sys, jobs, prefix, rays, R, s, gs, status);
        }
    }
    if (!dsurf) return;
    reduce_surface_grads(sys, gs, reinterpret_cast<double*>(smem), dsurf);
}

// ------------------------------------------------------------------ launch
size_t split_item_bytes() { return sizeof(int) * 2 + sizeof(float2) * 2; }

cudaError_t launch_bs_count(const LaunchCtx& L, const unsigned* vis, long long nwords,
                            unsigned long long* total) {
    cudaError_t e = cudaMemsetAsync(total, 0, sizeof(unsigned long long), L.stream);
    if (e != cudaSuccess) return e;
    long long grid = (nwords + 255) / 256;
    if (grid > (long long)L.num_sms * 8) grid = (long long)L.num_sms * 8;
    if (grid < 1) grid = 1;
    RW_MARK(L, "k_bs_count");
    k_bs_count<<<(unsigned)grid, 256, 0, L.stream>>>(vis, nwords, total);
    RW_MARK(L, nullptr);
    return cudaGetLastError();
}

template <typename K>
static cudaError_t persistent_launch_cfg(K kern, size_t smem, int num_sms, long long work,
                                         long long override_grid, long long* grid) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RW_THREADS, smem);
    if (e != cudaSuccess) return e;
    long long gsz = (long long)num_sms * (per_sm > 0 ? per_sm : 1);
    if (override_grid > 0) gsz = override_grid;
    if (gsz > work) gsz = work;
    *grid = gsz < 1 ? 1 : gsz;
    return cudaSuccess;
}

template <int M, int NS>
static cudaError_t launch_split_d(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                                  const long long* prefix, int njob, long long total,
                                  const RaysIn& rays, const float2* T, const float* amp,
                                  const float* gpsf, const unsigned* vis, const SplitBufs& B,
                                  long long nitems, int have_list, float* dphi, float* damp,
                                  double* dsurf, unsigned* status) {
    const long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    long long grid;
    cudaError_t e = cudaSuccess;
    if (!have_list) {
        // patch spectra and the work list (otherwise the forward taped both)
        size_t smem1 = sampled_scratch_offset(M) + 64;
        e = persistent_launch_cfg(k_bs_spectra<M>, smem1, L.num_sms, ntiles,
                                  pick_grid(L, RW_K_BS_SPECTRA, 0), &grid);
        if (e != cudaSuccess) return e;
        RW_MARK(L, "k_bs_spectra");
        k_bs_spectra<M><<<(unsigned)grid, RW_THREADS, smem1, L.stream>>>(sys, jobs, prefix, njob,
                                                                         total, rays, T, vis, B, status);
        RW_MARK(L, nullptr);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (nitems > 0) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bs_trace<M, NS>, RW_THREADS, 0);
        if (e != cudaSuccess) return e;
        long long g2 = pick_grid(L, RW_K_BS_TRACE, (long long)L.num_sms * (per_sm > 0 ? per_sm : 1) * 4);
        const long long need = (nitems + RW_THREADS - 1) / RW_THREADS;
        if (g2 > need) g2 = need;
        RW_MARK(L, "k_bs_trace");
        k_bs_trace<M, NS><<<(unsigned)g2, RW_THREADS, 0, L.stream>>>(sys, gpsf, B, nitems, dsurf,
                                                                      status);
        RW_MARK(L, nullptr);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    size_t smem3 = sampled_scratch_offset(M) + 256;   // + the patch-position reduction
    const size_t red = sizeof(double) * RW_MAXS * RW_NGRAD * (RW_THREADS / 32);
    if (smem3 < red) smem3 = red;
    e = persistent_launch_cfg(k_bs_scatter<M>, smem3, L.num_sms, ntiles,
                              pick_grid(L, RW_K_BS_SCATTER, 0), &grid);
    if (e != cudaSuccess) return e;
    RW_MARK(L, "k_bs_scatter");
    k_bs_scatter<M><<<(unsigned)grid, RW_THREADS, smem3, L.stream>>>(
        sys, jobs, prefix, njob, total, rays, T, amp, B, dphi, damp, dsurf, status);
    RW_MARK(L, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_backward_split(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                                  const long long* prefix, int njob, long long total,
                                  const RaysIn& rays, const float2* T, const float* amp,
                                  const float* gpsf, const unsigned* vis, const SplitBufs& B,
                                  long long nitems, int have_list, float* dphi, float* damp,
                                  double* dsurf, unsigned* status) {
    const int ns = sys.fast_ok ? sys.n_post : -1;
#define RW_BS(DD, NN) \
    launch_split_d<DD, NN>(L, sys, jobs, prefix, njob, total, rays, T, amp, gpsf, vis, B, nitems, have_list, dphi, damp, dsurf, status)
#define RW_BS_D(DD)                          \
    case DD:                                 \
        switch (ns) {                        \
            case 0: return RW_BS(DD, 0);     \
            case 2: return RW_BS(DD, 2);     \
            case 4: return RW_BS(DD, 4);     \
            case 6: return RW_BS(DD, 6);     \
            default: return RW_BS(DD, -1);   \
        }
    switch (sys.M) {
        RW_BS_D(16)
        RW_BS_D(32)
        RW_BS_D(64)
        RW_BS_D(96)
        RW_BS_D(128)
        default: return cudaErrorInvalidValue;
    }
#undef RW_BS_D
#undef RW_BS
}
