// A9: adjoint of the fused forward (incoherent and coherent sensor).
//
// Per incident ray the CTA recomputes the patch and its spectrum (nothing
// from the forward is stored).  For every secondary ray it re-traces to the
// sensor keeping the state entering each surface, gathers dL/dI at the four
// bilinear taps and runs the hand-written reverse of the sensor plane and of
// every surface (implicit-function derivative of the intersection, normal,
// Snell).  The gradient w.r.t. the amplitude gives dL/dU~, the one w.r.t.
// the emitted direction gives dL/dkappa and so dL/d(incident direction),
// the one w.r.t. the ray origin gives dL/d(hit point).
//
// Exhaustive emission: one secondary ray per propagating bin, a = a_in U~.
// Sampled emission (straight-through Gumbel-softmax, temperature 1): the
// value of each draw is the hard argmax; its gradient reaches the chosen
// bin's weight w = U~ / sqrt(N p) directly, and every bin's log-probability
// through the softmax Jacobian of the perturbed scores, with
// dL/dy_ij = Re(conj(dL/da_i) a_in w_j) + dL/dd_i . dir_j.
//
// dL/dU~ goes through the adjoint of the patch transform (the conjugate
// FFT of the zero-padded M x M buffer) to dL/dT on the D x D patch;
// dT/dphi = i (lambda0/lambda) T and dT/dA = exp(i psi) give the map
// gradients, added with atomics.  Surface
// gradients are kept per thread and reduced once per CTA into dsurf.
//
// Coherent sensor (Eq. 2, I = |U|^2): the caller passes gf = dL/dU = 2 (dL/dI) U
// of the recomputed field.  Each secondary ray is re-traced with its optical
// path; its window sum against gf gives dL/da, dL/dOPL, dL/d(sensor hit) and
// dL/d(direction) (tilt term and obliquity d_z).  dL/dOPL runs back through
// every segment n t (surfaces, DOE hit, pre-DOE trace).  With a = a_in U~,
// dL/dU~ = conj(a_in) dL/da; sampled: p ~ |U~|, w = U~ / (N p).  On a planar
// DOE the patch offsets are measured from the hit, U~ = X exp(-i k.(s0, t0))
// with (s0, t0) = (first sample) - hit, so dU~/dhit = i k U~ (zero in the
// incoherent case, where the gradient w.r.t. U~ is a real multiple of U~).
#include "rw_bwd_common.cuh"

// ------------------------------------------------------------------ sampled
// Shared scratch of the sampled adjoint (after the exhaustive layout).
__host__ __device__ inline size_t sampled_bwd_bytes(int M, int N) {
    return (size_t)M * M * (4 + 8 + 4) + (size_t)N * (4 + 4 + 4 + 8 + 12 + 4) + 64 * 4;
}

// Block-wide sum (all threads get the result); `red` holds >= 8 floats.
__device__ __forceinline__ float block_sum(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    for (int w = 0; w < RW_THREADS / 32; ++w) t += red[w];
    return t;
}

// Gumbel noise g = -log(-log u) of the four bins 4G..4G+3 of draw i.
__device__ __forceinline__ void gumbel_group(const DSys& sys, long long gid, int i, int G,
                                             float* g4) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)G, (uint32_t)i, (uint32_t)gid,
                                             (uint32_t)sys.rng_offset),
                                  (uint32_t)(sys.seed & 0xffffffffull), (uint32_t)(sys.seed >> 32));
    g4[0] = -logf(-logf(u01(w.x)));
    g4[1] = -logf(-logf(u01(w.y)));
    g4[2] = -logf(-logf(u01(w.z)));
    g4[3] = -logf(-logf(u01(w.w)));
}

template <int M, int NS, bool COH>
__device__ __forceinline__ void sampled_ray_adjoint(const DSys& sys, const RayAtDoe& R,
                                                    float k0, long long stream,
                                                    const float2* X, const float2* phu,
                                                    const float2* phv,
                                                    const float* __restrict__ gimg,
                                                    const float2* __restrict__ gf, float2* G,
                                                    unsigned char* scr, float* acc,
                                                    SurfGrads<NS>& SG, float* gs,
                                                    unsigned* status) {
    constexpr int NB = M * M;
    constexpr int S_ = Patch<M>::S;
    const int N = sys.n_ssr;
    const float norm = sys.norm;
    float* logp = reinterpret_cast<float*>(scr);
    float2* gwb = reinterpret_cast<float2*>(logp + NB);
    float* glogp = reinterpret_cast<float*>(gwb + NB);
    int* sel = reinterpret_cast<int*>(glogp + NB);
    float* mx = reinterpret_cast<float*>(sel + N);
    float* zs = mx + N;
    float2* ga = reinterpret_cast<float2*>(zs + N);
    float* gd = reinterpret_cast<float*>(ga + N);
    float* cdot = gd + 3 * N;
    float* red = cdot + N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float2 ain = make_float2(R.a_re, R.a_im);
    // ---- weights m = |U~|^2 (|U~| coherent) over propagating bins, p = m / S
    float part = 0.f;
    for (int f = threadIdx.x; f < NB; f += RW_THREADS) {
        const int jvi = f / M, jui = f - (f / M) * M;
        float dx, dy, dz;
        float m = 0.f;
        if (bin_direction(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz)) {
            const float2 U = spectrum_at<M>(X, phu, phv, jui, jvi, norm);
            m = U.x * U.x + U.y * U.y;
            if (COH) m = sqrtf(m);
            if (sys.uniform) m = 1.f;
        }
        logp[f] = m;
        gwb[f] = make_float2(0.f, 0.f);
        glogp[f] = 0.f;
        part += m;
    }
    const float S = block_sum(part, red);
    const float iS = S > 0.f ? 1.f / S : 0.f;
    for (int f = threadIdx.x; f < NB; f += RW_THREADS) {
        const float p = logp[f] * iS;
        logp[f] = p > 0.f ? logf(p) : -INFINITY;
    }
    __syncthreads();
    // ---- draws: argmax, running max and partition function (warp per draw)
    for (int i = warp; i < N; i += RW_THREADS / 32) {
        float best = -INFINITY, z = 0.f;
        int bj = 0x7fffffff;
        for (int Gq = lane; Gq * 4 < NB; Gq += 32) {
            float g4[4];
            gumbel_group(sys, stream, i, Gq, g4);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int jb = 4 * Gq + q;
                if (jb < NB && logp[jb] > -INFINITY) {
                    const float sc = logp[jb] + g4[q];
                    if (sc > best) {
                        z = (best > -INFINITY ? z * __expf(best - sc) : 0.f) + 1.f;
                        best = sc;
                        bj = jb;
                    } else {
                        z += __expf(sc - best);
                        if (sc == best && jb < bj) bj = jb;
                    }
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const float oz = __shfl_xor_sync(0xffffffffu, z, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            const float nb = fmaxf(best, ob);
            const float nz = (best > -INFINITY ? z * __expf(best - nb) : 0.f) +
                             (ob > -INFINITY ? oz * __expf(ob - nb) : 0.f);
            if (ob > best || (ob == best && oj < bj)) bj = oj;
            best = nb;
            z = nz;
        }
        if (lane == 0) { sel[i] = best > -INFINITY ? bj : -1; mx[i] = best; zs[i] = z; }
    }
    __syncthreads();
    // ---- every draw: trace + reverse of its (hard) secondary ray
    // weight scale sc(p) = 1 / sqrt(N p) (incoherent) or 1 / (N p) (coherent)
    const float sqN = sqrtf((float)N);
    constexpr float EXPO = COH ? -1.f : -0.5f;       // d log sc / d log p
    const float sN = COH ? (float)N : sqN;
    for (int i = threadIdx.x; i < N; i += RW_THREADS) {
        const int jb = sel[i];
        float2 g_a = make_float2(0.f, 0.f);
        float gdx = 0.f, gdy = 0.f, gdz = 0.f;
        if (jb >= 0) {
            const int jvi = jb / M, jui = jb - (jb / M) * M;
            float dx, dy, dz;
            if (bin_direction(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz)) {
                const float2 U = spectrum_at<M>(X, phu, phv, jui, jvi, norm);
                const float sc = __expf(EXPO * logp[jb]) / sN;
                const float2 a = cscale(cmul(ain, U), sc);
                float gx, gy, gz;
                bool hit;
                if constexpr (COH) {
                    float gopl;
                    hit = secondary_adjoint_coh(sys, R, k0, gf, dx, dy, dz, a, g_a, gx, gy, gz,
                                                gdx, gdy, gdz, gopl, gs, status);
                    if (hit) acc[6] += gopl;
                } else {
                    const float w = a.x * a.x + a.y * a.y;
                    float gw;
                    hit = secondary_adjoint<NS>(sys, R, gimg, dx, dy, dz, w, gw, gx, gy, gz, gdx,
                                                gdy, gdz, SG, gs, status);
                    if (hit) g_a = make_float2(2.f * a.x * gw, 2.f * a.y * gw);
                }
                if (hit) {
                    emission_adjoint(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz, gx, gy, gz,
                                     gdx, gdy, gdz, acc);
                    // hard path: a = a_in w_jb  ->  dL/dw_jb += conj(a_in) dL/da
                    const float2 gwv = cmulc(g_a, ain);
                    atomicAdd(&gwb[jb].x, gwv.x);
                    atomicAdd(&gwb[jb].y, gwv.y);
                } else {
                    g_a = make_float2(0.f, 0.f);
                    gdx = gdy = gdz = 0.f;
                }
            }
        }
        ga[i] = g_a;
        gd[3 * i] = gdx; gd[3 * i + 1] = gdy; gd[3 * i + 2] = gdz;
    }
    __syncthreads();
    // ---- soft path: dL/dlogp_j += sum_i soft_ij (g_y_ij - sum_k soft_ik g_y_ik)
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = warp; i < N; i += RW_THREADS / 32) {
            if (sel[i] < 0) continue;
            const float2 gai = ga[i];
            const float gdi0 = gd[3 * i], gdi1 = gd[3 * i + 1], gdi2 = gd[3 * i + 2];
            if (gai.x == 0.f && gai.y == 0.f && gdi0 == 0.f && gdi1 == 0.f && gdi2 == 0.f) {
                if (pass == 0 && lane == 0) cdot[i] = 0.f;
                continue;
            }
            const float iz = 1.f / zs[i], mxi = mx[i];
            const float ci = pass ? cdot[i] : 0.f;
            float accd = 0.f;
            for (int Gq = lane; Gq * 4 < NB; Gq += 32) {
                float g4[4];
                gumbel_group(sys, stream, i, Gq, g4);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int jb = 4 * Gq + q;
                    if (jb >= NB || !(logp[jb] > -INFINITY)) continue;
                    const float soft = __expf(logp[jb] + g4[q] - mxi) * iz;
                    const int jvi = jb / M, jui = jb - (jb / M) * M;
                    float dx, dy, dz;
                    bin_direction(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz);
                    const float2 U = spectrum_at<M>(X, phu, phv, jui, jvi, norm);
                    const float2 aw = cscale(cmul(ain, U), __expf(EXPO * logp[jb]) / sN);
                    const float gy = gai.x * aw.x + gai.y * aw.y + gdi0 * dx + gdi1 * dy + gdi2 * dz;
                    if (pass == 0) accd += soft * gy;
                    else atomicAdd(&glogp[jb], soft * (gy - ci));
                }
            }
            if (pass == 0) {
                for (int o = 16; o > 0; o >>= 1) accd += __shfl_xor_sync(0xffffffffu, accd, o);
                if (lane == 0) cdot[i] = accd;
            }
        }
        __syncthreads();
    }
    // ---- p = m / S, w = U~ sc(p), m = |U~|^2 or |U~|  ->  dL/dU~  ->  dL/dX
    float sg = 0.f, sgp = 0.f;
    for (int f = threadIdx.x; f < NB; f += RW_THREADS) {
        if (!(logp[f] > -INFINITY)) continue;
        const int jvi = f / M, jui = f - (f / M) * M;
        const float2 U = spectrum_at<M>(X, phu, phv, jui, jvi, norm);
        const float2 w = cscale(U, __expf(EXPO * logp[f]) / sN);
        const float2 gwv = gwb[f];
        // dL/dp from w (times p)
        sgp += EXPO * (gwv.x * w.x + gwv.y * w.y);
        sg += glogp[f];
    }
    const float Sg = block_sum(sg, red);
    const float Sgp = block_sum(sgp, red);
    for (int f = threadIdx.x; f < NB; f += RW_THREADS) {
        const int jvi = f / M, jui = f - (f / M) * M;
        int mu = jui + M / 2; if (mu >= M) mu -= M;
        int mv = jvi + M / 2; if (mv >= M) mv -= M;
        float2 gU = make_float2(0.f, 0.f);
        if (logp[f] > -INFINITY) {
            const float2 U = spectrum_at<M>(X, phu, phv, jui, jvi, norm);
            const float p = __expf(logp[f]);
            const float m = p * S;
            const float isq = __expf(EXPO * logp[f]) / sN;
            const float2 w = cscale(U, isq);
            const float2 gwv = gwb[f];
            const float gp = EXPO * (gwv.x * w.x + gwv.y * w.y) / p;
            // logp = log m - log S ; p = m / S
            const float gm = glogp[f] / m - Sg * iS + gp * iS - Sgp * iS;
            // dm/dU~: 2 U~ (m = |U~|^2), U~ / m (m = |U~|), 0 (uniform: m = 1)
            const float dm = sys.uniform ? 0.f : (COH ? 1.f / m : 2.f);
            gU = make_float2(U.x * dm * gm + gwv.x * isq, U.y * dm * gm + gwv.y * isq);
            if (COH && !sys.conformal) {
                const float im = gU.x * U.y - gU.y * U.x;          // Im(conj(gU) U)
                acc[0] -= sys.kstep * (float)(jui - M / 2) * im;
                acc[1] -= sys.kstep * (float)(jvi - M / 2) * im;
            }
        }
        const float2 ph = cmul(phu[jui], phv[jvi]);
        G[mv * S_ + mu] = cscale(cmulc(gU, ph), norm);
    }
}

// Coherent sensor: reverse of exhaustive bin f; writes its dL/dX.
template <int M>
__device__ __forceinline__ void exh_bin_adjoint_coh(const DSys& sys, const RayAtDoe& R, float k0,
                                                    const float2* X, const float2* phu,
                                                    const float2* phv,
                                                    const float2* __restrict__ gf, float2* G,
                                                    float2 ain, int f, float (&acc)[7],
                                                    float* gs, unsigned* status) {
    const int jvi = f / M, jui = f - (f / M) * M;
    int mu = jui + M / 2; if (mu >= M) mu -= M;
    int mv = jvi + M / 2; if (mv >= M) mv -= M;
    const float norm = sys.norm;
    float2 gU = make_float2(0.f, 0.f);
    float dx, dy, dz;
    if (bin_direction(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz)) {
        const float2 U = spectrum_at<M>(X, phu, phv, jui, jvi, norm);
        const float2 a = cmul(ain, U);
        float2 ga;
        float gx, gy, gz, gdx, gdy, gdz, gopl;
        if (secondary_adjoint_coh(sys, R, k0, gf, dx, dy, dz, a, ga, gx, gy, gz, gdx, gdy, gdz,
                                  gopl, gs, status)) {
            emission_adjoint(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz, gx, gy, gz, gdx, gdy,
                             gdz, acc);
            acc[6] += gopl;
            gU = cmulc(ga, ain);          // conj(a_in) * dL/da
            if (!sys.conformal) {
                const float im = gU.x * U.y - gU.y * U.x;          // Im(conj(gU) U)
                acc[0] -= sys.kstep * (float)(jui - M / 2) * im;
                acc[1] -= sys.kstep * (float)(jvi - M / 2) * im;
            }
        }
    }
    const float2 ph = cmul(phu[jui], phv[jvi]);
    G[mv * Patch<M>::S + mu] = cscale(cmulc(gU, ph), norm);
}

// Reverse of exhaustive bin f of the current incident ray; writes its dL/dX.
template <int M, int NS>
__device__ __forceinline__ void exh_bin_adjoint(const DSys& sys, const RayAtDoe& R,
                                                const float2* X, const float2* phu,
                                                const float2* phv, const float* __restrict__ gimg,
                                                float2* G, float2 ain, int f, float (&acc)[7],
                                                SurfGrads<NS>& SG, float* gs, unsigned* status) {
    const int jvi = f / M, jui = f - (f / M) * M;
    int mu = jui + M / 2; if (mu >= M) mu -= M;
    int mv = jvi + M / 2; if (mv >= M) mv -= M;
    const float norm = sys.norm;
    float2 gU = make_float2(0.f, 0.f);
    float dx, dy, dz;
    if (bin_direction<(NS >= 0)>(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz)) {
        const float2 U = spectrum_at<M>(X, phu, phv, jui, jvi, norm);
        const float2 a = cmul(ain, U);
        const float w = a.x * a.x + a.y * a.y;
        float gw, gx, gy, gz, gdx, gdy, gdz;
        if (secondary_adjoint<NS>(sys, R, gimg, dx, dy, dz, w, gw, gx, gy, gz, gdx, gdy, gdz, SG,
                                  gs, status)) {
            emission_adjoint(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz, gx, gy, gz, gdx, gdy,
                             gdz, acc);
            const float2 ga = make_float2(2.f * a.x * gw, 2.f * a.y * gw);
            gU = cmulc(ga, ain);          // conj(a_in) * dL/da
        }
    }
    // dL/dX[m] = conj(phu phv) norm dL/dU~
    const float2 ph = cmul(phu[jui], phv[jvi]);
    G[mv * Patch<M>::S + mu] = cscale(cmulc(gU, ph), norm);
}

// ------------------------------------------------------------------ kernel
template <int M>
struct BwdOcc { static constexpr int value = M >= 96 ? 1 : 2; };

template <int M, int NS, bool COH>
__global__ void __launch_bounds__(RW_THREADS, BwdOcc<M>::value)
k_backward(const DSys sys, const DJob* __restrict__ jobs, const long long* __restrict__ prefix,
           int njob, long long total, RaysIn rays, const float2* __restrict__ Tmaps,
           const float* __restrict__ amp, const float* __restrict__ gpsf,
           const float2* __restrict__ gfield, float* __restrict__ dphi,
           float* __restrict__ damp, double* __restrict__ dsurf, unsigned* status,
           const unsigned* __restrict__ vis, float* __restrict__ coh_rsum,
           double* __restrict__ coh_jsum) {
    constexpr int NACC = COH ? 7 : 6;     // dL/dP (3), dL/dkappa (2), dL/dK, dL/dOPL
    extern __shared__ __align__(16) unsigned char smem[];
    float2* X = reinterpret_cast<float2*>(smem);
    float2* tw = X + Patch<M>::ELEMS;
    float2* phu = tw + M;
    float2* phv = phu + M;
    RayAtDoe* info = reinterpret_cast<RayAtDoe*>(phv + M);
    float2* G = reinterpret_cast<float2*>(smem + sampled_scratch_offset(M));
    BwdRay* bray = reinterpret_cast<BwdRay*>(G + Patch<M>::ELEMS);
    float* red = reinterpret_cast<float*>(bray + RW_TILE);   // [8 warps][9]
    unsigned char* sscr = reinterpret_cast<unsigned char*>(red + 9 * (RW_THREADS / 32));
    fft_twiddles<M>(tw);
    SurfGrads<NS> SG;
    SG.zero();
    float gs[RW_MAXS * RW_NGRAD];
#pragma unroll
    for (int i = 0; i < RW_MAXS * RW_NGRAD; ++i) gs[i] = 0.f;
    const long long npix_map = (long long)sys.H * sys.W;
    const long long npx = (long long)sys.nx * sys.ny;
    const long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // work unit = (tile, slice of each ray's bins): coherent exhaustive launches split
    // the bins when the tiles cannot fill the GPU (see launch_backward_d)
    const int nslice = (COH && sys.nslice > 1) ? sys.nslice : 1;
    constexpr int CH = M * M / RW_THREADS;
    const int per = COH ? ((CH + nslice - 1) / nslice) * RW_THREADS : M * M;
    for (long long unit = blockIdx.x; unit < ntiles * nslice; unit += gridDim.x) {
        const long long tile = COH ? unit / nslice : unit;
        const int slice = COH ? (int)(unit - tile * nslice) : 0;
        const int f0 = slice * per, f1 = COH ? min(M * M, f0 + per) : M * M;
        __syncthreads();
        if (threadIdx.x < RW_TILE)
            incident_to_doe(sys, jobs, prefix, njob, total, rays, tile * RW_TILE + threadIdx.x,
                            info[threadIdx.x], status);
        __syncthreads();
        for (int r = 0; r < RW_TILE; ++r) {
            const RayAtDoe& R = info[r];
            if (!R.alive) continue;
            const DJob& J = jobs[R.job];
            const float2* T = Tmaps + (long long)J.slot * npix_map;
            gather_patch<M>(sys, R, T, X, phu, phv);
            __syncthreads();
            fft2d<M, false>(X, tw);
            const float2 ain = make_float2(R.a_re, R.a_im);
            const float* gimg = gpsf + (long long)J.out * npx;
            const float2* gf = COH ? gfield + (long long)J.out * npx : nullptr;
            float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (sys.emit == RW_EMIT_EXHAUSTIVE) {
                constexpr int KW = M * M / RW_THREADS;   // visibility words per warp and ray
                if (COH) {
                    if (nslice > 1) {
                        // bins outside the slice contribute nothing to this dL/dX
                        for (int f = threadIdx.x; f < Patch<M>::ELEMS; f += RW_THREADS)
                            G[f] = make_float2(0.f, 0.f);
                        __syncthreads();
                    }
                    for (int f = f0 + threadIdx.x; f < f1; f += RW_THREADS)
                        exh_bin_adjoint_coh<M>(sys, R, J.k0, X, phu, phv, gf, G, ain, f, acc, gs,
                                               status);
                } else if (vis && KW <= 32) {
                    // Only secondary rays that reached the sensor carry gradient: zero
                    // dL/dX, then compact this warp's visible bins (the forward's mask)
                    // and reverse them in converged rounds of 32.
                    for (int f = threadIdx.x; f < Patch<M>::ELEMS; f += RW_THREADS)
                        G[f] = make_float2(0.f, 0.f);
                    __syncthreads();
                    const unsigned* vw = vis + R.gid * (long long)(M * M / 32);
                    const unsigned myw = lane < KW ? __ldg(vw + lane * (RW_THREADS / 32) + warp) : 0u;
                    const int cnt = __popc(myw);
                    int incl = cnt;
                    for (int o = 1; o < 32; o <<= 1) {
                        const int n = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += n;
                    }
                    const int total_w = __shfl_sync(0xffffffffu, incl, 31);
                    const int excl = incl - cnt;
                    for (int start = 0; start < total_w; start += 32) {
                        const int idx = start + lane;
                        int kk = -1, rank = 0;
                        unsigned wsel = 0u;
                        for (int k = 0; k < KW; ++k) {
                            const int ek = __shfl_sync(0xffffffffu, excl, k);
                            const int ck = __shfl_sync(0xffffffffu, cnt, k);
                            const unsigned wk = __shfl_sync(0xffffffffu, myw, k);
                            if (idx >= ek && idx < ek + ck) { kk = k; wsel = wk; rank = idx - ek; }
                        }
                        if (kk >= 0) {
                            const int bit = (int)__fns(wsel, 0u, rank + 1);
                            exh_bin_adjoint<M, NS>(sys, R, X, phu, phv, gimg, G, ain,
                                                   kk * RW_THREADS + warp * 32 + bit, acc, SG,
                                                   gs, status);
                        }
                    }
                } else {
                    for (int f = threadIdx.x; f < M * M; f += RW_THREADS)
                        exh_bin_adjoint<M, NS>(sys, R, X, phu, phv, gimg, G, ain, f, acc, SG, gs,
                                               status);
                }
            } else {
                sampled_ray_adjoint<M, NS, COH>(sys, R, J.k0, R.gid + J.sid, X, phu, phv, gimg,
                                                gf, G, sscr, acc, SG, gs, status);
            }
            // ---- per-ray reduction of the geometric gradients
#pragma unroll
            for (int k = 0; k < NACC; ++k)
                for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
            __syncthreads();
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < NACC; ++k) red[warp * 9 + k] = acc[k];
            __syncthreads();
            if (threadIdx.x == 0) {
                float s[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int w = 0; w < RW_THREADS / 32; ++w)
                    for (int k = 0; k < NACC; ++k) s[k] += red[w * 9 + k];
                BwdRay& B = bray[r];
                B.gpx = s[0]; B.gpy = s[1]; B.gpz = s[2];
                // kappa_in = k0 n_in (d.u, d.v)
                const float kn_in = J.k0 * sys.n_in;
                B.gdx = kn_in * (s[3] * R.u[0] + s[4] * R.v[0]);
                B.gdy = kn_in * (s[3] * R.u[1] + s[4] * R.v[1]);
                B.gdz = kn_in * (s[3] * R.u[2] + s[4] * R.v[2]);
                B.gnin = (R.kin_u * s[3] + R.kin_v * s[4]) / sys.n_in;
                B.gnout = J.k0 * s[5];
                B.gopl = s[6];
                if (COH) {
                    // the incident side runs in k_coh_incident once every ray's
                    // dL/dOPL is known (see there)
                    float* o = coh_rsum + R.gid * 7;
                    if (nslice > 1) {
#pragma unroll
                        for (int k = 0; k < 7; ++k) atomicAdd(o + k, s[k]);   // zeroed by the host
                    } else {
#pragma unroll
                        for (int k = 0; k < 7; ++k) o[k] = s[k];
                    }
                    atomicAdd(coh_jsum + 2 * R.job, (double)s[6]);
                    if (slice == 0) atomicAdd(coh_jsum + 2 * R.job + 1, 1.0);
                }
            }
            // ---- adjoint patch transform and map scatter
            fft2d<M, true>(G, tw);
            map_scatter<M>(sys, R, T, amp, G, J.phase_scale, dphi, damp);
            __syncthreads();
        }
        // ---- incident side: DOE hit and pre-DOE surfaces, one lane per ray
        if (!COH && threadIdx.x < RW_TILE && info[threadIdx.x].alive) {
            const RayAtDoe& R = info[threadIdx.x];
            const BwdRay& B = bray[threadIdx.x];
            const DJob& J = jobs[R.job];
            const long long ri = J.off + (R.gid - prefix[R.job]);
            float x = rays.ox[ri], y = rays.oy[ri], zl = rays.oz[ri];
            float dx = rays.dx[ri], dy = rays.dy[ri], dz = rays.dz[ri];
            double dummy = 0.0;
            SurfIn st[RW_MAXS];
            for (int s = 0; s < sys.doe_index; ++s) {
                st[s].x = x; st[s].y = y; st[s].zl = zl - sys.s[s].gap;
                st[s].dx = dx; st[s].dy = dy; st[s].dz = dz;
                trace_one<false>(sys.s[s], x, y, zl, dx, dy, dz, dummy, status);
            }
            // index gradients of the DOE emission
            if (sys.nout_slot >= 0) gs[sys.nout_slot * RW_NGRAD + 7] += B.gnout;
            if (sys.doe_index > 0) gs[(sys.doe_index - 1) * RW_NGRAD + 7] += B.gnin;
            float gx = B.gpx, gy = B.gpy, gz = B.gpz;
            float gdx = B.gdx, gdy = B.gdy, gdz = B.gdz;
            if (!sys.conformal) {
                // planar DOE hit: h = p + t d, t = (z_doe - p_z) / d_z
                const float zld = zl - sys.s[sys.doe_index].gap;
                const float t = -zld / dz;
                const float gt = gx * dx + gy * dy + gz * dz;
                gdx += gx * t; gdy += gy * t; gdz += gz * t;
                gz += -gt / dz;
                gdz += -gt * t / dz;
                gs[sys.doe_index * RW_NGRAD + 0] += gt / dz;
                for (int s = sys.doe_index - 1; s >= 0; --s) {
                    float gnb = 0.f;
                    trace_one_adjoint(sys.s[s], st[s], gx, gy, gz, gdx, gdy, gdz,
                                      gs + s * RW_NGRAD, &gnb);
                    if (s > 0) gs[(s - 1) * RW_NGRAD + 7] += gnb;
                }
            }
        }
    }
    // ---- CTA reduction of surface-parameter gradients
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
    __syncthreads();
    double* dred = reinterpret_cast<double*>(smem);
    for (int s = 0; s < sys.nsurf; ++s) {
        for (int k = 0; k < RW_NGRAD; ++k) {
            float v = gs[s * RW_NGRAD + k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) dred[(s * RW_NGRAD + k) * (RW_THREADS / 32) + warp] = (double)v;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < sys.nsurf * RW_NGRAD; i += RW_THREADS) {
        double v = 0.0;
        for (int w = 0; w < RW_THREADS / 32; ++w) v += dred[i * (RW_THREADS / 32) + w];
        if (v != 0.0) atomicAdd(dsurf + i, v);
    }
}

// Coherent sensor, incident side.  A global phase of a job's field leaves
// |U|^2 unchanged, so the optical-path gradients of the job's incident rays
// sum to zero; the pre-DOE path derivatives are nearly the same for every
// ray (a lens's thickness, the run to the DOE), so in float the rounding of
// that zero sum, times the common path derivative, would swamp the small
// ray-to-ray differences that carry the gradient.  Every ray's dL/dOPL is
// therefore first reduced per job (k_backward), and here the job mean --
// zero in exact arithmetic -- is subtracted before the incident adjoint.
__global__ void __launch_bounds__(RW_THREADS)
k_coh_incident(const DSys sys, const DJob* __restrict__ jobs, const long long* __restrict__ prefix,
               int njob, long long total, RaysIn rays, const float* __restrict__ rsum,
               const double* __restrict__ jsum, double* __restrict__ dsurf, unsigned* status) {
    __shared__ double dred[RW_MAXS * RW_NGRAD * (RW_THREADS / 32)];
    float gs[RW_MAXS * RW_NGRAD];
#pragma unroll
    for (int i = 0; i < RW_MAXS * RW_NGRAD; ++i) gs[i] = 0.f;
    for (long long g = blockIdx.x * (long long)RW_THREADS + threadIdx.x; g < total;
         g += (long long)gridDim.x * RW_THREADS) {
        RayAtDoe R;
        incident_to_doe(sys, jobs, prefix, njob, total, rays, g, R, status);
        if (!R.alive) continue;
        float s[7];
#pragma unroll
        for (int k = 0; k < 7; ++k) s[k] = rsum[g * 7 + k];
        const double n = jsum[2 * R.job + 1];
        const float gopl = n > 0.0 ? (float)((double)s[6] - jsum[2 * R.job] / n) : s[6];
        incident_adjoint<true>(sys, jobs, prefix, rays, R, s, gs, status, gopl);
    }
    reduce_surface_grads(sys, gs, dred, dsurf);
}

inline size_t backward_smem_bytes(int M, int emit, int n_ssr) {
    size_t b = sampled_scratch_offset(M) + sizeof(float2) * (size_t)M * (M + 2) +
               sizeof(BwdRay) * RW_TILE + sizeof(float) * 9 * (RW_THREADS / 32);
    if (emit == RW_EMIT_SAMPLED) b += sampled_bwd_bytes(M, n_ssr);
    size_t red = sizeof(double) * RW_MAXS * RW_NGRAD * (RW_THREADS / 32);
    return b > red ? b : red;
}

size_t backward_smem_needed(const DSys& sys) { return backward_smem_bytes(sys.M, sys.emit, sys.n_ssr); }

template <int M, int NS, bool COH = false>
static cudaError_t launch_backward_d(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                                     const long long* prefix, int njob, long long total,
                                     const RaysIn& rays, const float2* T, const float* amp,
                                     const float* gpsf, const float2* gfield, float* dphi,
                                     float* damp, double* dsurf, unsigned* status,
                                     const unsigned* vis, float* coh_rsum = nullptr,
                                     double* coh_jsum = nullptr) {
    const size_t smem = backward_smem_bytes(M, sys.emit, sys.n_ssr);
    auto kern = k_backward<M, NS, COH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RW_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    long long grid = (long long)L.num_sms * per_sm;
    grid = pick_grid(L, RW_K_BACKWARD, grid);
    // coherent exhaustive: split each ray's bins when the tiles cannot fill the GPU
    DSys s = sys;
    s.nslice = 1;
    if (COH && sys.emit == RW_EMIT_EXHAUSTIVE && ntiles < grid) {
        const long long want = (grid + ntiles - 1) / ntiles;
        const long long most = (long long)M * M / RW_THREADS;
        s.nslice = (int)(want < most ? want : most);
    }
    if (grid > ntiles * s.nslice) grid = ntiles * s.nslice;
    if (grid < 1) grid = 1;
    RW_MARK(L, "k_backward");
    kern<<<(unsigned)grid, RW_THREADS, smem, L.stream>>>(s, jobs, prefix, njob, total, rays, T,
                                                          amp, gpsf, gfield, dphi, damp, dsurf,
                                                          status, vis, coh_rsum, coh_jsum);
    RW_MARK(L, nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess || !COH || !dsurf) return e;
    long long g2 = (total + RW_THREADS - 1) / RW_THREADS;
    const long long cap = (long long)L.num_sms * 4;
    if (g2 > cap) g2 = cap;
    if (g2 < 1) g2 = 1;
    RW_MARK(L, "k_coh_incident");
    k_coh_incident<<<(unsigned)g2, RW_THREADS, 0, L.stream>>>(sys, jobs, prefix, njob, total, rays,
                                                               coh_rsum, coh_jsum, dsurf, status);
    RW_MARK(L, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_backward(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                            const long long* prefix, int njob, long long total,
                            const RaysIn& rays, const float2* T, const float* amp,
                            const float* dl_dpsf, const float2* gfield, float* coh_rsum,
                            double* coh_jsum, float* dphi, float* damp, double* dsurf,
                            const unsigned* vis, unsigned* status, int* launches) {
    *launches = 1;
    const int ns = sys.fast_ok ? sys.n_post : -1;
    if (sys.coherent) {
        // the coherent sum needs each ray's optical path: generic trace only
        if (!gfield || !coh_rsum || !coh_jsum) return cudaErrorInvalidValue;
        if (dsurf) *launches = 2;
#define RW_BWD_COH(DD)                                                                          \
    case DD:                                                                                    \
        return launch_backward_d<DD, -1, true>(L, sys, jobs, prefix, njob, total, rays, T, amp, \
                                               dl_dpsf, gfield, dphi, damp, dsurf, status,      \
                                               nullptr, coh_rsum, coh_jsum);
        switch (sys.M) {
            RW_BWD_COH(16)
            RW_BWD_COH(32)
            RW_BWD_COH(64)
            RW_BWD_COH(96)
            default: return cudaErrorInvalidValue;
        }
#undef RW_BWD_COH
    }
#define RW_BWD(DD, NN) \
    launch_backward_d<DD, NN>(L, sys, jobs, prefix, njob, total, rays, T, amp, dl_dpsf, nullptr, dphi, damp, dsurf, status, vis)
#define RW_BWD_D(DD)                                      \
    case DD:                                              \
        switch (ns) {                                     \
            case 0: return RW_BWD(DD, 0);                 \
            case 2: return RW_BWD(DD, 2);                 \
            case 4: return RW_BWD(DD, 4);                 \
            case 6: return RW_BWD(DD, 6);                 \
            default: return RW_BWD(DD, -1);               \
        }
    switch (sys.M) {
        RW_BWD_D(16)
        RW_BWD_D(32)
        RW_BWD_D(64)
        RW_BWD_D(96)
        default: return cudaErrorInvalidValue;
    }
#undef RW_BWD_D
#undef RW_BWD
}
