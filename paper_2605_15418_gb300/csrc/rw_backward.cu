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
// Shared scratch of the sampled adjoint (after the patch, the tile's incident
// states and the per-ray reduction buffers; dL/dX overwrites X in place):
//   rec[M*M]  float2: (p_j, kn_j), later (p_j, dL/dlog p_j)
//   sel[N]    chosen bin per draw
//   sa[N], sb[N] float4, sc2[N] float2: per-draw sums, then h~ and c~
//   hU[N]     float2: hard-path dL/dU~ of the draw's bin
//   red[64]
__host__ __device__ inline size_t sampled_bwd_bytes(int M, int N) {
    const size_t n4 = ((size_t)N + 3) & ~size_t(3);
    return (size_t)M * M * 8 + n4 * 4 + (size_t)N * (16 + 16 + 8 + 8) + 64 * 4;
}

// Block-wide sum (all threads get the result); `red` holds >= 8 floats.
__device__ __forceinline__ float block_sum(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    main_sync();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    main_sync();
    float t = 0.f;
    for (int w = 0; w < RW_THREADS / 32; ++w) t += red[w];
    return t;
}

// X[.] position of bin f (natural order) in the FFT output (row stride M + 1).
template <int M>
__device__ __forceinline__ int xpos(int f) {
    const int jvi = f / M, jui = f - (f / M) * M;
    int mu = jui + M / 2; if (mu >= M) mu -= M;
    int mv = jvi + M / 2; if (mv >= M) mv -= M;
    return mv * Patch<M>::S + mu;
}

// Pass A of the sampled adjoint (see sampled_ray_adjoint): lane = draw, the
// warp's 32 draws walk the bins in step (per-bin records and weights are
// broadcast reads), two Philox blocks per step; the t-weighted sums are
// straight-line code and the rare screening candidates are scored after
// them.  Every thread of the block takes part (helper warps included).  Not
// inlined, so that the loop has registers of its own.
template <int M>
__device__ __noinline__ void gumbel_pass_a(const float2* __restrict__ rec,
                                           const float2* __restrict__ X, int* __restrict__ sel,
                                           float4* __restrict__ sa, float4* __restrict__ sb,
                                           int N, uint32_t ray, uint32_t off, uint32_t k0,
                                           uint32_t k1) {
    constexpr int NG = M * M / 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i0 = warp * 32; i0 < N; i0 += (int)blockDim.x) {
        const uint32_t i = (uint32_t)(i0 + lane);
        float Z = 0.f, Su = 0.f, Sv = 0.f, Sn = 0.f, Sr = 0.f, Si = 0.f;
        float best = -INFINITY;
        int bj = 0x7fffffff;
        for (int G = 0; G < NG; G += 2) {
            const uint4 wa = philox4x32_10(make_uint4((uint32_t)G, i, ray, off), k0, k1);
            const uint4 wb = philox4x32_10(make_uint4((uint32_t)G + 1u, i, ray, off), k0, k1);
            const uint32_t ws[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
            const int f0 = 4 * G;                       // 8 bins of one row (8 | M)
            const int jv = f0 / M, ju0 = f0 - jv * M;
            const int xb = xpos<M>(f0);
            float z8 = 0.f, zq = 0.f;
            unsigned mask = 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float2 pk = rec[f0 + q];
                const float2 wt = X[xb + q];
                const float E = gumbel_E_fast(ws[q]);
                const float t = pk.x * rcp_approx(E);
                z8 += t;
                zq = fmaf((float)q, t, zq);
                Sn = fmaf(t, pk.y, Sn);
                Sr = fmaf(t, wt.x, Sr);
                Si = fmaf(t, wt.y, Si);
                // a bin that cannot be drawn (p = 0) passes only when E < 1e-6
                // and then scores -inf, which never wins
                mask |= (unsigned)(E < fmaf(RW_GUMBEL_TAU * 1.001f, pk.x, 1e-6f)) << q;
            }
            Z += z8;
            Su += fmaf((float)(ju0 - M / 2), z8, zq);
            Sv = fmaf((float)(jv - M / 2), z8, Sv);
            if (mask) {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if ((mask >> q) & 1u)
                        gumbel_keep(gumbel_score(rec[f0 + q].x, ws[q]), f0 + q, best, bj);
            }
        }
        if ((int)i < N) {
            if (!(best > RW_GUMBEL_FLOOR)) {
                best = -INFINITY;
                bj = 0x7fffffff;
                gumbel_full_scan<M, 2>(reinterpret_cast<const float*>(rec), i, ray, off, k0, k1,
                                       best, bj);
            }
            sel[i] = best > -INFINITY ? bj : -1;
            sa[i] = make_float4(Z, Su, Sv, Sn);
            sb[i] = make_float4(Sr, Si, 0.f, 0.f);
        }
    }
}

constexpr int lanes_per_group(int ng, int nt) {
    for (int ks = 1; ks <= 32; ks *= 2)
        if ((ng * ks) % nt == 0) return ks;
    return ng < nt ? nt / ng : 1;
}

// Pass B of the sampled adjoint: a lane owns a group of 4 bins (KS lanes
// share one when there are fewer groups than threads) and walks the draws,
// two Philox blocks per step, accumulating e_ij h~_i and e_ij c~_i; then
// recf[2 j + 1] = dL/dlog p_j.  Not inlined, like pass A.
template <int M, int NT>
__device__ __noinline__ void gumbel_pass_b(float* __restrict__ recf, const float2* __restrict__ X,
                                           const int* __restrict__ sel,
                                           const float4* __restrict__ sa,
                                           const float2* __restrict__ sc2, int N, uint32_t ray,
                                           uint32_t off, uint32_t k0, uint32_t k1, float kin_u,
                                           float kin_v, float ks) {
    constexpr int NG = M * M / 4;
    // lanes per bin group (they split the draws): the fewest that give all NT
    // threads the same number of groups
    constexpr int KS = lanes_per_group(NG, NT);
    static_assert(KS <= 32 && (KS & (KS - 1)) == 0, "lanes per group: a power of two <= 32");
    for (int tt = threadIdx.x; tt < NG * KS; tt += NT) {
        const int G = tt / KS, s0 = tt - (tt / KS) * KS;
        float a4[4][6];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 6; ++k) a4[q][k] = 0.f;
        // draws whose bin is -1 carry h~ = c~ = 0: no test needed; four Philox
        // blocks (four draws) per step
        int i = s0;
        for (; i + 3 * KS < N; i += 4 * KS) {
            uint4 w[4];
            float4 h[4];
            float2 h2[4];
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                w[d] = philox4x32_10(make_uint4((uint32_t)G, (uint32_t)(i + d * KS), ray, off),
                                     k0, k1);
                h[d] = sa[i + d * KS];
                h2[d] = sc2[i + d * KS];
            }
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const uint32_t ws[4] = {w[d].x, w[d].y, w[d].z, w[d].w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float e = rcp_approx(gumbel_E_fast(ws[q]));
                    a4[q][0] = fmaf(e, h[d].x, a4[q][0]);
                    a4[q][1] = fmaf(e, h[d].y, a4[q][1]);
                    a4[q][2] = fmaf(e, h[d].z, a4[q][2]);
                    a4[q][3] = fmaf(e, h[d].w, a4[q][3]);
                    a4[q][4] = fmaf(e, h2[d].x, a4[q][4]);
                    a4[q][5] = fmaf(e, h2[d].y, a4[q][5]);
                }
            }
        }
        for (; i < N; i += KS) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)G, (uint32_t)i, ray, off), k0, k1);
            const float4 h = sa[i];
            const float2 h2 = sc2[i];
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float e = rcp_approx(gumbel_E_fast(ws[q]));
                a4[q][0] = fmaf(e, h.x, a4[q][0]);
                a4[q][1] = fmaf(e, h.y, a4[q][1]);
                a4[q][2] = fmaf(e, h.z, a4[q][2]);
                a4[q][3] = fmaf(e, h.w, a4[q][3]);
                a4[q][4] = fmaf(e, h2.x, a4[q][4]);
                a4[q][5] = fmaf(e, h2.y, a4[q][5]);
            }
        }
        if (KS > 1) {
#pragma unroll
            for (int o = 1; o < KS; o <<= 1)
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int k = 0; k < 6; ++k)
                        a4[q][k] += __shfl_xor_sync(0xffffffffu, a4[q][k], o);
        }
        if (s0 == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int f = 4 * G + q;
                const int jvi = f / M, jui = f - (f / M) * M;
                const float pj = recf[2 * f];
                float gl = 0.f;
                if (pj > 0.f) {
                    const float2 w = X[xpos<M>(f)];
                    const float ku = kin_u + ks * (float)(jui - M / 2);
                    const float kv = kin_v + ks * (float)(jvi - M / 2);
                    gl = pj * (a4[q][0] * w.x + a4[q][1] * w.y + a4[q][2] * ku + a4[q][3] * kv +
                               a4[q][4] * recf[2 * f + 1] - a4[q][5]);
                }
                recf[2 * f + 1] = gl;
            }
        }
    }
}

// Straight-through Gumbel-softmax adjoint of one incident ray (temperature 1).
// Draw i's relaxed one-hot is soft_ij = t_ij / Z_i with t_ij = p_j / E_ij,
// E_ij = -log u_ij (exp of the perturbed score log p_j + g_ij) and
// Z_i = sum_j t_ij.  With G_ij = dL/dy_ij = Re(conj(q_i) w_j) + gd_i . dir_j
// (q_i = conj(a_in) dL/da_i, w_j = U~_j sc(p_j) the bin's weight, gd_i = dL/dd_i)
// the softmax Jacobian gives
//   dL/dlog p_j = sum_i soft_ij (G_ij - c_i),   c_i = sum_k soft_ik G_ik,
// and because G is bilinear in (q_i, gd_i) and (w_j, dir_j), with
// dir_j = (kappa_u u + kappa_v v + kn_j n) / K and kappa affine in the bin
// index, both sums are two passes of six accumulators over the (draw, bin)
// pairs:
//   pass A, per draw (the 32 lanes of a warp are 32 draws walking the bins
//     in step): Z_i and the t-weighted sums of j_u, j_v, kn_j, w_j -> c_i,
//     together with the screened argmax (the forward's draw);
//   pass B, per bin (a lane owns 4 bins and walks the draws):
//     H_j = sum_i e_ij h~_i and C_j = sum_i e_ij c~_i, e = 1/E,
//     h~_i = (q_i, gd_i.u/K, gd_i.v/K, gd_i.n/K) / Z_i, c~_i = c_i / Z_i,
//     dL/dlog p_j = p_j (<H_j, (w_j, kappa_u, kappa_v, kn_j)> - C_j).
// No soft value is stored and no atomic is issued per pair.
// Shared scratch of sampled_ray_adjoint after the patch (also read by the
// helper warps of k_backward).
struct SampledScr {
    float2* rec;     // [M*M] (p_j, kn_j); .y becomes dL/dlog p_j after pass B
    int* sel;        // [n_ssr] the forward's bin of each draw
    float4* sa;      // [n_ssr] pass A sums (Z, S_u, S_v, S_n), then h~
    float4* sb;      // [n_ssr] pass A sums of w (re, im)
    float2* sc2;     // [n_ssr] (h~_n, c~)
    float2* hU;      // [n_ssr] hard-path dL/dU~ of the draw's bin
    float* red;      // block reductions
    __device__ SampledScr(unsigned char* scr, int NB, int N) {
        rec = reinterpret_cast<float2*>(scr);
        sel = reinterpret_cast<int*>(rec + NB);
        sa = reinterpret_cast<float4*>(sel + ((N + 3) & ~3));
        sb = sa + N;
        sc2 = reinterpret_cast<float2*>(sb + N);
        hU = sc2 + N;
        red = reinterpret_cast<float*>(hU + N);
    }
};

// Barriers: the four marked "CTA" are taken by every thread of the block
// (helper warps included, see sampled_helpers); the rest by the main threads.
template <int M, int NS, bool COH, int NT>
__device__ __forceinline__ void sampled_ray_adjoint(const DSys& sys, const RayAtDoe& R,
                                                    float k0, long long stream,
                                                    float2* X, const float2* phu,
                                                    const float2* phv,
                                                    const float* __restrict__ gimg,
                                                    const float2* __restrict__ gf,
                                                    unsigned char* scr, float* acc,
                                                    SurfGrads<NS>& SG, float* gs,
                                                    unsigned* status) {
    constexpr int NB = M * M;
    constexpr int NG = NB / 4;
    constexpr int S_ = Patch<M>::S;
    const int N = sys.n_ssr;
    const float norm = sys.norm;
    const SampledScr P(scr, NB, N);
    float2* rec = P.rec;
    float* recf = reinterpret_cast<float*>(rec);
    int* sel = P.sel;
    float4* sa = P.sa;
    float4* sb = P.sb;
    float2* sc2 = P.sc2;
    float2* hU = P.hU;
    float* red = P.red;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float2 ain = make_float2(R.a_re, R.a_im);
    const float sN = COH ? (float)N : sqrtf((float)N);
    constexpr float EXPO = COH ? -1.f : -0.5f;       // d log sc / d log p
    // ---- p_j (shared with the forward), kn_j, and X <- w~_j = U~_j sc(p_j) in place
    const float S = sampled_probs<M, 2>(sys, R, X, phu, phv, recf, red);
    const float iS = S > 0.f ? 1.f / S : 0.f;
    for (int f = threadIdx.x; f < NB; f += RW_THREADS) {
        const int jvi = f / M, jui = f - (f / M) * M;
        const float pj = recf[2 * f];
        const float ku = R.kin_u + sys.kstep * (float)(jui - M / 2);
        const float kv = R.kin_v + sys.kstep * (float)(jvi - M / 2);
        const float kt2 = ku * ku + kv * kv, K2 = R.K * R.K;
        recf[2 * f + 1] = kt2 < K2 ? sqrtf(K2 - kt2) : 0.f;
        float2 w = make_float2(0.f, 0.f);
        if (pj > 0.f) {
            const float sc = COH ? 1.f / (N * pj) : rsqrtf(N * pj);
            w = cscale(spectrum_at<M>(X, phu, phv, jui, jvi, norm), sc);
        }
        X[xpos<M>(f)] = w;
    }
    __syncthreads();                                               // CTA
    const uint32_t k0w = (uint32_t)(sys.seed & 0xffffffffull), k1w = (uint32_t)(sys.seed >> 32);
    const uint32_t ray = (uint32_t)stream, off = (uint32_t)sys.rng_offset;
    // ---- pass A: per draw, the forward's screened argmax and the t-weighted sums
    gumbel_pass_a<M>(rec, X, sel, sa, sb, N, ray, off, k0w, k1w);
    __syncthreads();                                               // CTA
    // ---- every draw: trace + reverse of its (hard) secondary ray; h~, c~ and
    // the hard path's dL/dU~ of its bin
    const float ks = sys.kstep;
    float sgp = 0.f;
    for (int i = threadIdx.x; i < N; i += RW_THREADS) {
        const int jb = sel[i];
        float2 q = make_float2(0.f, 0.f);
        float gdx = 0.f, gdy = 0.f, gdz = 0.f;
        float2 hu = make_float2(0.f, 0.f);
        if (jb >= 0) {
            const int jvi = jb / M, jui = jb - (jb / M) * M;
            float dx, dy, dz;
            if (bin_direction(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz)) {
                const float2 w = X[xpos<M>(jb)];
                const float2 a = cmul(ain, w);
                float2 g_a = make_float2(0.f, 0.f);
                float gx, gy, gz;
                bool hit;
                if constexpr (COH) {
                    float gopl;
                    hit = secondary_adjoint_coh(sys, R, k0, gf, dx, dy, dz, a, g_a, gx, gy, gz,
                                                gdx, gdy, gdz, gopl, gs, status);
                    if (hit) acc[6] += gopl;
                } else {
                    const float wi = a.x * a.x + a.y * a.y;
                    float gw;
                    hit = secondary_adjoint<NS>(sys, R, gimg, dx, dy, dz, wi, gw, gx, gy, gz, gdx,
                                                gdy, gdz, SG, gs, status);
                    if (hit) g_a = make_float2(2.f * a.x * gw, 2.f * a.y * gw);
                }
                if (hit) {
                    emission_adjoint(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz, gx, gy, gz,
                                     gdx, gdy, gdz, acc);
                    // hard path: a = a_in w_jb  ->  dL/dw_jb = conj(a_in) dL/da
                    q = cmulc(g_a, ain);
                    const float pj = recf[2 * jb];
                    const float sc = COH ? 1.f / (N * pj) : rsqrtf(N * pj);
                    const float2 U = cscale(w, 1.f / sc);
                    const float gpw = EXPO * (q.x * w.x + q.y * w.y);   // dL/dlog p via sc(p)
                    sgp += gpw;
                    const float dm = sys.uniform ? 0.f : (COH ? 1.f / (pj * S) : 2.f);
                    const float gm = gpw / pj * iS;
                    hu = make_float2(U.x * dm * gm + q.x * sc, U.y * dm * gm + q.y * sc);
                    if (COH && !sys.conformal) {
                        const float im = hu.x * U.y - hu.y * U.x;          // Im(conj(gU) U)
                        acc[0] -= ks * (float)(jui - M / 2) * im;
                        acc[1] -= ks * (float)(jvi - M / 2) * im;
                    }
                } else {
                    gdx = gdy = gdz = 0.f;
                }
            }
        }
        const float4 A = sa[i];
        const float Z = jb >= 0 ? A.x : 0.f;
        float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 h2 = make_float2(0.f, 0.f);
        if (jb >= 0 && Z > 0.f) {
            const float2 B = make_float2(sb[i].x, sb[i].y);
            const float gdu = gdx * R.u[0] + gdy * R.u[1] + gdz * R.u[2];
            const float gdv = gdx * R.v[0] + gdy * R.v[1] + gdz * R.v[2];
            const float gdn = gdx * R.n[0] + gdy * R.n[1] + gdz * R.n[2];
            const float iZ = 1.f / Z, iK = R.invK;
            const float zc = q.x * B.x + q.y * B.y +
                             (gdu * fmaf(ks, A.y, R.kin_u * Z) + gdv * fmaf(ks, A.z, R.kin_v * Z) +
                              gdn * A.w) * iK;
            h = make_float4(q.x * iZ, q.y * iZ, gdu * iK * iZ, gdv * iK * iZ);
            h2 = make_float2(gdn * iK * iZ, zc * iZ * iZ);
        }
        sa[i] = h;
        sc2[i] = h2;
        hU[i] = hu;
    }
    const float Sgp = block_sum(sgp, red);
    // ---- pass B: per bin, the draws' softmax weights against h~ and c~ (the
    // uniform density does not depend on U~: no soft path)
    __syncthreads();                                               // CTA
    if (!sys.uniform)
        gumbel_pass_b<M, NT>(recf, X, sel, sa, sc2, N, ray, off, k0w, k1w, R.kin_u, R.kin_v, ks);
    __syncthreads();                                               // CTA
    float sg = 0.f;
    if (!sys.uniform)
        for (int f = threadIdx.x; f < NB; f += RW_THREADS) sg += recf[2 * f + 1];
    const float Sg = block_sum(sg, red);
    // ---- soft chain p = m / S, m = |U~|^2 (|U~| coherent, 1 uniform) -> dL/dU~,
    // written as dL/dX = conj(phase) norm dL/dU~ over X in place
    for (int f = threadIdx.x; f < NB; f += RW_THREADS) {
        const int jvi = f / M, jui = f - (f / M) * M;
        const int xp = xpos<M>(f);
        const float pj = recf[2 * f];
        float2 gU = make_float2(0.f, 0.f);
        if (pj > 0.f && !sys.uniform) {
            const float sc = COH ? 1.f / (N * pj) : rsqrtf(N * pj);
            const float2 U = cscale(X[xp], 1.f / sc);
            const float m = pj * S;
            const float gm = recf[2 * f + 1] / m - (Sg + Sgp) * iS;
            const float dm = COH ? 1.f / m : 2.f;
            gU = make_float2(U.x * dm * gm, U.y * dm * gm);
            if (COH && !sys.conformal) {
                const float im = gU.x * U.y - gU.y * U.x;
                acc[0] -= ks * (float)(jui - M / 2) * im;
                acc[1] -= ks * (float)(jvi - M / 2) * im;
            }
        }
        const float2 ph = cmul(phu[jui], phv[jvi]);
        X[xp] = cscale(cmulc(gU, ph), norm);
    }
    main_sync();
    // ---- hard path of every draw into its bin
    for (int i = threadIdx.x; i < N; i += RW_THREADS) {
        const int jb = sel[i];
        const float2 hu = hU[i];
        if (jb < 0 || (hu.x == 0.f && hu.y == 0.f)) continue;
        const int jvi = jb / M, jui = jb - (jb / M) * M;
        const float2 ph = cmul(phu[jui], phv[jvi]);
        const float2 gx = cscale(cmulc(hu, ph), norm);
        float2* dst = X + xpos<M>(jb);
        atomicAdd(&dst->x, gx.x);
        atomicAdd(&dst->y, gx.y);
    }
    main_sync();
}

// Coherent sensor: reverse of exhaustive bin f; writes its dL/dX.
template <int M>
__device__ __forceinline__ void exh_bin_adjoint_coh(const DSys& sys, const RayAtDoe& R, float k0,
                                                    const float2* X, const float2* phu,
                                                    const float2* phv,
                                                    const float2* __restrict__ gf, float2* G,
                                                    float2 ain, int f, float (&acc)[RW_RS],
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
                                                float2* G, float2 ain, int f, float (&acc)[RW_RS],
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

// Helper warps of the sampled adjoint: threads RW_THREADS.. of the block.
// They walk the same tiles and rays as the main threads, meet them at the
// CTA barriers (tile start, and around the two Gumbel passes of every live
// ray) and run their share of the passes, whose (draw, bin) pairs are nearly
// all of the sampled adjoint's work; everything else is left to the main
// threads.  More warps on an SM hide the passes' dependent-latency stalls.
template <int M, int NT>
__device__ __noinline__ void sampled_helpers(const DSys& sys, long long total,
                                             const RayAtDoe* info, float2* X,
                                             unsigned char* sscr) {
    constexpr int NB = M * M;
    const int N = sys.n_ssr;
    const SampledScr P(sscr, NB, N);
    const uint32_t k0w = (uint32_t)(sys.seed & 0xffffffffull), k1w = (uint32_t)(sys.seed >> 32);
    const uint32_t off = (uint32_t)sys.rng_offset;
    const long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();                     // CTA: tile start
        __syncthreads();                     // CTA: the tile's rays are at the DOE
        for (int r = 0; r < RW_TILE; ++r) {
            const RayAtDoe& R = info[r];
            if (!R.alive) continue;
            const uint32_t ray = (uint32_t)R.rid;
            __syncthreads();                 // CTA: p_j, kn_j and w~_j ready
            gumbel_pass_a<M>(P.rec, X, P.sel, P.sa, P.sb, N, ray, off, k0w, k1w);
            __syncthreads();                 // CTA: pass A done
            __syncthreads();                 // CTA: h~ and c~ ready
            if (!sys.uniform)
                gumbel_pass_b<M, NT>(reinterpret_cast<float*>(P.rec), X, P.sel, P.sa, P.sc2, N,
                                     ray, off, k0w, k1w, R.kin_u, R.kin_v, sys.kstep);
            __syncthreads();                 // CTA: pass B done
        }
    }
}

// HW helper warps (sampled emission only, see sampled_helpers); HW = 0 is
// the plain kernel.
template <int M, int NS, bool COH, int HW = 0>
__global__ void __launch_bounds__(RW_THREADS + 32 * HW, BwdOcc<M>::value)
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
    // sampled emission writes dL/dX over X in place; exhaustive keeps X and dL/dX apart
    const bool smp = sys.emit != RW_EMIT_EXHAUSTIVE;
    float2* G = smp ? X : reinterpret_cast<float2*>(smem + sampled_scratch_offset(M));
    BwdRay* bray = reinterpret_cast<BwdRay*>(smem + sampled_scratch_offset(M) +
                                             (smp ? 0 : sizeof(float2) * Patch<M>::ELEMS));
    float* red = reinterpret_cast<float*>(bray + RW_TILE);   // [8 warps][RW_RS]
    unsigned char* sscr = reinterpret_cast<unsigned char*>(red + RW_RS * (RW_THREADS / 32));
    if constexpr (HW > 0) {
        if (threadIdx.x >= RW_THREADS) {
            sampled_helpers<M, RW_THREADS + 32 * HW>(sys, total, info, X, sscr);
            return;
        }
    }
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
        __syncthreads();                                           // CTA
        if (threadIdx.x < RW_TILE)
            incident_to_doe(sys, jobs, prefix, njob, total, rays, tile * RW_TILE + threadIdx.x,
                            info[threadIdx.x], status);
        __syncthreads();                                           // CTA
        for (int r = 0; r < RW_TILE; ++r) {
            const RayAtDoe& R = info[r];
            if (!R.alive) continue;
            const DJob& J = jobs[R.job];
            const float2* T = Tmaps + (long long)J.slot * npix_map;
            gather_patch<M>(sys, R, T, X, phu, phv);
            main_sync();
            fft2d<M, false>(X, tw);
            const float2 ain = make_float2(R.a_re, R.a_im);
            const float* gimg = gpsf + (long long)J.out * npx;
            const float2* gf = COH ? gfield + (long long)J.out * npx : nullptr;
            float acc[RW_RS];
#pragma unroll
            for (int k = 0; k < RW_RS; ++k) acc[k] = 0.f;
            if (sys.emit == RW_EMIT_EXHAUSTIVE) {
                constexpr int KW = M * M / RW_THREADS;   // visibility words per warp and ray
                if (COH) {
                    if (nslice > 1) {
                        // bins outside the slice contribute nothing to this dL/dX
                        for (int f = threadIdx.x; f < Patch<M>::ELEMS; f += RW_THREADS)
                            G[f] = make_float2(0.f, 0.f);
                        main_sync();
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
                    main_sync();
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
                sampled_ray_adjoint<M, NS, COH, RW_THREADS + 32 * HW>(
                    sys, R, J.k0, R.rid, X, phu, phv, gimg, gf, sscr, acc, SG, gs, status);
            }
            // ---- per-ray reduction of the geometric gradients (with a conformal
            // DOE also the frame sums)
            const int nk = sys.conformal ? RW_RS_GATHER : NACC;
#pragma unroll
            for (int k = 0; k < RW_RS_GATHER; ++k)
                if (k < nk)
                    for (int o = 16; o > 0; o >>= 1)
                        acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
            main_sync();
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < RW_RS_GATHER; ++k)
                    if (k < nk) red[warp * RW_RS + k] = acc[k];
            main_sync();
            if (threadIdx.x == 0) {
                float* sb = bray[r].s;
                for (int k = 0; k < RW_RS; ++k) sb[k] = 0.f;
                for (int w = 0; w < RW_THREADS / 32; ++w)
                    for (int k = 0; k < nk; ++k) sb[k] += red[w * RW_RS + k];
                if (COH) {
                    // the incident side runs in k_coh_incident once every ray's
                    // dL/dOPL is known (see there)
                    float* o = coh_rsum + R.gid * sys.nrs;
                    if (nslice > 1) {
                        for (int k = 0; k < nk; ++k) atomicAdd(o + k, sb[k]);   // zeroed by the host
                    } else {
                        for (int k = 0; k < nk; ++k) o[k] = sb[k];
                    }
                    atomicAdd(coh_jsum + 2 * R.job, (double)sb[6]);
                    if (slice == 0) atomicAdd(coh_jsum + 2 * R.job + 1, 1.0);
                }
            }
            // ---- adjoint patch transform and map scatter (with a conformal DOE
            // also the gradient of the patch sample positions)
            fft2d<M, true>(G, tw);
            float gq[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            map_scatter<M>(sys, R, T, amp, G, J.phase_scale, dphi, damp,
                           sys.conformal ? gq : nullptr);
            if (sys.conformal) {
#pragma unroll
                for (int k = 0; k < 6; ++k)
                    for (int o = 16; o > 0; o >>= 1) gq[k] += __shfl_xor_sync(0xffffffffu, gq[k], o);
                main_sync();
                if (lane == 0)
#pragma unroll
                    for (int k = 0; k < 6; ++k) red[warp * RW_RS + k] = gq[k];
                main_sync();
                if (threadIdx.x == 0) {
                    float* sb = bray[r].s;
                    for (int k = 0; k < 6; ++k) {
                        float v = 0.f;
                        for (int w = 0; w < RW_THREADS / 32; ++w) v += red[w * RW_RS + k];
                        sb[RW_RS_GATHER + k] = v;
                        if (COH) {
                            float* o = coh_rsum + R.gid * sys.nrs + RW_RS_GATHER + k;
                            if (nslice > 1) atomicAdd(o, v); else *o = v;
                        }
                    }
                }
            }
            main_sync();
        }
        // ---- incident side: DOE hit and pre-DOE surfaces, one lane per ray
        if (!COH && threadIdx.x < RW_TILE && info[threadIdx.x].alive)
            incident_adjoint(sys, jobs, prefix, rays, info[threadIdx.x], bray[threadIdx.x].s, gs,
                             status);
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
    main_sync();
    double* dred = reinterpret_cast<double*>(smem);
    for (int s = 0; s < sys.nsurf; ++s) {
        for (int k = 0; k < RW_NGRAD; ++k) {
            float v = gs[s * RW_NGRAD + k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) dred[(s * RW_NGRAD + k) * (RW_THREADS / 32) + warp] = (double)v;
        }
    }
    main_sync();
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
        float s[RW_RS];
#pragma unroll
        for (int k = 0; k < RW_RS; ++k) s[k] = k < sys.nrs ? rsum[g * sys.nrs + k] : 0.f;
        const double n = jsum[2 * R.job + 1];
        const float gopl = n > 0.0 ? (float)((double)s[6] - jsum[2 * R.job] / n) : s[6];
        incident_adjoint<true>(sys, jobs, prefix, rays, R, s, gs, status, gopl);
    }
    reduce_surface_grads(sys, gs, dred, dsurf);
}

inline size_t backward_smem_bytes(int M, int emit, int n_ssr) {
    size_t b = sampled_scratch_offset(M) + sizeof(BwdRay) * RW_TILE +
               sizeof(float) * RW_RS * (RW_THREADS / 32);
    if (emit == RW_EMIT_SAMPLED) b += sampled_bwd_bytes(M, n_ssr);   // dL/dX over X
    else b += sizeof(float2) * (size_t)M * (M + 2);
    size_t red = sizeof(double) * RW_MAXS * RW_NGRAD * (RW_THREADS / 32);
    return b > red ? b : red;
}

size_t backward_smem_needed(const DSys& sys) { return backward_smem_bytes(sys.M, sys.emit, sys.n_ssr); }

// Helper warps of the sampled adjoint at M = 96 (one CTA per SM): 8 more
// warps, so 16 per SM, at 128 registers a thread.
#define RW_BWD_HELPERS 8

template <int M, int NS, bool COH = false, int HW = 0>
static cudaError_t launch_backward_d(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                                     const long long* prefix, int njob, long long total,
                                     const RaysIn& rays, const float2* T, const float* amp,
                                     const float* gpsf, const float2* gfield, float* dphi,
                                     float* damp, double* dsurf, unsigned* status,
                                     const unsigned* vis, float* coh_rsum = nullptr,
                                     double* coh_jsum = nullptr) {
    if constexpr (HW == 0 && !COH && M == 96) {
        if (sys.emit == RW_EMIT_SAMPLED)
            return launch_backward_d<M, NS, COH, RW_BWD_HELPERS>(L, sys, jobs, prefix, njob, total,
                                                                 rays, T, amp, gpsf, gfield, dphi,
                                                                 damp, dsurf, status, vis);
    }
    constexpr int NT = RW_THREADS + 32 * HW;
    const size_t smem = backward_smem_bytes(M, sys.emit, sys.n_ssr);
    auto kern = k_backward<M, NS, COH, HW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
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
    kern<<<(unsigned)grid, NT, smem, L.stream>>>(s, jobs, prefix, njob, total, rays, T,
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
