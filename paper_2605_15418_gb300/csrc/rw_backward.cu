// A9: adjoint of the fused forward (incoherent sensor, exhaustive emission).
//
// Per incident ray the CTA recomputes the patch and its spectrum (nothing
// from the forward is stored), then every thread, for each of its bins,
//   re-traces the secondary ray to the sensor keeping the state entering
//   each surface, gathers dL/dI at its four bilinear taps, and runs the
//   hand-written reverse of the sensor plane and of every surface
//   (implicit-function derivative of the intersection, normal, Snell);
//   the gradient w.r.t. the amplitude a = a_in U~ gives dL/dU~, the one
//   w.r.t. the emitted direction gives dL/dkappa and so dL/d(incident
//   direction), the one w.r.t. the ray origin gives dL/d(hit point).
// dL/dU~ goes through the adjoint of the patch transform (the conjugate
// FFT) to dL/dT on the D x D patch, and dT/dphi = i (lambda0/lambda) T,
// dT/dA = exp(i psi) give the map gradients, added to dphi/damp with
// atomics.  Surface-parameter gradients are kept per thread and reduced
// once per CTA into dsurf (double).
#include "rw_kernels.cuh"

struct BwdRay {
    float gpx, gpy, gpz;      // dL/d(hit point)
    float gdx, gdy, gdz;      // dL/d(incident direction at the DOE)
    float gnin, gnout;        // dL/d(index before / after the DOE)
};

__device__ __forceinline__ void bilinear_grad(const DSys& sys, float cx, float cy, float x,
                                              float y, const float* __restrict__ gimg,
                                              float& gw, float& gx, float& gy) {
    gw = 0.f; gx = 0.f; gy = 0.f;
    const float u = (x - cx) * sys.inv_spitch + 0.5f * sys.nx - 0.5f;
    const float v = (y - cy) * sys.inv_spitch + 0.5f * sys.ny - 0.5f;
    if (!(u > -1.f && v > -1.f && u < (float)sys.nx && v < (float)sys.ny)) return;
    const float fi = floorf(u), fj = floorf(v);
    const int i0 = (int)fi, j0 = (int)fj;
    const float fu = u - fi, fv = v - fj;
    const int nx = sys.nx, ny = sys.ny;
    float g00 = 0.f, g10 = 0.f, g01 = 0.f, g11 = 0.f;
    if (j0 >= 0) {
        if (i0 >= 0) g00 = __ldg(gimg + j0 * nx + i0);
        if (i0 + 1 < nx) g10 = __ldg(gimg + j0 * nx + i0 + 1);
    }
    if (j0 + 1 < ny) {
        if (i0 >= 0) g01 = __ldg(gimg + (j0 + 1) * nx + i0);
        if (i0 + 1 < nx) g11 = __ldg(gimg + (j0 + 1) * nx + i0 + 1);
    }
    gw = (1.f - fu) * (1.f - fv) * g00 + fu * (1.f - fv) * g10 + (1.f - fu) * fv * g01 + fu * fv * g11;
    const float gfu = (1.f - fv) * (g10 - g00) + fv * (g11 - g01);
    const float gfv = (1.f - fu) * (g01 - g00) + fu * (g11 - g10);
    gx = gfu * sys.inv_spitch;
    gy = gfv * sys.inv_spitch;
}

// Reverse of the sensor plane xs = x + ts d, ts = -zs / dz, then of the
// emission d = (ku u + kv v + kn n) / K; accumulates dL/d(hit), dL/dkappa and
// dL/dK of the incident ray into acc[0..5].
__device__ __forceinline__ void sensor_plane_adjoint(float gxs, float gys, float ex, float ey,
                                                     float ez, float ts, float& gx, float& gy,
                                                     float& gz, float& gdx, float& gdy,
                                                     float& gdz) {
    gx = gxs;
    gy = gys;
    const float gts = gxs * ex + gys * ey;
    gdx = gxs * ts;
    gdy = gys * ts;
    const float iez = 1.f / ez;
    gz = -gts * iez;
    gdz = -gts * ts * iez;
}

__device__ __forceinline__ void emission_adjoint(const DSys& sys, const RayAtDoe& R, int ju,
                                                 int jv, float dx, float dy, float dz,
                                                 float gx, float gy, float gz, float gdx,
                                                 float gdy, float gdz, float* acc) {
    const float ku = R.kin_u + sys.kstep * (float)ju;
    const float kv = R.kin_v + sys.kstep * (float)jv;
    const float K = R.K;
    const float kn2 = fmaxf(K * K - ku * ku - kv * kv, 0.f);
    float ikn;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(ikn) : "f"(kn2));
    const float gdu = gdx * R.u[0] + gdy * R.u[1] + gdz * R.u[2];
    const float gdv = gdx * R.v[0] + gdy * R.v[1] + gdz * R.v[2];
    const float gdn = gdx * R.n[0] + gdy * R.n[1] + gdz * R.n[2];
    const float gku = (gdu - ku * ikn * gdn) * R.invK;
    const float gkv = (gdv - kv * ikn * gdn) * R.invK;
    const float gdd = gdx * dx + gdy * dy + gdz * dz;
    const float gK = gdn * ikn - gdd * R.invK;
    acc[0] += gx; acc[1] += gy; acc[2] += gz;
    acc[3] += gku; acc[4] += gkv;
    acc[5] += gK;
}

template <int D>
struct BwdOcc { static constexpr int value = D == 64 ? 3 : (D == 96 ? 1 : 2); };

template <int D, int NS>
__global__ void __launch_bounds__(RW_THREADS, BwdOcc<D>::value)
k_backward(const DSys sys, const DJob* __restrict__ jobs, const long long* __restrict__ prefix,
           int njob, long long total, RaysIn rays, const float2* __restrict__ Tmaps,
           const float* __restrict__ amp, const float* __restrict__ gpsf,
           float* __restrict__ dphi, float* __restrict__ damp, double* __restrict__ dsurf,
           unsigned* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2* X = reinterpret_cast<float2*>(smem);
    float2* tw = X + D * D;
    float2* phu = tw + D;
    float2* phv = phu + D;
    RayAtDoe* info = reinterpret_cast<RayAtDoe*>(phv + D);
    float2* G = reinterpret_cast<float2*>(smem + sampled_scratch_offset(D));
    BwdRay* bray = reinterpret_cast<BwdRay*>(G + D * D);
    float* red = reinterpret_cast<float*>(bray + RW_TILE);   // [8 warps][9]
    fft_twiddles<D>(tw);
    float gs[RW_MAXS * RW_NGRAD];
#pragma unroll
    for (int i = 0; i < RW_MAXS * RW_NGRAD; ++i) gs[i] = 0.f;
    // specialised path: per-surface gradients in registers (z, c, n_after)
    constexpr int NR = NS > 0 ? NS : 1;
    float fz[NR], fc[NR], fn[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) { fz[i] = 0.f; fc[i] = 0.f; fn[i] = 0.f; }
    float f_doe_n = 0.f;
    const long long npix_map = (long long)sys.H * sys.W;
    const long long npx = (long long)sys.nx * sys.ny;
    const long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
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
            gather_patch<D>(sys, R, T, X, phu, phv);
            __syncthreads();
            fft2d<D, false>(X, tw);
            const float2 ain = make_float2(R.a_re, R.a_im);
            const float* gimg = gpsf + (long long)R.job * npx;
            float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int f = threadIdx.x; f < D * D; f += RW_THREADS) {
                const int jvi = f / D, jui = f - (f / D) * D;
                int mu = jui + D / 2; if (mu >= D) mu -= D;
                int mv = jvi + D / 2; if (mv >= D) mv -= D;
                float2 gU = make_float2(0.f, 0.f);
                float dx, dy, dz;
                if (NS >= 0) {
                    if (bin_direction<true>(sys, R, jui - D / 2, jvi - D / 2, dx, dy, dz)) {
                        const float2 U = spectrum_at<D>(X, phu, phv, jui, jvi);
                        const float2 a = cmul(ain, U);
                        const float w = a.x * a.x + a.y * a.y;
                        SurfIn st[NR];
                        float x = R.px, y = R.py, zl = R.pz;
                        float ex = dx, ey = dy, ez = dz;
                        bool ok = true;
#pragma unroll
                        for (int i = 0; i < NS; ++i) {
                            if (ok) {
                                st[i].x = x; st[i].y = y; st[i].zl = zl - sys.post[i].gap;
                                st[i].dx = ex; st[i].dy = ey; st[i].dz = ez;
                                ok = fast_step(sys.post[i], x, y, zl, ex, ey, ez);
                            }
                        }
                        if (ok) {
                            const float zs = zl - sys.sensor_gap;
                            const float ts = -zs * rcp_fast(ez);
                            const float xs = fmaf(ts, ex, x), ys = fmaf(ts, ey, y);
                            float gw, gxs, gys;
                            bilinear_grad(sys, R.cx, R.cy, xs, ys, gimg, gw, gxs, gys);
                            gxs *= w;
                            gys *= w;
                            if (gw != 0.f || gxs != 0.f || gys != 0.f) {
                                float gx, gy, gz, gdx, gdy, gdz;
                                sensor_plane_adjoint(gxs, gys, ex, ey, ez, ts, gx, gy, gz, gdx,
                                                     gdy, gdz);
#pragma unroll
                                for (int i = NS - 1; i >= 0; --i) {
                                    float gnb = 0.f;
                                    fast_step_adjoint(sys.post[i], st[i], gx, gy, gz, gdx, gdy,
                                                      gdz, fz[i], fc[i], fn[i], gnb);
                                    if (i > 0) fn[i > 0 ? i - 1 : 0] += gnb; else f_doe_n += gnb;
                                }
                                emission_adjoint(sys, R, jui - D / 2, jvi - D / 2, dx, dy, dz,
                                                 gx, gy, gz, gdx, gdy, gdz, acc);
                                const float2 ga = make_float2(2.f * a.x * gw, 2.f * a.y * gw);
                                gU = cmulc(ga, ain);
                            }
                        }
                    }
                } else if (bin_direction(sys, R, jui - D / 2, jvi - D / 2, dx, dy, dz)) {
                    const float2 U = spectrum_at<D>(X, phu, phv, jui, jvi);
                    const float2 a = cmul(ain, U);
                    const float w = a.x * a.x + a.y * a.y;
                    // ---- forward re-trace, keeping the input of every surface
                    SurfIn st[RW_MAXS];
                    float x = R.px, y = R.py, zl = R.pz;
                    float ex = dx, ey = dy, ez = dz;
                    double dummy = 0.0;
                    bool ok = true;
                    for (int s = sys.doe_index + 1; s < sys.nsurf && ok; ++s) {
                        st[s].x = x; st[s].y = y; st[s].zl = zl - sys.s[s].gap;
                        st[s].dx = ex; st[s].dy = ey; st[s].dz = ez;
                        ok = trace_one<false>(sys.s[s], x, y, zl, ex, ey, ez, dummy, status);
                    }
                    if (ok && ez != 0.f) {
                        const float zs = zl - sys.sensor_gap;
                        const float ts = -zs / ez;
                        const float xs = fmaf(ts, ex, x), ys = fmaf(ts, ey, y);
                        float gw, gxs, gys;
                        bilinear_grad(sys, R.cx, R.cy, xs, ys, gimg, gw, gxs, gys);
                        // the deposit is w * (bilinear weight): position gradients scale by w
                        gxs *= w;
                        gys *= w;
                        if (gw != 0.f || gxs != 0.f || gys != 0.f) {
                            // ---- sensor plane: xs = x + ts ex, ts = -zs / ez
                            float gx = gxs, gy = gys;
                            const float gts = gxs * ex + gys * ey;
                            float gdx = gxs * ts, gdy = gys * ts;
                            float gz = -gts / ez;
                            float gdz = -gts * ts / ez;
                            // ---- surfaces in reverse
                            for (int s = sys.nsurf - 1; s > sys.doe_index; --s) {
                                float gnb = 0.f;
                                trace_one_adjoint(sys.s[s], st[s], gx, gy, gz, gdx, gdy, gdz,
                                                  gs + s * RW_NGRAD, &gnb);
                                gs[(s - 1) * RW_NGRAD + 7] += gnb;
                            }
                            // ---- emission: d = (ku u + kv v + kn n) / K
                            const float ku = R.kin_u + sys.kstep * (float)(jui - D / 2);
                            const float kv = R.kin_v + sys.kstep * (float)(jvi - D / 2);
                            const float K = R.K;
                            const float kn = sqrtf(fmaxf(K * K - ku * ku - kv * kv, 0.f));
                            const float gdu = gdx * R.u[0] + gdy * R.u[1] + gdz * R.u[2];
                            const float gdv = gdx * R.v[0] + gdy * R.v[1] + gdz * R.v[2];
                            const float gdn = gdx * R.n[0] + gdy * R.n[1] + gdz * R.n[2];
                            const float gku = (gdu - ku / kn * gdn) / K;
                            const float gkv = (gdv - kv / kn * gdn) / K;
                            const float gdd = gdx * dx + gdy * dy + gdz * dz;
                            const float gK = gdn / kn - gdd / K;
                            acc[0] += gx; acc[1] += gy; acc[2] += gz;
                            acc[3] += gku; acc[4] += gkv;
                            acc[5] += gK;
                            // ---- amplitude: w = |a|^2, a = a_in U
                            const float2 ga = make_float2(2.f * a.x * gw, 2.f * a.y * gw);
                            gU = cmulc(ga, ain);          // conj(a_in) * g_a
                        }
                    }
                }
                // dL/dX[m] = conj(phu phv) / D^2 * dL/dU~
                const float2 ph = cmul(phu[jui], phv[jvi]);
                G[mv * D + mu] = cscale(cmulc(gU, ph), 1.f / (float)(D * D));
            }
            // ---- per-ray reduction of the geometric gradients
#pragma unroll
            for (int k = 0; k < 6; ++k)
                for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < 6; ++k) red[warp * 9 + k] = acc[k];
            __syncthreads();
            if (threadIdx.x == 0) {
                float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int w = 0; w < RW_THREADS / 32; ++w)
                    for (int k = 0; k < 6; ++k) s[k] += red[w * 9 + k];
                BwdRay& B = bray[r];
                B.gpx = s[0]; B.gpy = s[1]; B.gpz = s[2];
                // kappa_in = k0 n_in (d.u, d.v)
                const float kn_in = J.k0 * sys.n_in;
                B.gdx = kn_in * (s[3] * R.u[0] + s[4] * R.v[0]);
                B.gdy = kn_in * (s[3] * R.u[1] + s[4] * R.v[1]);
                B.gdz = kn_in * (s[3] * R.u[2] + s[4] * R.v[2]);
                B.gnin = (R.kin_u * s[3] + R.kin_v * s[4]) / sys.n_in;
                B.gnout = J.k0 * s[5];
            }
            // ---- adjoint patch transform and map scatter
            fft2d<D, true>(G, tw);
            const float scale = J.phase_scale;
            const int H = sys.H, W = sys.W;
            for (int f = threadIdx.x; f < D * D; f += RW_THREADS) {
                const int b = f / D, a = f - (f / D) * D;
                const float2 gT = G[f];
                if (sys.gather == RW_GATHER_NEAREST) {
                    const int rr = R.r0 + b, cc = R.c0 + a;
                    if ((unsigned)rr < (unsigned)H && (unsigned)cc < (unsigned)W) {
                        const long long p = (long long)rr * W + cc;
                        const float2 t = __ldg(&T[p]);
                        if (dphi) atomicAdd(dphi + p, scale * (t.x * gT.y - t.y * gT.x));
                        if (damp) {
                            const float A = __ldg(amp + p);
                            if (A != 0.f) atomicAdd(damp + p, (t.x * gT.x + t.y * gT.y) / A);
                        }
                    }
                } else {
                    const float oa = (float)(a - D / 2), ob = (float)(b - D / 2);
                    const float fu = R.s0 + oa * R.u[0] + ob * R.v[0];
                    const float fv = R.t0 + oa * R.u[1] + ob * R.v[1];
                    const float iuf = floorf(fu), ivf = floorf(fv);
                    const float wu = fu - iuf, wv = fv - ivf;
                    const int i0 = R.c0 + (int)iuf, j0 = R.r0 + (int)ivf;
                    const float wt[4] = {(1.f - wu) * (1.f - wv), wu * (1.f - wv),
                                         (1.f - wu) * wv, wu * wv};
                    const int di[4] = {0, 1, 0, 1}, dj[4] = {0, 0, 1, 1};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int rr = j0 + dj[q], cc = i0 + di[q];
                        if ((unsigned)rr < (unsigned)H && (unsigned)cc < (unsigned)W) {
                            const long long p = (long long)rr * W + cc;
                            const float2 t = __ldg(&T[p]);
                            const float2 g = cscale(gT, wt[q]);
                            if (dphi) atomicAdd(dphi + p, scale * (t.x * g.y - t.y * g.x));
                            if (damp) {
                                const float A = __ldg(amp + p);
                                if (A != 0.f) atomicAdd(damp + p, (t.x * g.x + t.y * g.y) / A);
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
        // ---- incident side: DOE hit and pre-DOE surfaces, one lane per ray
        if (threadIdx.x < RW_TILE && info[threadIdx.x].alive) {
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
            gs[sys.doe_index * RW_NGRAD + 7] += B.gnout;
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
    if (NS >= 0) {
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const int si = sys.doe_index + 1 + i;
            gs[si * RW_NGRAD + 0] += fz[i];
            gs[si * RW_NGRAD + 1] += fc[i];
            gs[si * RW_NGRAD + 7] += fn[i];
        }
        gs[sys.doe_index * RW_NGRAD + 7] += f_doe_n;
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

inline size_t backward_smem_bytes(int D) {
    size_t b = sampled_scratch_offset(D) + sizeof(float2) * (size_t)D * D +
               sizeof(BwdRay) * RW_TILE + sizeof(float) * 9 * (RW_THREADS / 32);
    size_t red = sizeof(double) * RW_MAXS * RW_NGRAD * (RW_THREADS / 32);
    return b > red ? b : red;
}

template <int D, int NS>
static cudaError_t launch_backward_d(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                                     const long long* prefix, int njob, long long total,
                                     const RaysIn& rays, const float2* T, const float* amp,
                                     const float* gpsf, float* dphi, float* damp, double* dsurf,
                                     unsigned* status) {
    const size_t smem = backward_smem_bytes(D);
    auto kern = k_backward<D, NS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RW_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long long ntiles = (total + RW_TILE - 1) / RW_TILE;
    long long grid = (long long)L.num_sms * per_sm;
    if (L.grid_override > 0) grid = L.grid_override;
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, RW_THREADS, smem, L.stream>>>(sys, jobs, prefix, njob, total, rays, T,
                                                          amp, gpsf, dphi, damp, dsurf, status);
    return cudaGetLastError();
}

cudaError_t launch_backward(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                            const long long* prefix, int njob, long long total,
                            const RaysIn& rays, const float2* T, const float* amp,
                            const float* dl_dpsf, float* dphi, float* damp, double* dsurf,
                            int /*scratch_slots*/, unsigned* status, int* launches) {
    if (sys.emit != RW_EMIT_EXHAUSTIVE) return cudaErrorNotSupported;
    *launches = 1;
    const int ns = sys.fast_ok ? sys.n_post : -1;
#define RW_BWD(DD, NN) \
    launch_backward_d<DD, NN>(L, sys, jobs, prefix, njob, total, rays, T, amp, dl_dpsf, dphi, damp, dsurf, status)
#define RW_BWD_D(DD)                                      \
    case DD:                                              \
        switch (ns) {                                     \
            case 0: return RW_BWD(DD, 0);                 \
            case 2: return RW_BWD(DD, 2);                 \
            case 4: return RW_BWD(DD, 4);                 \
            case 6: return RW_BWD(DD, 6);                 \
            default: return RW_BWD(DD, -1);               \
        }
    switch (sys.D) {
        RW_BWD_D(16)
        RW_BWD_D(32)
        RW_BWD_D(64)
        RW_BWD_D(96)
        default: return cudaErrorInvalidValue;
    }
#undef RW_BWD_D
#undef RW_BWD
}
