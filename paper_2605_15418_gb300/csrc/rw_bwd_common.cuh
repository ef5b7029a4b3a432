// Pieces of the adjoint shared by the fused kernel (rw_backward.cu) and the
// split kernels (rw_bwd_split.cu): reverse of one secondary ray, of its
// emission, of the map gather, and of the incident side.
#pragma once
#include "rw_kernels.cuh"

// Per-ray sums of one incident ray of a tile (layout of RW_RS).
struct BwdRay {
    float s[RW_RS];
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

// Per-thread accumulators of surface-parameter gradients for the
// specialised path: only constant indices, so they stay in registers.  The
// generic path and the incident side use a separate per-thread array `gs`.
template <int NS>
struct SurfGrads {
    static constexpr int NR = NS > 0 ? NS : 1;
    float fz[NR], fc[NR], fn[NR];    // z, c, n_after of post[i]
    float f_doe_n;                   // n_after of the DOE surface
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < NR; ++i) { fz[i] = 0.f; fc[i] = 0.f; fn[i] = 0.f; }
        f_doe_n = 0.f;
    }
};

// Re-trace one secondary ray (origin = DOE hit of R, direction d, deposit
// weight w = |a|^2) and reverse it.  On success returns dL/dw, dL/d(origin)
// and dL/d(direction) and adds the surface-parameter gradients to SG.
template <int NS>
__device__ __forceinline__ bool secondary_adjoint(const DSys& sys, const RayAtDoe& R,
                                                  const float* __restrict__ gimg, float dx,
                                                  float dy, float dz, float w, float& gw,
                                                  float& gx, float& gy, float& gz, float& gdx,
                                                  float& gdy, float& gdz, SurfGrads<NS>& SG,
                                                  float* gs, unsigned* status) {
    constexpr int NR = SurfGrads<NS>::NR;
    float x = R.px, y = R.py, zl = R.pz;
    float ex = dx, ey = dy, ez = dz;
    bool ok = true;
    if constexpr (NS >= 0) {
        SurfIn st[NR];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            if (ok) {
                st[i].x = x; st[i].y = y; st[i].zl = zl - sys.post[i].gap;
                st[i].dx = ex; st[i].dy = ey; st[i].dz = ez;
                ok = fast_step(sys.post[i], x, y, zl, ex, ey, ez);
            }
        }
        if (!ok) return false;
        const float zs = zl - sys.sensor_gap;
        const float ts = -zs / ez;                 // as in the forward: correctly rounded
        const float xs = fmaf(ts, ex, x), ys = fmaf(ts, ey, y);
        float gxs, gys;
        bilinear_grad(sys, R.cx, R.cy, xs, ys, gimg, gw, gxs, gys);
        gxs *= w;   // the deposit is w times the tap weight
        gys *= w;
        if (gw == 0.f && gxs == 0.f && gys == 0.f) return false;
        // sensor plane: xs = x + ts e, ts = -zs / ez
        const float gts = gxs * ex + gys * ey;
        gx = gxs; gy = gys;
        gdx = gxs * ts; gdy = gys * ts;
        const float iez = rcp_fast(ez);
        gz = -gts * iez;
        gdz = -gts * ts * iez;
#pragma unroll
        for (int i = NS - 1; i >= 0; --i) {
            float gnb = 0.f;
            fast_step_adjoint(sys.post[i], st[i], gx, gy, gz, gdx, gdy, gdz, SG.fz[i], SG.fc[i],
                              SG.fn[i], gnb);
            if (i > 0) SG.fn[i > 0 ? i - 1 : 0] += gnb; else SG.f_doe_n += gnb;
        }
        return true;
    } else {
        SurfIn st[RW_MAXS];
        double dummy = 0.0;
        for (int s = sys.doe_index + 1; s < sys.nsurf && ok; ++s) {
            st[s].x = x; st[s].y = y; st[s].zl = zl - sys.s[s].gap;
            st[s].dx = ex; st[s].dy = ey; st[s].dz = ez;
            ok = trace_one<false>(sys.s[s], x, y, zl, ex, ey, ez, dummy, status);
        }
        if (!ok || ez == 0.f) return false;
        const float zs = zl - sys.sensor_gap;
        const float ts = -zs / ez;
        const float xs = fmaf(ts, ex, x), ys = fmaf(ts, ey, y);
        float gxs, gys;
        bilinear_grad(sys, R.cx, R.cy, xs, ys, gimg, gw, gxs, gys);
        gxs *= w;
        gys *= w;
        if (gw == 0.f && gxs == 0.f && gys == 0.f) return false;
        const float gts = gxs * ex + gys * ey;
        gx = gxs; gy = gys;
        gdx = gxs * ts; gdy = gys * ts;
        gz = -gts / ez;
        gdz = -gts * ts / ez;
        for (int s = sys.nsurf - 1; s > sys.doe_index; --s) {
            float gnb = 0.f;
            trace_one_adjoint(sys.s[s], st[s], gx, gy, gz, gdx, gdy, gdz,
                              gs + s * RW_NGRAD, &gnb);
            gs[(s - 1) * RW_NGRAD + 7] += gnb;
        }
        return true;
    }
}

// ------------------------------------------------------------------ coherent sensor
// Reverse of one ray's Eq. 2 sum.  The ray adds c_p = A exp(i theta_p) to
// pixel p, with A = a d_z and theta_p = k OPL + k n_s (d_x (X_p - x) +
// d_y (Y_p - y)).  For gf = dL/dU (dL = sum_p Re(conj(gf_p) dU_p)) and
// w_p = gf_p exp(-i theta_p) this returns W0 = sum w_p, WX = sum w_p (X_p - x)
// and WY = sum w_p (Y_p - y) over the same pixels the forward sums; then
// dL/dA = W0 and dL/dtheta_p = -Im(A conj(w_p)).
__device__ __forceinline__ bool coherent_sums(const DSys& sys, float k0, float cx, float cy,
                                              float x, float y, double opl, float dx, float dy,
                                              const float2* __restrict__ gf, float2& W0,
                                              float2& WX, float2& WY) {
    W0 = WX = WY = make_float2(0.f, 0.f);
    int i_lo, i_hi, j_lo, j_hi;
    float phb;
    if (!coherent_range(sys, k0, cx, cy, x, y, opl, i_lo, i_hi, j_lo, j_hi, phb)) return false;
    const float kx = k0 * sys.n_sensor * dx, ky = k0 * sys.n_sensor * dy;
    // Along a row: one sincos every 8 pixels and rotations by the per-pixel
    // step kx * pitch, run as two interleaved chains (pixels q and q + 4 of a
    // group).  With ry constant in a row and rx = rx_lo + k pitch, the row
    // needs only R = sum_k w_k and K = sum_k k w_k:
    // W0 += R, WY += ry R, WX += rx_lo R + pitch K.
    float st_s, st_c;
    sincosf(kx * sys.spitch, &st_s, &st_c);
    const float s2c = st_c * st_c - st_s * st_s, s2s = 2.f * st_c * st_s;
    const float s4c = s2c * s2c - s2s * s2s, s4s = 2.f * s2c * s2s;
    const float rx_lo = cx + ((float)i_lo - 0.5f * sys.nx + 0.5f) * sys.spitch - x;
    for (int j = j_lo; j <= j_hi; ++j) {
        const float Y = cy + ((float)j - 0.5f * sys.ny + 0.5f) * sys.spitch;
        const float ry = Y - y;
        const float2* grow = gf + j * sys.nx;
        float ra_x = 0.f, ra_y = 0.f, rb_x = 0.f, rb_y = 0.f;     // row sums, chains A and B
        float ka_x = 0.f, ka_y = 0.f, kb_x = 0.f, kb_y = 0.f;     // k-weighted row sums
        for (int i0 = i_lo; i0 <= i_hi; i0 += 8) {
            const float rx0 = cx + ((float)i0 - 0.5f * sys.nx + 0.5f) * sys.spitch - x;
            float sa, ca;
            sincosf(phb + kx * rx0 + ky * ry, &sa, &ca);
            float cb = ca * s4c - sa * s4s, sb = sa * s4c + ca * s4s;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int ia = i0 + q, ib = i0 + 4 + q;
                if (ia <= i_hi) {
                    const float2 g = __ldg(grow + ia);
                    const float wr = g.x * ca + g.y * sa, wi = g.y * ca - g.x * sa;
                    const float k = (float)(ia - i_lo);
                    ra_x += wr; ra_y += wi;
                    ka_x = fmaf(k, wr, ka_x); ka_y = fmaf(k, wi, ka_y);
                }
                if (ib <= i_hi) {
                    const float2 g = __ldg(grow + ib);
                    const float wr = g.x * cb + g.y * sb, wi = g.y * cb - g.x * sb;
                    const float k = (float)(ib - i_lo);
                    rb_x += wr; rb_y += wi;
                    kb_x = fmaf(k, wr, kb_x); kb_y = fmaf(k, wi, kb_y);
                }
                const float ta = ca * st_c - sa * st_s;
                sa = sa * st_c + ca * st_s;
                ca = ta;
                const float tb = cb * st_c - sb * st_s;
                sb = sb * st_c + cb * st_s;
                cb = tb;
            }
        }
        const float Rx = ra_x + rb_x, Ry = ra_y + rb_y;
        const float Kx = ka_x + kb_x, Ky = ka_y + kb_y;
        W0.x += Rx; W0.y += Ry;
        WY.x = fmaf(ry, Rx, WY.x); WY.y = fmaf(ry, Ry, WY.y);
        WX.x += rx_lo * Rx + sys.spitch * Kx;
        WX.y += rx_lo * Ry + sys.spitch * Ky;
    }
    return true;
}

// Coherent sensor: re-trace one secondary ray with its optical path
// (origin = DOE hit of R, direction d, amplitude a) and reverse it, optical
// path included.  On success returns dL/da, dL/d(origin), dL/d(direction) and
// dL/dOPL at the DOE and adds the surface-parameter gradients to gs.
__device__ __forceinline__ bool secondary_adjoint_coh(const DSys& sys, const RayAtDoe& R,
                                                      float k0, const float2* __restrict__ gf,
                                                      float dx, float dy, float dz, float2 a,
                                                      float2& ga, float& gx, float& gy,
                                                      float& gz, float& gdx, float& gdy,
                                                      float& gdz, float& gopl, float* gs,
                                                      unsigned* status) {
    float x = R.px, y = R.py, zl = R.pz;
    double opl = R.opl;
    float ex = dx, ey = dy, ez = dz;
    SurfIn st[RW_MAXS];
    bool ok = true;
    for (int s = sys.doe_index + 1; s < sys.nsurf && ok; ++s) {
        st[s].x = x; st[s].y = y; st[s].zl = zl - sys.s[s].gap;
        st[s].dx = ex; st[s].dy = ey; st[s].dz = ez;
        ok = trace_one<true>(sys.s[s], x, y, zl, ex, ey, ez, opl, status);
    }
    if (!ok) return false;
    float xs = x, ys = y, ts;
    if (!sensor_segment<true>(sys, xs, ys, zl, ex, ey, ez, opl, ts)) return false;
    float2 W0, WX, WY;
    if (!coherent_sums(sys, k0, R.cx, R.cy, xs, ys, opl, ex, ey, gf, W0, WX, WY)) return false;
    const float2 A = make_float2(a.x * ez, a.y * ez);
    const float h0 = A.x * W0.y - A.y * W0.x;     // sum_p dL/dtheta_p
    const float hx = A.x * WX.y - A.y * WX.x;     //   ... (X_p - x)
    const float hy = A.x * WY.y - A.y * WY.x;     //   ... (Y_p - y)
    const float kn = k0 * sys.n_sensor;
    gopl = k0 * h0;
    const float gxs = -kn * ex * h0, gys = -kn * ey * h0;
    ga = make_float2(W0.x * ez, W0.y * ez);
    // sensor plane: (xs, ys) = (x, y) + ts e, OPL += n_s ts, ts = (gap - zl) / ez
    const float gts = gxs * ex + gys * ey + sys.n_sensor * gopl;
    gx = gxs; gy = gys;
    gdx = fmaf(gxs, ts, kn * hx);
    gdy = fmaf(gys, ts, kn * hy);
    gz = -gts / ez;
    gdz = (W0.x * a.x + W0.y * a.y) - gts * ts / ez;
    // the index at the sensor enters the tilt term and the last segment
    if (sys.nsen_slot >= 0)
        gs[sys.nsen_slot * RW_NGRAD + 7] += k0 * (ex * hx + ey * hy) + ts * gopl;
    for (int s = sys.nsurf - 1; s > sys.doe_index; --s) {
        float gnb = 0.f;
        trace_one_adjoint<true>(sys.s[s], st[s], gx, gy, gz, gdx, gdy, gdz, gs + s * RW_NGRAD,
                                &gnb, gopl);
        gs[(s - 1) * RW_NGRAD + 7] += gnb;
    }
    return true;
}

// Reverse of d = (ku u + kv v + kn n) / K for bin (ju, jv): adds dL/d(origin),
// dL/dkappa_u, dL/dkappa_v and dL/dK to acc[0..5] and, with a conformal DOE,
// dL/d(u, v, n) to acc[RW_RS_FRAME ..] (acc then holds RW_RS entries).
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
    acc[0] += gx; acc[1] += gy; acc[2] += gz;
    acc[3] += (gdu - ku * ikn * gdn) * R.invK;
    acc[4] += (gdv - kv * ikn * gdn) * R.invK;
    acc[5] += gdn * ikn - (gdx * dx + gdy * dy + gdz * dz) * R.invK;
    if (sys.conformal) {
        // d = (a_u u + a_v v + a_n n) depends on the frame of the curved DOE
        const float au = ku * R.invK, av = kv * R.invK, an = kn2 * ikn * R.invK;
        acc[RW_RS_FRAME + 0] += au * gdx; acc[RW_RS_FRAME + 1] += au * gdy;
        acc[RW_RS_FRAME + 2] += au * gdz;
        acc[RW_RS_FRAME + 3] += av * gdx; acc[RW_RS_FRAME + 4] += av * gdy;
        acc[RW_RS_FRAME + 5] += av * gdz;
        acc[RW_RS_FRAME + 6] += an * gdx; acc[RW_RS_FRAME + 7] += an * gdy;
        acc[RW_RS_FRAME + 8] += an * gdz;
    }
}


// Reverse of the patch gather: dL/dT on the D x D patch (the top-left
// corner of the M x M buffer G, natural order after the conjugate FFT; the
// padding carries no map samples) -> dphi = (lambda0/lambda) Im(conj(T) g),
// dA = Re(conj(T) g) / A, added to the maps with atomics.  Two phase
// profiles (T = A (e1 + e2), ek = exp(i s phik)): dphik = s Im(conj(A ek) g)
// into dphi[k H W], dA = Re(conj(e1 + e2) g).
__device__ __forceinline__ void map_grad_at(const DSys& sys, long long p, float2 t, float2 g,
                                            const float* __restrict__ amp, float scale,
                                            float* __restrict__ dphi, float* __restrict__ damp) {
    if (sys.two_phase) {
        float s1, c1, s2, c2;
        sincosf(__ldg(sys.phi + p) * scale, &s1, &c1);
        sincosf(__ldg(sys.phi2 + p) * scale, &s2, &c2);
        const float A = amp ? __ldg(amp + p) : 1.f;
        if (dphi) {
            atomicAdd(dphi + p, scale * A * (c1 * g.y - s1 * g.x));
            atomicAdd(dphi + (long long)sys.H * sys.W + p, scale * A * (c2 * g.y - s2 * g.x));
        }
        if (damp) atomicAdd(damp + p, (c1 + c2) * g.x + (s1 + s2) * g.y);
        return;
    }
    if (dphi) atomicAdd(dphi + p, scale * (t.x * g.y - t.y * g.x));
    if (damp) {
        const float A = __ldg(amp + p);
        if (A != 0.f) atomicAdd(damp + p, (t.x * g.x + t.y * g.y) / A);
    }
}

// With gq (conformal DOE, bilinear gather), also the patch positions'
// gradient: per sample, g_u = Re(conj(dL/dT) dT/d(fractional column)) and
// g_v likewise, summed times 1, a and b into gq[0..5] (per thread).
template <int M>
__device__ __forceinline__ void map_scatter(const DSys& sys, const RayAtDoe& R,
                                            const float2* __restrict__ T,
                                            const float* __restrict__ amp, const float2* G,
                                            float scale, float* __restrict__ dphi,
                                            float* __restrict__ damp, float* gq = nullptr) {
    const int H = sys.H, W = sys.W, D = sys.D;
    if (sys.gather == RW_GATHER_NEAREST && dphi && !damp && !sys.two_phase && D == M &&
        R.r0 >= 0 &&
        R.r0 + M <= H && R.c0 >= 0 && R.c0 + M <= W) {
        // interior patch: loads of T in batches of 4 ahead of their atomics
        constexpr int PER = M * M / RW_THREADS, B = PER < 4 ? PER : 4;
        const float2* Tb = T + (long long)R.r0 * W + R.c0;
        float* Db = dphi + (long long)R.r0 * W + R.c0;
#pragma unroll
        for (int k0 = 0; k0 < PER; k0 += B) {
            float2 t[B];
#pragma unroll
            for (int k = 0; k < B; ++k) {
                const int f = threadIdx.x + (k0 + k) * RW_THREADS;
                if (k0 + k < PER) t[k] = __ldg(Tb + (long long)(f / M) * W + (f % M));
            }
#pragma unroll
            for (int k = 0; k < B; ++k) {
                const int f = threadIdx.x + (k0 + k) * RW_THREADS;
                if (k0 + k < PER) {
                    const int b = f / M, a = f % M;
                    const float2 gT = G[b * Patch<M>::S + a];
                    atomicAdd(Db + (long long)b * W + a, scale * (t[k].x * gT.y - t[k].y * gT.x));
                }
            }
        }
        return;
    }
    // walk the M x M grid (compile-time shifts) and skip the padding
    for (int f = threadIdx.x; f < M * M; f += RW_THREADS) {
        const int b = f / M, a = f - (f / M) * M;
        if (a >= D || b >= D) continue;
        const float2 gT = G[b * Patch<M>::S + a];
        if (sys.gather == RW_GATHER_NEAREST) {
            const int rr = R.r0 + b, cc = R.c0 + a;
            if ((unsigned)rr < (unsigned)H && (unsigned)cc < (unsigned)W) {
                const long long p = (long long)rr * W + cc;
                map_grad_at(sys, p, __ldg(&T[p]), gT, amp, scale, dphi, damp);
            }
        } else {
            const float oa = (float)(a - D / 2), ob = (float)(b - D / 2);
            const float fu = R.s0 + oa * R.u[0] + ob * R.v[0];
            const float fv = R.t0 + oa * R.u[1] + ob * R.v[1];
            const float iuf = floorf(fu), ivf = floorf(fv);
            const float wu = fu - iuf, wv = fv - ivf;
            const int i0 = R.c0 + (int)iuf, j0 = R.r0 + (int)ivf;
            const float wt[4] = {(1.f - wu) * (1.f - wv), wu * (1.f - wv), (1.f - wu) * wv, wu * wv};
            const int di[4] = {0, 1, 0, 1}, dj[4] = {0, 0, 1, 1};
            float2 tv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int rr = j0 + dj[q], cc = i0 + di[q];
                const bool in = (unsigned)rr < (unsigned)H && (unsigned)cc < (unsigned)W;
                const long long p = (long long)rr * W + cc;
                tv[q] = in ? __ldg(&T[p]) : make_float2(0.f, 0.f);
                if (in) map_grad_at(sys, p, tv[q], cscale(gT, wt[q]), amp, scale, dphi, damp);
            }
            if (gq) {
                // T = sum of taps: dT/dwu, dT/dwv of the bilinear weights
                const float2 du = make_float2((1.f - wv) * (tv[1].x - tv[0].x) + wv * (tv[3].x - tv[2].x),
                                              (1.f - wv) * (tv[1].y - tv[0].y) + wv * (tv[3].y - tv[2].y));
                const float2 dv = make_float2((1.f - wu) * (tv[2].x - tv[0].x) + wu * (tv[3].x - tv[1].x),
                                              (1.f - wu) * (tv[2].y - tv[0].y) + wu * (tv[3].y - tv[1].y));
                const float gu = gT.x * du.x + gT.y * du.y, gv = gT.x * dv.x + gT.y * dv.y;
                gq[0] += gu; gq[1] += oa * gu; gq[2] += ob * gu;
                gq[3] += gv; gq[4] += oa * gv; gq[5] += ob * gv;
            }
        }
    }
}

// Reverse of a conformal DOE's hit and tangent frame for one incident ray.
// The ray arrives at (x, y, zld) (zld local to the DOE vertex) along d; the
// forward recomputed here: run t to the substrate (conformal_hit), hit Q,
// unit normal N(Q) (sphere: (-c Qx, -c Qy, sqrt(1 - c^2 s)); Gaussian bump:
// (m, 1) / |(m, 1)|, m = 2 iw2 e (Qx, Qy), e = h exp(-s iw2), iw2 = 1/(2 w^2)),
// n_o = N oriented along d, u = normalise(x - n_ox n_o), v = n_o x u, and the
// outgoing normal n = n_o (transmissive) or -n_o (mirror).
// In: s, the ray's per-ray sums (dL/d hit, dL/dkappa, frame and patch-gather
// sums); gd, dL/dd from the incident wavevector already.  Out: dL/d(x, y,
// zld) in (gx, gy, gz), dL/dd added to gd, and the substrate's z, c (sphere)
// or z, height, width (bump) gradients added to gdoe[0..2].
__device__ __forceinline__ void conformal_doe_adjoint(const DSys& sys, const DSurf& S,
                                                      const RayAtDoe& R,
                                                      float kn_in, float x, float y, double zld,
                                                      float dx, float dy, float dz,
                                                      const float* s, float gopl_t,
                                                      float& gx, float& gy, float& gz,
                                                      float& gdx, float& gdy, float& gdz,
                                                      float* gdoe) {
    double td;
    gx = gy = gz = 0.f;
    if (!conformal_hit(S, x, y, zld, dx, dy, dz, td, nullptr)) return;
    const float t = (float)td;
    const float Qx = (float)((double)x + td * dx), Qy = (float)((double)y + td * dy);
    const float Qz = (float)(zld + td * dz);
    const float s2 = Qx * Qx + Qy * Qy;
    const bool bump = S.kind == RW_GAUSS;
    // ---- forward: normal, frame
    float Nx, Ny, Nz, iw2 = 0.f, ex = 0.f, mx = 0.f, my = 0.f, inv = 1.f;
    const float c = (float)S.cd;
    if (bump) {
        iw2 = (float)(0.5 / (S.kd * S.kd));
        ex = (float)S.cd * expf(-s2 * iw2);
        mx = 2.f * iw2 * ex * Qx; my = 2.f * iw2 * ex * Qy;
        inv = rsqrtf(mx * mx + my * my + 1.f);
        Nx = mx * inv; Ny = my * inv; Nz = inv;
    } else {
        Nx = -c * Qx; Ny = -c * Qy; Nz = sqrtf(fmaxf(1.f - c * c * s2, 0.f));
    }
    const float sg = (Nx * dx + Ny * dy + Nz * dz < 0.f) ? -1.f : 1.f;
    // the frame the forward used (formed in double, rounded once): the sums
    // s[] were taken against it, so the projections below must use the same
    // vectors, or their ~1e-7 difference leaks into small gradients
    const float fo = sys.reflective ? -1.f : 1.f;
    const float nox = fo * R.n[0], noy = fo * R.n[1], noz = fo * R.n[2];
    const float ax = 1.f - nox * nox, ay = -nox * noy, az = -nox * noz;
    const float la = sqrtf(ax * ax + ay * ay + az * az), ila = 1.f / la;
    const float ux = R.u[0], uy = R.u[1], uz = R.u[2];
    // ---- gradients on the frame: emitted directions, incident wavevector
    // kappa_in = k0 n_in (d.u, d.v), and the patch sample positions
    // Q + a p u + b p v read at their (x, y) (map column = x / p + const)
    const float ip = 1.f / sys.pitchf;
    float gUx = s[7] + kn_in * s[3] * dx + s[17], gUy = s[8] + kn_in * s[3] * dy + s[20];
    float gUz = s[9] + kn_in * s[3] * dz;
    const float gVx = s[10] + kn_in * s[4] * dx + s[18], gVy = s[11] + kn_in * s[4] * dy + s[21];
    const float gVz = s[12] + kn_in * s[4] * dz;
    const float fn = sys.reflective ? -1.f : 1.f;
    float gNx = fn * s[13], gNy = fn * s[14], gNz = fn * s[15];
    float gQx = s[0] + s[16] * ip, gQy = s[1] + s[19] * ip, gQz = s[2];
    // v = n_o x u
    gNx += uy * gVz - uz * gVy; gNy += uz * gVx - ux * gVz; gNz += ux * gVy - uy * gVx;
    gUx += gVy * noz - gVz * noy; gUy += gVz * nox - gVx * noz; gUz += gVx * noy - gVy * nox;
    // u = a / |a|, a = x - n_ox n_o
    const float gu_u = gUx * ux + gUy * uy + gUz * uz;
    const float gax = (gUx - gu_u * ux) * ila, gay = (gUy - gu_u * uy) * ila;
    const float gaz = (gUz - gu_u * uz) * ila;
    const float ga_n = gax * nox + gay * noy + gaz * noz;
    gNx += -nox * gax - ga_n; gNy += -nox * gay; gNz += -nox * gaz;
    // n_o = sg N
    gNx *= sg; gNy *= sg; gNz *= sg;
    float gpar1 = 0.f, gpar2 = 0.f;       // c | (height, width)
    if (bump) {
        const float gn_n = gNx * Nx + gNy * Ny + gNz * Nz;
        const float gmx = (gNx - gn_n * Nx) * inv, gmy = (gNy - gn_n * Ny) * inv;
        const float a1 = 2.f * iw2 * ex;
        const float dmx_x = a1 * (1.f - 2.f * iw2 * Qx * Qx), dmy_y = a1 * (1.f - 2.f * iw2 * Qy * Qy);
        const float dm_xy = -4.f * iw2 * iw2 * ex * Qx * Qy;
        gQx += gmx * dmx_x + gmy * dm_xy;
        gQy += gmx * dm_xy + gmy * dmy_y;
        const float w = (float)S.kd;
        const float eh = expf(-s2 * iw2);                       // de/dh
        gpar1 += 2.f * iw2 * eh * (gmx * Qx + gmy * Qy);
        gpar2 += -2.f * ex * (1.f - iw2 * s2) / (w * w * w) * (gmx * Qx + gmy * Qy);
    } else {
        const float iNz = 1.f / Nz;
        gQx += -c * gNx - c * c * Qx * gNz * iNz;
        gQy += -c * gNy - c * c * Qy * gNz * iNz;
        gpar1 += -Qx * gNx - Qy * gNy - c * s2 * gNz * iNz;
    }
    // ---- the hit Q = p + t d with F(Q) = 0
    float Ft, Fqx, Fqy, Fqz, Fp1, Fp2 = 0.f;
    if (bump) {
        const float w = (float)S.kd;
        Ft = dz + 2.f * iw2 * ex * (Qx * dx + Qy * dy);
        Fqx = 2.f * iw2 * ex * Qx; Fqy = 2.f * iw2 * ex * Qy; Fqz = 1.f;
        Fp1 = -expf(-s2 * iw2);
        Fp2 = -s2 * ex / (w * w * w);
    } else {
        Ft = 2.f * c * (Qx * dx + Qy * dy + Qz * dz) - 2.f * dz;
        Fqx = 2.f * c * Qx; Fqy = 2.f * c * Qy; Fqz = 2.f * c * Qz - 2.f;
        Fp1 = s2 + Qz * Qz;
    }
    const float g_t = gQx * dx + gQy * dy + gQz * dz + gopl_t;
    const float gam = -g_t / Ft;
    gx = gQx + gam * Fqx; gy = gQy + gam * Fqy; gz = gQz + gam * Fqz;
    gdx += t * gx; gdy += t * gy; gdz += t * gz;
    gdoe[0] += -gam * Fqz;
    gdoe[1] += gam * Fp1 + gpar1;
    if (bump) gdoe[2] += gam * Fp2 + gpar2;
}

// Incident side of one ray from its per-ray sums s (layout of RW_RS): reverse
// of the DOE hit (planar, or a conformal substrate with its frame and patch
// gather) and of the pre-DOE surfaces; adds surface gradients to gs.  OPLG:
// the optical path at the DOE carries the gradient gopl (coherent sensor),
// reversed through every segment n t.
template <bool OPLG = false>
__device__ __forceinline__ void incident_adjoint(const DSys& sys, const DJob* __restrict__ jobs,
                                                 const long long* __restrict__ prefix,
                                                 const RaysIn& rays, const RayAtDoe& R,
                                                 const float* s, float* gs, unsigned* status,
                                                 float gopl = 0.f) {
    const DJob& J = jobs[R.job];
    const float kn_in = J.k0 * sys.n_in;
    float gx = s[0], gy = s[1], gz = s[2];
    float gdx = kn_in * (s[3] * R.u[0] + s[4] * R.v[0]);
    float gdy = kn_in * (s[3] * R.u[1] + s[4] * R.v[1]);
    float gdz = kn_in * (s[3] * R.u[2] + s[4] * R.v[2]);
    // index gradients of the emission: kappa_in = k0 n_in (d.u, d.v), K = k0 n_out
    if (sys.nout_slot >= 0) gs[sys.nout_slot * RW_NGRAD + 7] += J.k0 * s[5];
    if (sys.doe_index > 0)
        gs[(sys.doe_index - 1) * RW_NGRAD + 7] += (R.kin_u * s[3] + R.kin_v * s[4]) / sys.n_in;
    const long long ri = J.off + (R.gid - prefix[R.job]);
    float x = rays.ox[ri], y = rays.oy[ri], zl = rays.oz[ri];
    float dx = rays.dx[ri], dy = rays.dy[ri], dz = rays.dz[ri];
    const double oz = (double)zl;
    double dummy = 0.0;
    SurfIn st[RW_MAXS];
    for (int si = 0; si < sys.doe_index; ++si) {
        st[si].x = x; st[si].y = y; st[si].zl = zl - sys.s[si].gap;
        st[si].dx = dx; st[si].dy = dy; st[si].dz = dz;
        trace_one<false>(sys.s[si], x, y, zl, dx, dy, dz, dummy, status);
    }
    const DSurf& SD = sys.s[sys.doe_index];
    if (sys.conformal) {
        // the conformal hit, frame and gather, as incident_to_doe forms them
        const double zld = (sys.doe_index == 0)
                               ? (oz - SD.z)
                               : ((double)zl - (SD.z - sys.s[sys.doe_index - 1].z));
        float hx, hy, hz;
        conformal_doe_adjoint(sys, SD, R, kn_in, x, y, zld, dx, dy, dz, s,
                              OPLG ? sys.n_in * gopl : 0.f, hx, hy, hz, gdx, gdy, gdz,
                              gs + sys.doe_index * RW_NGRAD);
        if (OPLG && sys.doe_index > 0) {
            double td;
            if (conformal_hit(SD, x, y, zld, dx, dy, dz, td, nullptr))
                gs[(sys.doe_index - 1) * RW_NGRAD + 7] += (float)td * gopl;
        }
        gx = hx; gy = hy; gz = hz;
    } else {
        // planar DOE hit: h = p + t d, t = (z_doe - p_z) / d_z
        const float zld = zl - SD.gap;
        const float t = -zld / dz;
        float gt = gx * dx + gy * dy + gz * dz;
        if (OPLG) {
            // OPL at the DOE = OPL before + n_in t
            gt += sys.n_in * gopl;
            if (sys.doe_index > 0) gs[(sys.doe_index - 1) * RW_NGRAD + 7] += t * gopl;
        }
        gdx += gx * t; gdy += gy * t; gdz += gz * t;
        gz += -gt / dz;
        gdz += -gt * t / dz;
        gs[sys.doe_index * RW_NGRAD + 0] += gt / dz;
    }
    for (int si = sys.doe_index - 1; si >= 0; --si) {
        float gnb = 0.f;
        trace_one_adjoint<OPLG>(sys.s[si], st[si], gx, gy, gz, gdx, gdy, gdz, gs + si * RW_NGRAD,
                                &gnb, gopl);
        if (si > 0) gs[(si - 1) * RW_NGRAD + 7] += gnb;
    }
}

// CTA reduction of per-thread surface gradients gs into dsurf (double);
// `dred` is shared scratch of RW_MAXS * RW_NGRAD * warps doubles.
__device__ __forceinline__ void reduce_surface_grads(const DSys& sys, const float* gs,
                                                     double* dred, double* __restrict__ dsurf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    for (int si = 0; si < sys.nsurf; ++si)
        for (int k = 0; k < RW_NGRAD; ++k) {
            float v = gs[si * RW_NGRAD + k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) dred[(si * RW_NGRAD + k) * (RW_THREADS / 32) + warp] = (double)v;
        }
    __syncthreads();
    for (int i = threadIdx.x; i < sys.nsurf * RW_NGRAD; i += RW_THREADS) {
        double v = 0.0;
        for (int w = 0; w < RW_THREADS / 32; ++w) v += dred[i * (RW_THREADS / 32) + w];
        if (v != 0.0) atomicAdd(dsurf + i, v);
    }
}
