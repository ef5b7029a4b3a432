// Exact culling of secondary-ray blocks that cannot reach the sensor.
//
// The bins of one incident ray form a regular grid in the tangential
// wavevector (k_u, k_v).  For a rectangular block of bins we trace the whole
// block at once in affine arithmetic: every quantity is held as
//     c + a e1 + b e2 + p e3 + q e4 + [-r, r],   e1..e4 in [-1, 1],
// where k_u = k_u,c + h_u e1 and k_v = k_v,c + h_v e2 span the block and
// x = x_c + h_x e3, y = y_c + h_y e4 span the DOE hit points of a group of
// neighbouring incident rays of one job (planar DOE; a single ray has
// h_x = h_y = 0), so one test covers the block for the whole group, and r
// bounds everything nonlinear (products of the noise terms, linearisation
// remainders of sqrt and 1/x, and the FP32 rounding of each operation, which
// is absorbed by widening r by a relative 1e-6 per operation -- far above
// the few-ulp error of the operation itself).  The result encloses the exact
// real-number trace of every ray of the block through the plane/sphere
// surfaces behind the DOE to the sensor plane.  If the enclosure of the
// sensor position lies outside the sensor window by more than a margin of
// two pixels, no ray of the block can deposit: the FP32 trace of one ray
// differs from its exact trace by orders of magnitude less than that
// margin.  Aperture clips are ignored (they only remove rays), and any step
// whose range is not provably one-signed (a square root, a division, the
// orientation of a normal, total internal reflection) keeps the block.
#pragma once
#include "rw_fast.cuh"

struct AF {
    float c, a, b, p, q, r;
};

#define RW_AF_REL 1e-6f

__device__ __forceinline__ float af_lin_sum(const AF& x) {
    return fabsf(x.a) + fabsf(x.b) + fabsf(x.p) + fabsf(x.q);
}
__device__ __forceinline__ float af_rad(const AF& x) { return af_lin_sum(x) + x.r; }
__device__ __forceinline__ float af_lo(const AF& x) { return x.c - af_rad(x) * (1.f + 4.f * RW_AF_REL); }
__device__ __forceinline__ float af_hi(const AF& x) { return x.c + af_rad(x) * (1.f + 4.f * RW_AF_REL); }

// widen r to cover the rounding of the operation that produced x
__device__ __forceinline__ AF af_fix(AF x) {
    x.r = x.r * (1.f + 4.f * RW_AF_REL) + RW_AF_REL * (fabsf(x.c) + af_lin_sum(x)) + 1e-30f;
    return x;
}
__device__ __forceinline__ AF af_pt(float v) { return AF{v, 0.f, 0.f, 0.f, 0.f, 0.f}; }
__device__ __forceinline__ AF af_add(const AF& x, const AF& y) {
    return af_fix(AF{x.c + y.c, x.a + y.a, x.b + y.b, x.p + y.p, x.q + y.q, x.r + y.r});
}
__device__ __forceinline__ AF af_sub(const AF& x, const AF& y) {
    return af_fix(AF{x.c - y.c, x.a - y.a, x.b - y.b, x.p - y.p, x.q - y.q, x.r + y.r});
}
__device__ __forceinline__ AF af_neg(const AF& x) { return AF{-x.c, -x.a, -x.b, -x.p, -x.q, x.r}; }
__device__ __forceinline__ AF af_addc(const AF& x, float s) {
    return af_fix(AF{x.c + s, x.a, x.b, x.p, x.q, x.r});
}
__device__ __forceinline__ AF af_scale(const AF& x, float s) {
    return af_fix(AF{x.c * s, x.a * s, x.b * s, x.p * s, x.q * s, x.r * fabsf(s)});
}
__device__ __forceinline__ AF af_mul(const AF& x, const AF& y) {
    const float rx = af_rad(x), ry = af_rad(y);
    return af_fix(AF{x.c * y.c, fmaf(x.c, y.a, y.c * x.a), fmaf(x.c, y.b, y.c * x.b),
                     fmaf(x.c, y.p, y.c * x.p), fmaf(x.c, y.q, y.c * x.q),
                     fmaf(fabsf(x.c), y.r, fmaf(fabsf(y.c), x.r, rx * ry))});
}
// alpha x + zeta +- delta, with alpha applied to the affine part
__device__ __forceinline__ AF af_lin(const AF& x, float alpha, float g_lo, float g_hi) {
    const float zeta = 0.5f * (g_lo + g_hi);
    const float delta = 0.5f * fabsf(g_hi - g_lo) + RW_AF_REL * (fabsf(g_lo) + fabsf(g_hi));
    return af_fix(AF{fmaf(alpha, x.c, zeta), alpha * x.a, alpha * x.b, alpha * x.p,
                     alpha * x.q, fmaf(fabsf(alpha), x.r, delta)});
}
// sqrt on [lo, hi], lo > 0: slope just below f'(hi) keeps g = f - alpha x
// increasing, so its range is [g(lo), g(hi)].
__device__ __forceinline__ bool af_sqrt(const AF& x, AF& out) {
    const float lo = af_lo(x), hi = af_hi(x);
    if (!(lo > 0.f)) return false;
    const float fl = sqrtf(lo), fh = sqrtf(hi);
    const float alpha = (0.5f / fh) * (1.f - 4.f * RW_AF_REL);
    out = af_lin(x, alpha, fmaf(-alpha, lo, fl), fmaf(-alpha, hi, fh));
    return true;
}
// 1/x on [lo, hi] not containing 0: slope just above f'(hi) = -1/hi^2 keeps
// g = f - alpha x decreasing on a positive interval (range [g(hi), g(lo)]).
__device__ __forceinline__ bool af_inv(const AF& x, AF& out) {
    float lo = af_lo(x), hi = af_hi(x);
    const bool neg = hi < 0.f;
    if (neg) { const float t = -hi; hi = -lo; lo = t; }
    if (!(lo > 0.f)) return false;
    const AF xp = neg ? af_neg(x) : x;
    const float fl = 1.f / lo, fh = 1.f / hi;
    const float alpha = -(fh * fh) * (1.f - 4.f * RW_AF_REL);
    const AF r = af_lin(xp, alpha, fmaf(-alpha, lo, fl), fmaf(-alpha, hi, fh));
    out = neg ? af_neg(r) : r;
    return true;
}

// One plane or sphere of the specialised post-DOE trace (see fast_step).
__device__ __forceinline__ bool af_step(const PSurf& S, AF& x, AF& y, AF& zl, AF& dx, AF& dy,
                                        AF& dz) {
    zl = af_addc(zl, -S.gap);
    AF idz;
    if (!af_inv(dz, idz)) return false;
    const AF t0 = af_neg(af_mul(zl, idz));
    x = af_add(x, af_mul(t0, dx));
    y = af_add(y, af_mul(t0, dy));
    const float c = S.c;
    if (S.kind != RW_PLANE) {
        const AF B = af_sub(af_scale(af_add(af_mul(x, dx), af_mul(y, dy)), c), dz);
        const AF C = af_scale(af_add(af_mul(x, x), af_mul(y, y)), c);
        const AF disc = af_sub(af_mul(B, B), af_scale(C, c));
        AF sq;
        if (!af_sqrt(disc, sq)) return false;
        AF q;
        if (af_hi(B) < 0.f) q = af_sub(sq, B);
        else if (af_lo(B) > 0.f) q = af_neg(af_add(B, sq));
        else return false;
        AF iq;
        if (!af_inv(q, iq)) return false;
        const AF t1 = af_mul(C, iq);
        x = af_add(x, af_mul(t1, dx));
        y = af_add(y, af_mul(t1, dy));
        zl = af_mul(t1, dz);
    } else {
        zl = af_pt(0.f);
    }
    const AF s = af_add(af_mul(x, x), af_mul(y, y));
    AF nz;
    if (!af_sqrt(af_addc(af_scale(s, -c * c), 1.f), nz)) return false;
    AF nx = af_scale(x, -c), ny = af_scale(y, -c);
    AF ci = af_add(af_add(af_mul(nx, dx), af_mul(ny, dy)), af_mul(nz, dz));
    if (af_hi(ci) < 0.f) {
        nx = af_neg(nx); ny = af_neg(ny); nz = af_neg(nz); ci = af_neg(ci);
    } else if (!(af_lo(ci) > 0.f)) {
        return false;
    }
    const float eta = S.eta;
    // k = 1 - eta^2 (1 - ci^2)
    const AF k = af_addc(af_scale(af_addc(af_neg(af_mul(ci, ci)), 1.f), -eta * eta), 1.f);
    AF sk;
    if (!af_sqrt(k, sk)) return false;
    const AF beta = af_sub(sk, af_scale(ci, eta));
    dx = af_add(af_scale(dx, eta), af_mul(beta, nx));
    dy = af_add(af_scale(dy, eta), af_mul(beta, ny));
    dz = af_add(af_scale(dz, eta), af_mul(beta, nz));
    return true;
}

// True when no secondary ray with tangential wavevector in
// [ku_c - hu, ku_c + hu] x [kv_c - hv, kv_c + hv] leaving the DOE at a point
// of [xc - hx, xc + hx] x [yc - hy, yc + hy] (z, frame, K and the sensor
// window from R) can deposit on the sensor (incoherent bilinear splat,
// margin of two pixels).  hx, hy > 0 only for a planar DOE.
template <int NS>
__device__ __noinline__ bool af_block_misses_sensor(const DSys& sys, const RayAtDoe& R, float ku_c,
                                                    float hu, float kv_c, float hv, float xc,
                                                    float hx, float yc, float hy) {
    const AF ku = AF{ku_c, hu, 0.f, 0.f, 0.f, 0.f}, kv = AF{kv_c, 0.f, hv, 0.f, 0.f, 0.f};
    AF kn;
    const AF kt2 = af_add(af_mul(ku, ku), af_mul(kv, kv));
    if (!af_sqrt(af_addc(af_neg(kt2), R.K * R.K), kn)) return false;
    const float iK = R.invK;
    AF dx, dy, dz;
    if (!sys.conformal) {
        dx = af_scale(ku, iK);
        dy = af_scale(kv, R.v[1] * iK);
        dz = af_scale(kn, R.n[2] * iK);
    } else {
        dx = af_scale(af_add(af_add(af_scale(ku, R.u[0]), af_scale(kv, R.v[0])),
                             af_scale(kn, R.n[0])), iK);
        dy = af_scale(af_add(af_add(af_scale(ku, R.u[1]), af_scale(kv, R.v[1])),
                             af_scale(kn, R.n[1])), iK);
        dz = af_scale(af_add(af_add(af_scale(ku, R.u[2]), af_scale(kv, R.v[2])),
                             af_scale(kn, R.n[2])), iK);
    }
    AF x = AF{xc, 0.f, 0.f, hx, 0.f, 0.f}, y = AF{yc, 0.f, 0.f, 0.f, hy, 0.f};
    AF zl = af_pt(R.pz);
#pragma unroll
    for (int i = 0; i < NS; ++i)
        if (!af_step(sys.post[i], x, y, zl, dx, dy, dz)) return false;
    zl = af_addc(zl, -sys.sensor_gap);
    AF idz;
    if (!af_inv(dz, idz)) return false;
    const AF t = af_neg(af_mul(zl, idz));
    const AF X = af_add(x, af_mul(t, dx)), Y = af_add(y, af_mul(t, dy));
    // a deposit needs |x - cx| < (nx/2 + 1/2) pitch (same for y)
    const float limx = (0.5f * sys.nx + 2.5f) * sys.spitch;
    const float limy = (0.5f * sys.ny + 2.5f) * sys.spitch;
    return af_hi(X) < R.cx - limx || af_lo(X) > R.cx + limx || af_hi(Y) < R.cy - limy ||
           af_lo(Y) > R.cy + limy;
}
