// Specialised post-DOE tracing for systems whose surfaces behind the DOE are
// planes and spheres (the common case): the surface count is a template
// parameter, so the loop unrolls, surface constants become immediate
// constant-bank operands and per-surface state stays in registers.
//
// Precision: the divisions and square roots whose error moves the point
// along the ray (absorbed by the next intersection) or scales a quantity of
// relative size << 1 use the approximate hardware forms (relative error
// ~2^-22); Snell's cos(theta_t), which sets the new direction, and the run
// to the sensor plane, the longest lever, are correctly rounded.
#pragma once
#include "rw_device.cuh"

#define RW_FAST_MAX 8

__device__ __forceinline__ float sqrt_fast(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// One plane or sphere, local coordinates (see trace_one).  On return zl is
// relative to this surface's vertex.
__device__ __forceinline__ bool fast_step(const PSurf& S, float& x, float& y, float& zl,
                                          float& dx, float& dy, float& dz) {
    zl -= S.gap;
    const float idz = rcp_fast(dz);
    const float t0 = -zl * idz;
    x = fmaf(t0, dx, x);
    y = fmaf(t0, dy, y);                    // on the vertex plane
    float t1 = 0.f;
    const float c = S.c;
    if (S.kind != RW_PLANE) {
        const float B = fmaf(c, fmaf(x, dx, y * dy), -dz);
        const float C = c * fmaf(x, x, y * y);
        const float disc = fmaf(B, B, -c * C);
        if (disc < 0.f) return false;
        const float q = -B - copysignf(sqrt_fast(disc), B);
        t1 = C * rcp_fast(q);
        x = fmaf(t1, dx, x);
        y = fmaf(t1, dy, y);
    }
    zl = t1 * dz;
    const float s = fmaf(x, x, y * y);
    if (S.r_ap2 > 0.f && s > S.r_ap2) return false;
    const float a = fmaf(-c * c, s, 1.f);
    if (a <= 0.f) return false;
    float nx = -c * x, ny = -c * y, nz = sqrt_fast(a);
    float ci = fmaf(nx, dx, fmaf(ny, dy, nz * dz));
    if (ci < 0.f) { nx = -nx; ny = -ny; nz = -nz; ci = -ci; }
    const float eta = S.eta;
    const float k = fmaf(-eta * eta, fmaf(-ci, ci, 1.f), 1.f);
    if (k < 0.f) return false;
    const float beta = sqrtf(k) - eta * ci;     // sets the direction: correctly rounded
    dx = fmaf(eta, dx, beta * nx);
    dy = fmaf(eta, dy, beta * ny);
    dz = fmaf(eta, dz, beta * nz);
    return true;
}

// Trace NS post-DOE surfaces and the sensor plane; position left in (x, y).
template <int NS>
__device__ __forceinline__ bool fast_to_sensor(const DSys& sys, float& x, float& y, float& zl,
                                               float& dx, float& dy, float& dz) {
#pragma unroll
    for (int i = 0; i < NS; ++i)
        if (!fast_step(sys.post[i], x, y, zl, dx, dy, dz)) return false;
    zl -= sys.sensor_gap;
    const float t = -zl / dz;                     // the longest run: correctly rounded
    x = fmaf(t, dx, x);
    y = fmaf(t, dy, y);
    return true;
}

// Reverse of fast_step for a ray that passed.  `in` is the state entering
// the surface (zl already relative to this vertex).  (gx..gdz) hold the
// gradient w.r.t. the outgoing hit point / direction on entry and w.r.t. the
// incoming point / direction on exit.  Adds d/d(z_vertex), d/dc and
// d/d(n_after) of this surface to gzv, gc, gna and d/d(n_before) to gnb.
__device__ __forceinline__ void fast_step_adjoint(const PSurf& S, const SurfIn& in, float& gx,
                                                  float& gy, float& gz, float& gdx, float& gdy,
                                                  float& gdz, float& gzv, float& gc,
                                                  float& gna, float& gnb) {
    const float c = S.c;
    // ---- recompute the forward
    const float t0 = -in.zl * rcp_fast(in.dz);
    float x1 = fmaf(t0, in.dx, in.x), y1 = fmaf(t0, in.dy, in.y);
    float t1 = 0.f;
    if (S.kind != RW_PLANE) {
        const float B = fmaf(c, fmaf(x1, in.dx, y1 * in.dy), -in.dz);
        const float C = c * fmaf(x1, x1, y1 * y1);
        const float disc = fmaf(B, B, -c * C);
        const float q = -B - copysignf(sqrt_fast(fmaxf(disc, 0.f)), B);
        t1 = C * rcp_fast(q);
    }
    const float t = t0 + t1;
    const float xh = fmaf(t1, in.dx, x1), yh = fmaf(t1, in.dy, y1);
    const float s = fmaf(xh, xh, yh * yh);
    const float q = sqrt_fast(fmaf(-c * c, s, 1.f));
    const float iq = rcp_fast(q);
    float nx = -c * xh, ny = -c * yh, nz = q;
    float ci = fmaf(nx, in.dx, fmaf(ny, in.dy, nz * in.dz));
    float sgn = 1.f;
    if (ci < 0.f) { sgn = -1.f; ci = -ci; }
    const float onx = sgn * nx, ony = sgn * ny, onz = sgn * nz;
    const float eta = S.eta;
    const float kk = fmaf(-eta * eta, fmaf(-ci, ci, 1.f), 1.f);
    const float ct = sqrt_fast(fmaxf(kk, 0.f));
    const float ict = rcp_fast(ct);
    const float beta = ct - eta * ci;
    // ---- Snell: d' = eta d + beta(ci, eta) n_o
    const float gdn = fmaf(gdx, onx, fmaf(gdy, ony, gdz * onz));
    const float g_ci = gdn * (eta * eta * ci * ict - eta);
    const float g_eta = fmaf(gdx, in.dx, fmaf(gdy, in.dy, gdz * in.dz)) +
                        gdn * (-eta * fmaf(-ci, ci, 1.f) * ict - ci);
    const float gnx = sgn * fmaf(beta, gdx, g_ci * in.dx);
    const float gny = sgn * fmaf(beta, gdy, g_ci * in.dy);
    const float gnz = sgn * fmaf(beta, gdz, g_ci * in.dz);
    float g_dx = fmaf(eta, gdx, g_ci * onx);
    float g_dy = fmaf(eta, gdy, g_ci * ony);
    float g_dz = fmaf(eta, gdz, g_ci * onz);
    const float ina = S.inv_n_after;
    gna -= g_eta * eta * ina;
    gnb += g_eta * ina;
    // ---- sphere normal n = (-c x, -c y, q), q = sqrt(1 - c^2 s)
    const float ghx = gx - c * gnx - c * c * xh * iq * gnz;
    const float ghy = gy - c * gny - c * c * yh * iq * gnz;
    const float ghz = gz;
    if (S.kind != RW_PLANE) gc += -xh * gnx - yh * gny - c * s * iq * gnz;
    // ---- hit h = p + t d
    const float g_t = fmaf(ghx, in.dx, fmaf(ghy, in.dy, ghz * in.dz));
    g_dx = fmaf(ghx, t, g_dx);
    g_dy = fmaf(ghy, t, g_dy);
    g_dz = fmaf(ghz, t, g_dz);
    // ---- t from G = p_z + t d_z - sag(s), sag' = c / (2q)
    const float ciq = c * iq;
    const float Gt = in.dz - ciq * fmaf(xh, in.dx, yh * in.dy);
    const float gam = -g_t * rcp_fast(Gt);
    const float dGx = -ciq * xh, dGy = -ciq * yh;
    gx = fmaf(gam, dGx, ghx);
    gy = fmaf(gam, dGy, ghy);
    gz = ghz + gam;
    gdx = fmaf(gam * t, dGx, g_dx);
    gdy = fmaf(gam * t, dGy, g_dy);
    gdz = fmaf(gam, t, g_dz);
    gzv -= gam;
    if (S.kind != RW_PLANE) gc -= gam * s * iq * rcp_fast(1.f + q);
}
