// Device-side descriptors and ray-surface arithmetic of the ray-wave path.
//
// Rays between surfaces are traced in FP32 in *local* coordinates: the
// ray's z is kept relative to the vertex of the surface it last met, and
// moving on to the next surface subtracts the (float) vertex gap.  Keeping
// z small keeps FP32 positions at sub-nanometre resolution on the sensor.
//
// Surface model (vertex form, rotationally symmetric):
//   sag(s) = c s / (1 + sqrt(1 - (1+k) c^2 s)) + A4 s^2 + A6 s^3 + A8 s^4 + A10 s^5,
//   s = x^2 + y^2;  normal = (-2x sag', -2y sag', 1) / |.|;
//   Snell: d' = eta d + (sqrt(1 - eta^2 (1 - cos^2)) - eta cos) n.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/raywave.h"

#define RW_THREADS 256
#define RW_TILE 32           // incident rays traced together by warp 0
#define RW_MAXS RW_MAX_SURFACES

// Thread groups.  Most kernels run one group of RW_THREADS threads per CTA.
// A kernel may run several (threads g * RW_THREADS .. of the block form
// group g): the tensor-core forward runs two groups on separate rays, and
// the sampled adjoint adds helper warps (group 1) that only join its Gumbel
// passes.  Shared device code indexes work by ltid() and syncs with
// main_sync(), so that it runs unchanged in any group.
__device__ __forceinline__ int ltid() { return (int)(threadIdx.x % RW_THREADS); }

// Barrier of the calling thread's group: the CTA barrier when the CTA is one
// group, else named barrier 1 + g for the RW_THREADS threads of group g.
__device__ __forceinline__ void main_sync() {
    if (blockDim.x == RW_THREADS) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(1u + threadIdx.x / RW_THREADS), "n"(RW_THREADS)
                      : "memory");
}

// main_sync() that also returns whether v holds for any thread of the group.
__device__ __forceinline__ bool group_or(bool v) {
    if (blockDim.x == RW_THREADS) return __syncthreads_or(v) != 0;
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
        " bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(1u + threadIdx.x / RW_THREADS), "n"(RW_THREADS)
        : "memory");
    return r != 0;
}

// Per-incident-ray sums of the adjoint, as reduced over the ray's secondary
// rays and patch samples and handed to the incident side:
//   [0..2] dL/d(hit point), [3] dL/dkappa_u, [4] dL/dkappa_v, [5] dL/dK,
//   [6] dL/dOPL at the DOE (coherent sensor);
//   conformal DOE only: [7..9] dL/du, [10..12] dL/dv, [13..15] dL/dn (the
//   outgoing normal) from the emitted directions, [16..21] the patch
//   gather's sums of dL/d(fractional map column) times 1, a, b and of
//   dL/d(fractional map row) times 1, a, b (a, b: sample offsets in pixels).
#define RW_RS 22
#define RW_RS_FRAME 7
#define RW_RS_GATHER 16

#define RW_ST_NOTCONV 1u
#define RW_ST_CAPACITY 2u
#define RW_ST_TIMEOUT 4u

struct DSurf {
    int kind;
    float c, k, A4, A6, A8, A10;
    float n_before, n_after;
    float r_ap2;       // <= 0: no clip
    float gap;         // z_vertex - z of the previous local reference (float)
    double z;          // global vertex z
    double cd;         // curvature (Gaussian bump: height) in double, FP64 hit refinement
    double kd;         // conic constant (Gaussian bump: width), in double
    // double copies for the FP64 trace before the DOE (see trace_one_d)
    double A4d, A6d, A8d, A10d, nbd, nad, r_ap2d;
};

// Post-DOE plane/sphere in the form the specialised trace uses.
struct PSurf {
    int kind;
    float c, gap, r_ap2, eta, inv_n_after;
};

struct DSys {
    int nsurf, doe_index;
    DSurf s[RW_MAXS];
    PSurf post[8];     // surfaces behind the DOE (when n_post <= 8, no aspheres)
    int n_post;        // number of surfaces behind the DOE
    int fast_ok;       // 1: post[] is valid for the specialised trace
    double n_object;
    // DOE
    int H, W, D, gather, emit, n_ssr, phase_model, conformal;
    int reflective;    // secondary rays return into the incident medium
    int two_phase;     // U = A (exp(i phi) + exp(i phi2))
    int uniform;       // sampled emission from the uniform density over propagating bins
    int nslice;        // coherent exhaustive launches: each ray's bins in this many slices,
                       // one CTA work unit per (tile, slice); 1 elsewhere
    const float* phi;  // device phase maps (read by the two-phase adjoint)
    const float* phi2;
    int nout_slot;     // surface whose n_after is n_out (-1: object space)
    int nsen_slot;     // surface whose n_after is the sensor medium (-1: object space)
    int M;             // transform size P D (zero-padded patch)
    int cull;          // 1: exhaustive incoherent forward drops blocks that miss the sensor
    int nrs;           // per-ray adjoint sums kept: 6 (planar), 7 (planar, coherent), RW_RS
    float norm;        // spectrum scale: 1/M^2 (coherent sensor) or 1/(D M)
    double pitch;
    float pitchf, inv_pitch;
    unsigned long long seed, rng_offset;
    float n_in, n_out;
    double n_in_d;
    float kstep;       // 2 pi / (M p): wavevector step of the patch spectrum
    // sensor
    double sensor_z;
    float sensor_gap;  // z_sensor - z of the last surface
    int nx, ny;
    float spitch, inv_spitch;
    int coherent, window;
    float n_sensor;
};

struct DJob {
    double lambda;
    float k0;          // 2 pi / lambda
    float phase_scale; // lambda0 / lambda (HEIGHT) or 1
    long long off, cnt;
    float cx, cy;
    double cxd, cyd;   // the same in double (sensor run from a last-surface DOE)
    int slot;          // wavelength slot of the transmission map
    int out;           // index of the job's image in the psf / dL/dpsf arrays
};

// Incident ray state at the DOE (one per incident ray of a tile).
struct RayAtDoe {
    int alive, job;
    float px, py, pz;       // hit, local to the DOE vertex (z) / global (x, y)
    float u[3], v[3], n[3];
    float kin_u, kin_v, K;  // tangential incident wavevector, k0 n_out
    float invK;
    // bin directions in units of K: tangential components of bin 0 and the
    // step per bin, formed in double and rounded once (a wavevector of order
    // 1e4 / mm kept in float would carry ~4e-8 rad of rounding into every
    // secondary direction), and the rounding residuals (near-grazing bins)
    float tu, tv, tstep;
    float tu_lo, tv_lo, tstep_lo;
    float a_re, a_im;
    double opl;
    double pxd, pyd;        // hit in double (patch indexing)
    int c0, r0;             // nearest: window origin; bilinear: pixel of the hit
    float s0, t0;           // nearest: offset of sample 0 from the hit / (M p);
                            // bilinear: fractional pixel coordinate of the hit
    float cx, cy;           // sensor window centre of the job
    // DOE the last surface: hit minus window centre and the axial run to the
    // sensor plane, formed in double and kept as float pairs (hi, lo) for the
    // secondary rays' run to the sensor (see sensor_offset)
    float sx, sx_lo, sy, sy_lo, sl, sl_lo;
    long long gid;          // position of the ray in the launch's job order
    long long rid;          // index of the ray in the caller's ray arrays: its sampling stream
};

struct RaysIn {
    const float *ox, *oy, *oz, *dx, *dy, *dz, *are, *aim;
    const double* opl;
};

// ---------------------------------------------------------------- complex
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Length of a float direction, in double.
__device__ __forceinline__ double dnorm(float dx, float dy, float dz) {
    const double x = dx, y = dy, z = dz;
    return sqrt(x * x + y * y + z * z);
}

// ---------------------------------------------------------------- sag
struct Sag { float z, dz, ddz; bool ok; float q; };

__device__ __forceinline__ Sag sag_eval(const DSurf& S, float s) {
    Sag r;
    if (S.kind == RW_PLANE) { r.z = 0.f; r.dz = 0.f; r.ddz = 0.f; r.ok = true; r.q = 1.f; return r; }
    float kap = (S.kind == RW_ASPHERE) ? 1.f + S.k : 1.f;
    float arg = 1.f - kap * S.c * S.c * s;
    r.ok = arg > 0.f;
    float q = sqrtf(r.ok ? arg : 1.f);
    r.q = q;
    r.z = S.c * s / (1.f + q);
    r.dz = S.c / (2.f * q);
    r.ddz = kap * S.c * S.c * S.c / (4.f * q * q * q);
    if (S.kind == RW_ASPHERE) {
        float s2 = s * s;
        r.z += S.A4 * s2 + S.A6 * s2 * s + S.A8 * s2 * s2 + S.A10 * s2 * s2 * s;
        r.dz += 2.f * S.A4 * s + 3.f * S.A6 * s2 + 4.f * S.A8 * s2 * s + 5.f * S.A10 * s2 * s2;
        r.ddz += 2.f * S.A4 + 6.f * S.A6 * s + 12.f * S.A8 * s2 + 20.f * S.A10 * s2 * s;
    }
    return r;
}

// Intersection with a surface whose vertex is at local z = 0.  Returns t
// along d (from the current point) or false.  Sphere: the root is taken from
// the vertex plane, t = t0 + C/q, which avoids cancellation; the even
// asphere refines it with Newton's method.
__device__ __forceinline__ bool intersect_local(const DSurf& S, float x, float y, float zl,
                                                float dx, float dy, float dz, float& t,
                                                unsigned* status) {
    if (dz == 0.f) return false;
    float t0 = -zl / dz;
    if (S.kind == RW_PLANE) { t = t0; return true; }
    float x1 = fmaf(t0, dx, x), y1 = fmaf(t0, dy, y);
    float c = S.c;
    float B = c * (x1 * dx + y1 * dy) - dz;
    float C = c * (x1 * x1 + y1 * y1);
    float disc = B * B - c * C;
    if (disc < 0.f) return false;
    float q = -B - copysignf(sqrtf(disc), B);
    if (q == 0.f) return false;
    float t1 = C / q;
    if (S.kind == RW_ASPHERE) {
        // Newton on g(t1) = t1 dz - sag(s(t1)) from the vertex plane point
        bool conv = false;
        for (int it = 0; it < 30; ++it) {
            float xh = fmaf(t1, dx, x1), yh = fmaf(t1, dy, y1);
            Sag sg = sag_eval(S, xh * xh + yh * yh);
            if (!sg.ok) return false;
            float g = t1 * dz - sg.z;
            float gp = dz - sg.dz * 2.f * (xh * dx + yh * dy);
            if (gp == 0.f) return false;
            float step = g / gp;
            t1 -= step;
            // a few FP32 ulps of t1: a one-ulp limit cycle must still count as converged
            if (fabsf(step) <= 5e-7f * (fabsf(t1) + 1e-3f)) { conv = true; break; }
        }
        if (!conv) { if (status) atomicOr(status, RW_ST_NOTCONV); return false; }
    }
    t = t0 + t1;
    return true;
}

__device__ __forceinline__ void surf_normal(const DSurf& S, float xh, float yh, float& nx,
                                            float& ny, float& nz, bool& ok) {
    if (S.kind == RW_PLANE) { nx = 0.f; ny = 0.f; nz = 1.f; ok = true; return; }
    Sag sg = sag_eval(S, xh * xh + yh * yh);
    ok = sg.ok;
    float mx = -2.f * xh * sg.dz, my = -2.f * yh * sg.dz;
    float inv = rsqrtf(mx * mx + my * my + 1.f);
    nx = mx * inv; ny = my * inv; nz = inv;
}

// Vector Snell with the normal oriented along d.  Returns false on TIR.
__device__ __forceinline__ bool refract(float& dx, float& dy, float& dz, float nx, float ny,
                                        float nz, float eta) {
    float ci = nx * dx + ny * dy + nz * dz;
    if (ci < 0.f) { nx = -nx; ny = -ny; nz = -nz; ci = -ci; }
    float k = 1.f - eta * eta * (1.f - ci * ci);
    if (k < 0.f) return false;
    float beta = sqrtf(k) - eta * ci;
    dx = eta * dx + beta * nx;
    dy = eta * dy + beta * ny;
    dz = eta * dz + beta * nz;
    return true;
}

// ---------------------------------------------------------------- FP64 trace before the DOE
// The incident rays are traced to the DOE in double: the patch is sampled at
// the DOE hit point, and on a map with pixel-scale structure a hit that is
// off by 1e-3 of a pixel (0.5 nm at 0.5 um pitch) changes the spectrum by
// ~1e-3 -- about what an FP32 direction error of 1e-7 does over a few mm.
// One trace per incident ray, so the cost is that of a few hundred FP64
// operations against the thousands of bins behind it.
struct SagD { double z, dz; bool ok; };

__device__ __forceinline__ SagD sag_eval_d(const DSurf& S, double s) {
    SagD r;
    if (S.kind == RW_PLANE) { r.z = 0.0; r.dz = 0.0; r.ok = true; return r; }
    const double kap = (S.kind == RW_ASPHERE) ? 1.0 + S.kd : 1.0;
    const double arg = 1.0 - kap * S.cd * S.cd * s;
    r.ok = arg > 0.0;
    const double q = sqrt(r.ok ? arg : 1.0);
    r.z = S.cd * s / (1.0 + q);
    r.dz = S.cd / (2.0 * q);
    if (S.kind == RW_ASPHERE) {
        const double s2 = s * s;
        r.z += s2 * (S.A4d + s * (S.A6d + s * (S.A8d + s * S.A10d)));
        r.dz += s * (2.0 * S.A4d + s * (3.0 * S.A6d + s * (4.0 * S.A8d + s * 5.0 * S.A10d)));
    }
    return r;
}

// t along d from (x, y, zl) (zl local to the vertex) to the surface; the
// even asphere by Newton from the base-sphere root, to 1e-12 relative.
__device__ __forceinline__ bool intersect_local_d(const DSurf& S, double x, double y, double zl,
                                                  double dx, double dy, double dz, double& t,
                                                  unsigned* status) {
    if (dz == 0.0) return false;
    const double t0 = -zl / dz;
    if (S.kind == RW_PLANE) { t = t0; return true; }
    const double x1 = x + t0 * dx, y1 = y + t0 * dy;
    const double c = S.cd;
    const double B = c * (x1 * dx + y1 * dy) - dz;
    const double C = c * (x1 * x1 + y1 * y1);
    const double disc = B * B - c * C;
    if (disc < 0.0) return false;
    const double q = -B - copysign(sqrt(disc), B);
    if (q == 0.0) return false;
    double t1 = C / q;
    if (S.kind == RW_ASPHERE) {
        bool conv = false;
        for (int it = 0; it < 50; ++it) {
            const double xh = x1 + t1 * dx, yh = y1 + t1 * dy;
            const SagD sg = sag_eval_d(S, xh * xh + yh * yh);
            if (!sg.ok) return false;
            const double g = t1 * dz - sg.z;
            const double gp = dz - sg.dz * 2.0 * (xh * dx + yh * dy);
            if (gp == 0.0) return false;
            const double step = g / gp;
            t1 -= step;
            if (fabs(step) <= 1e-12 * (fabs(t1) + fabs(sg.z) + 1e-3)) { conv = true; break; }
        }
        if (!conv) { if (status) atomicOr(status, RW_ST_NOTCONV); return false; }
    }
    t = t0 + t1;
    return true;
}

__device__ __forceinline__ bool refract_d(double& dx, double& dy, double& dz, double nx,
                                          double ny, double nz, double eta) {
    double ci = nx * dx + ny * dy + nz * dz;
    if (ci < 0.0) { nx = -nx; ny = -ny; nz = -nz; ci = -ci; }
    const double k = 1.0 - eta * eta * (1.0 - ci * ci);
    if (k < 0.0) return false;
    const double beta = sqrt(k) - eta * ci;
    dx = eta * dx + beta * nx;
    dy = eta * dy + beta * ny;
    dz = eta * dz + beta * nz;
    return true;
}

// One surface before the DOE in double, global z; adds n_before * t |d| to opl.
__device__ __forceinline__ bool trace_one_d(const DSurf& S, double& x, double& y, double& z,
                                            double& dx, double& dy, double& dz, double& opl,
                                            unsigned* status) {
    double t;
    if (!intersect_local_d(S, x, y, z - S.z, dx, dy, dz, t, status)) return false;
    const double dn = sqrt(dx * dx + dy * dy + dz * dz);
    x += t * dx; y += t * dy; z += t * dz;
    if (S.r_ap2d > 0.0 && x * x + y * y > S.r_ap2d) return false;
    double nx = 0.0, ny = 0.0, nz = 1.0;
    if (S.kind != RW_PLANE) {
        const SagD sg = sag_eval_d(S, x * x + y * y);
        if (!sg.ok) return false;
        const double mx = -2.0 * x * sg.dz, my = -2.0 * y * sg.dz;
        const double inv = 1.0 / sqrt(mx * mx + my * my + 1.0);
        nx = mx * inv; ny = my * inv; nz = inv;
    }
    if (!refract_d(dx, dy, dz, nx, ny, nz, S.nbd / S.nad)) return false;
    opl += S.nbd * t * dn;
    return true;
}

// One surface in local coordinates.  On entry zl is relative to the
// previous reference; on exit relative to this surface's vertex.
// Adds n_before * t to opl.  Returns false if the ray is dropped.
//
// With OPL the path length is kept to double precision (the coherent sum
// turns 1e-7 mm of path into 1e-3 rad of phase): the run to the vertex
// plane, t0 = (gap - zl) / d_z, is formed from the exact double difference
// of the two floats, the ray is put on that plane (local z = 0) and the
// short remaining run t1 to the surface is found from there.  The distance
// travelled is (t0 + t1) |d|: a float direction is unit only to ~1e-7.
template <bool OPL>
__device__ __forceinline__ bool trace_one(const DSurf& S, float& x, float& y, float& zl,
                                          float& dx, float& dy, float& dz, double& opl,
                                          unsigned* status) {
    if (OPL) {
        if (dz == 0.f) return false;
        const double dn = dnorm(dx, dy, dz);
        const double t0 = ((double)S.gap - (double)zl) / (double)dz;
        x = fmaf((float)t0, dx, x);
        y = fmaf((float)t0, dy, y);
        float t1;
        if (!intersect_local(S, x, y, 0.f, dx, dy, dz, t1, status)) return false;
        x = fmaf(t1, dx, x); y = fmaf(t1, dy, y); zl = t1 * dz;
        if (S.r_ap2 > 0.f && x * x + y * y > S.r_ap2) return false;
        float nx, ny, nz; bool ok;
        surf_normal(S, x, y, nx, ny, nz, ok);
        if (!ok) return false;
        if (!refract(dx, dy, dz, nx, ny, nz, S.n_before / S.n_after)) return false;
        opl += (double)S.n_before * (t0 + (double)t1) * dn;
        return true;
    }
    zl -= S.gap;
    float t;
    if (!intersect_local(S, x, y, zl, dx, dy, dz, t, status)) return false;
    x = fmaf(t, dx, x); y = fmaf(t, dy, y); zl = fmaf(t, dz, zl);
    if (S.r_ap2 > 0.f && x * x + y * y > S.r_ap2) return false;
    float nx, ny, nz; bool ok;
    surf_normal(S, x, y, nx, ny, nz, ok);
    if (!ok) return false;
    if (!refract(dx, dy, dz, nx, ny, nz, S.n_before / S.n_after)) return false;
    if (OPL) opl += (double)S.n_before * (double)t;
    return true;
}

// ---------------------------------------------------------------- adjoint
// Saved forward state of one surface interaction: the ray entering it (in
// this surface's local coordinates).
struct SurfIn { float x, y, zl, dx, dy, dz; };

// Parameter-gradient slots per surface: z, c, k, A4, A6, A8, A10, n_after.
#define RW_NGRAD 8

// Reverse of trace_one for an unclipped, refracted ray.  Given the input
// state `in` (local, after the gap shift) and gradients (gx, gy, gz, gdx, gdy,
// gdz) w.r.t. the output hit point and refracted direction, overwrite them
// with gradients w.r.t. the input point/direction and add parameter
// gradients to g[0..7] of this surface and to *g_nbefore (index before).
// OPLG: the ray's optical path also carries a gradient gopl (coherent
// sensor); the segment n_before * t adds n_before gopl to dL/dt and
// t gopl to dL/dn_before (gopl itself passes through unchanged).
template <bool OPLG = false>
__device__ __forceinline__ void trace_one_adjoint(const DSurf& S, const SurfIn& in,
                                                  float& gx, float& gy, float& gz,
                                                  float& gdx, float& gdy, float& gdz,
                                                  float* g, float* g_nbefore,
                                                  float gopl = 0.f) {
    // ---- recompute forward
    float t;
    intersect_local(S, in.x, in.y, in.zl, in.dx, in.dy, in.dz, t, nullptr);
    float xh = fmaf(t, in.dx, in.x), yh = fmaf(t, in.dy, in.y);
    float sh = xh * xh + yh * yh;
    Sag sg = sag_eval(S, sh);
    float a = -2.f * sg.dz;                       // m = (a x, a y, 1), n = m / |m|
    float mx = a * xh, my = a * yh;
    float inv = rsqrtf(mx * mx + my * my + 1.f);
    float nx = mx * inv, ny = my * inv, nz = inv;
    float ci = nx * in.dx + ny * in.dy + nz * in.dz;
    float sgn = 1.f;
    if (ci < 0.f) { sgn = -1.f; ci = -ci; }
    float onx = sgn * nx, ony = sgn * ny, onz = sgn * nz;  // oriented normal
    float eta = S.n_before / S.n_after;
    float kk = 1.f - eta * eta * (1.f - ci * ci);
    float ct = sqrtf(fmaxf(kk, 0.f));
    float beta = ct - eta * ci;
    // ---- Snell: d' = eta d + beta n_o, beta(ci, eta)
    float gdn = gdx * onx + gdy * ony + gdz * onz;     // g_d' . n_o
    float dbeta_dci = eta * eta * ci / ct - eta;
    float dbeta_deta = -eta * (1.f - ci * ci) / ct - ci;
    float g_ci = gdn * dbeta_dci;
    float g_eta = gdx * in.dx + gdy * in.dy + gdz * in.dz + gdn * dbeta_deta;
    // gradient w.r.t. oriented normal: beta g_d' + g_ci d
    float gno_x = beta * gdx + g_ci * in.dx;
    float gno_y = beta * gdy + g_ci * in.dy;
    float gno_z = beta * gdz + g_ci * in.dz;
    // gradient w.r.t. input direction (through eta d and ci = n_o . d)
    float g_dx = eta * gdx + g_ci * onx;
    float g_dy = eta * gdy + g_ci * ony;
    float g_dz = eta * gdz + g_ci * onz;
    // eta = n_before / n_after
    g[7] += -g_eta * eta / S.n_after;                 // d/dn_after
    *g_nbefore += g_eta / S.n_after;
    // ---- normal n = m/|m| (unoriented = sgn * oriented)
    float gnx = sgn * gno_x, gny = sgn * gno_y, gnz = sgn * gno_z;
    float gn_dot_n = gnx * nx + gny * ny + gnz * nz;
    float gmx = (gnx - gn_dot_n * nx) * inv;
    float gmy = (gny - gn_dot_n * ny) * inv;
    // m_z = 1 is constant
    float g_a = gmx * xh + gmy * yh;
    float g_xh = gmx * a, g_yh = gmy * a;
    // a = -2 sag'(s), s = xh^2 + yh^2
    float g_sagp = -2.f * g_a;
    g_xh += g_sagp * sg.ddz * 2.f * xh;
    g_yh += g_sagp * sg.ddz * 2.f * yh;
    // sag' parameter derivatives
    if (S.kind != RW_PLANE) {
        float q = sg.q, q3 = q * q * q;
        g[1] += g_sagp * (1.f / (2.f * q3));                       // d sag'/dc
        if (S.kind == RW_ASPHERE) {
            g[2] += g_sagp * (S.c * S.c * S.c * sh / (4.f * q3)); // d sag'/dk
            float s2 = sh * sh;
            g[3] += g_sagp * 2.f * sh;
            g[4] += g_sagp * 3.f * s2;
            g[5] += g_sagp * 4.f * s2 * sh;
            g[6] += g_sagp * 5.f * s2 * s2;
        }
    }
    // ---- hit point h = p + t d (p = input point); total gradient on h
    float ghx = gx + g_xh, ghy = gy + g_yh, ghz = gz;
    float g_t = ghx * in.dx + ghy * in.dy + ghz * in.dz;
    if (OPLG) {
        g_t += S.n_before * gopl;
        *g_nbefore += t * gopl;
    }
    g_dx += ghx * t; g_dy += ghy * t; g_dz += ghz * t;
    float g_px = ghx, g_py = ghy, g_pz = ghz;
    // ---- t from G(t; p, d, theta) = (p_z + t d_z) - sag(s(t)) = 0 (local z)
    float Gt = in.dz - sg.dz * 2.f * (xh * in.dx + yh * in.dy);
    float gam = -g_t / Gt;
    // dG/dp = (-2 sag' xh, -2 sag' yh, 1); dG/dd = t * dG/dp; dG/dz_vertex = -1
    float dGx = -2.f * sg.dz * xh, dGy = -2.f * sg.dz * yh;
    g_px += gam * dGx; g_py += gam * dGy; g_pz += gam;
    g_dx += gam * dGx * t; g_dy += gam * dGy * t; g_dz += gam * t;
    g[0] += -gam;                                     // d/dz_vertex
    if (S.kind != RW_PLANE) {
        float q = sg.q;
        // dG/dc = -d sag/dc = -s / (q (1 + q))
        g[1] += gam * (-(sh / (q * (1.f + q))));
        if (S.kind == RW_ASPHERE) {
            float cc = S.c;
            g[2] += gam * (-(cc * cc * cc * sh * sh / (2.f * q * (1.f + q) * (1.f + q))));
            float s2 = sh * sh;
            g[3] += gam * (-s2);
            g[4] += gam * (-s2 * sh);
            g[5] += gam * (-s2 * s2);
            g[6] += gam * (-s2 * s2 * sh);
        }
    }
    gx = g_px; gy = g_py; gz = g_pz;
    gdx = g_dx; gdy = g_dy; gdz = g_dz;
}
