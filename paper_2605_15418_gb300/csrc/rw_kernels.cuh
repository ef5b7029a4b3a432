// Per-incident-ray building blocks shared by the forward, emit and adjoint
// kernels, plus the host-side launcher declarations.
#pragma once
#include <cmath>

#include "rw_device.cuh"
#include "rw_fast.cuh"
#include "rw_fft.cuh"
#include "rw_cull.cuh"
#include "rw_tc.cuh"

enum { MODE_SPLAT = 0, MODE_COHERENT = 1, MODE_EMIT = 2 };

// Optional per-launch timing: mark(user, name) is called just before kernel
// `name` is launched on the stream and mark(user, nullptr) just after, so the
// caller can record CUDA events around every launch.
struct ProfHook {
    void* user;
    void (*mark)(void* user, const char* kernel);
};

struct LaunchCtx {
    cudaStream_t stream;
    int num_sms;
    long long grid_override;   // > 0 forces the persistent grid size of every kernel
    long long grid[RW_NK];     // > 0: tuned grid size of kernel RW_K_* (wins over the above)
    const ProfHook* prof;      // may be null
};

// Grid of kernel `kind`: tuned size, else the forced size, else `dflt`.
inline long long pick_grid(const LaunchCtx& L, int kind, long long dflt) {
    if (L.grid[kind] > 0) return L.grid[kind];
    if (L.grid_override > 0) return L.grid_override;
    return dflt;
}

#define RW_MARK(L, name)                                          \
    do {                                                          \
        if ((L).prof) (L).prof->mark((L).prof->user, (name));     \
    } while (0)

struct GenJob {
    long long off, n;          // first ray, grid side
    double spacing, x0, y0;
    float dx, dy, dz, pad;
};

// Host side of A0: check every job against n_rays and fill g[0..njob) and
// prefix[0..njob] (exclusive prefix sum of the ray counts).  Returns nullptr,
// or the reason the jobs are invalid.  Shared by rw_generate_rays and its
// allocation-free variant so that both build the same table.
inline const char* gen_table_fill(const rw_job* jobs, int njob, long long n_rays, GenJob* g,
                                  long long* prefix) {
    prefix[0] = 0;
    for (int i = 0; i < njob; ++i) {
        const rw_job& j = jobs[i];
        if (j.grid_n < 0 || j.ray_count != j.grid_n * j.grid_n)
            return "job ray_count must equal grid_n^2";
        if (j.ray_offset < 0 || j.ray_offset + j.ray_count > n_rays)
            return "job ray range outside the ray arrays";
        const double tx = std::tan(j.theta_x), ty = std::tan(j.theta_y);
        const double nrm = std::sqrt(tx * tx + ty * ty + 1.0);
        g[i].off = j.ray_offset;
        g[i].n = j.grid_n;
        g[i].spacing = j.spacing;
        g[i].x0 = j.x0;
        g[i].y0 = j.y0;
        g[i].dx = (float)(tx / nrm);
        g[i].dy = (float)(ty / nrm);
        g[i].dz = (float)(1.0 / nrm);
        g[i].pad = 0.f;
        prefix[i + 1] = prefix[i] + j.ray_count;
    }
    return nullptr;
}

// Work list of visible secondary rays of the split adjoint (and the forward's
// tape of it): per incident ray its state at the DOE and its items, each item
// one secondary ray that reached the sensor (ray, bin, U~), in bin order.
struct SplitBufs {
    RayAtDoe* rinfo;             // [n] incident state at the DOE
    int* iray;                   // [cap] work list: incident ray
    int* ibin;                   // [cap] bin
    float2* iU;                  // [cap] U~ of that bin
    float2* igU;                 // [cap] dL/dU~
    long long* voff;             // [n] first work item of ray
    int* vcnt;                   // [n] number of work items of ray
    float* rsum;                 // [n][6] per-ray geometric sums
    unsigned long long* counter; // work-list allocator (may exceed cap: overflow)
    long long cap;
    // forward with a mask: epoch[0] counts such launches (graph replays
    // included), epoch[1] is the count at the launch that wrote the tape
    unsigned long long* epoch;
};

struct RaysOut {
    float *ox, *oy, *oz, *dx, *dy, *dz, *are, *aim;
    double* opl;
};

struct EmitOut {
    float *dx, *dy, *dz, *are, *aim;
    int* bin;
    float *hx, *hy, *hz;
    double* opl;
};

// ------------------------------------------------------------------ sizes
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
// patch X (M rows of stride M + 1, room for M rows of M + 2 staged samples),
// twiddles, two phase vectors, the tile's incident states
__host__ __device__ inline size_t sampled_scratch_offset(int M) {
    return align16(sizeof(float2) * (size_t)(M * (M + 2) + 3 * M) + sizeof(RayAtDoe) * RW_TILE);
}
// block culling (exhaustive emission): one bit per 8 x 8 block of bins and
// incident ray (set: the block is kept); the forward stages the current
// ray's visibility words and the tape's per-warp counts in shared memory
__host__ __device__ constexpr int cull_keep_words(int M) { return ((M / 8) * (M / 8) + 31) / 32; }
__host__ __device__ constexpr size_t cull_scratch_bytes(int M) {
    return ((sizeof(unsigned) * (size_t)(M * M / 32 + RW_THREADS / 32 + 4)) + 15) & ~size_t(15);
}
// Candidate queue of the sampled forward's draws, per warp: RW_GQ entries of
// (Philox word, lane << 16 | bin), each lane's packed best key
// (order(score) << 32 | ~bin: the maximum is the best score, then the lowest
// bin) and a fill counter.
#define RW_GQ 512
// with helper warps (16 warps in all) each warp's queue holds half as many
#define RW_GQ_HELPED 256
__host__ __device__ constexpr size_t gumbel_warp_queue_bytes(int gq) {
    return (size_t)gq * 8 + 32 * 8 + 16;
}
__host__ __device__ constexpr size_t gumbel_queue_bytes(int nwarps = RW_THREADS / 32,
                                                        int gq = RW_GQ) {
    return (size_t)nwarps * gumbel_warp_queue_bytes(gq);
}
// sampled forward scratch: p and screening words per bin, chosen bin per
// draw, reduction, then the per-warp candidate queues (16-byte aligned)
__host__ __device__ inline size_t sampled_queue_offset(int M, int n_ssr) {
    return align16(8 * (size_t)M * M + sizeof(int) * (size_t)n_ssr + 128);
}
// hw: helper warps of the sampled forward (see k_forward)
inline size_t forward_smem_bytes(int M, int emit = RW_EMIT_EXHAUSTIVE, int n_ssr = 0,
                                 int hw = 0) {
    size_t b = sampled_scratch_offset(M);
    if (emit == RW_EMIT_SAMPLED)
        b += sampled_queue_offset(M, n_ssr) +
             (hw ? gumbel_queue_bytes(RW_THREADS / 32 + hw, RW_GQ_HELPED) : gumbel_queue_bytes());
    else b += cull_scratch_bytes(M);
    return b;
}

// ------------------------------------------------------------------ Philox4x32-10
// Salmon et al., SC'11: ten rounds with multipliers 0xD2511F53, 0xCD9E8D57
// and Weyl key increments 0x9E3779B9, 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}
// (0, 1) uniform from 23 bits; exact in float.
__device__ __forceinline__ float u01(uint32_t w) {
    return ((float)(w >> 9) + 0.5f) * 1.1920928955078125e-7f;
}

// ------------------------------------------------------------------ jobs
__device__ __forceinline__ int find_job(const long long* prefix, int njob, long long g) {
    int lo = 0, hi = njob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------ A2 conformal hit
// Run t from the ray point (x, y, zld) (zld: local to the DOE vertex) to a
// conformal DOE substrate, in double.  Sphere: FP32 root refined by two FP64
// Newton steps on c |Q|^2 - 2 Q_z = 0.  Gaussian bump sag(s) = h
// exp(-s / (2 w^2)): Newton in double on g(t) = zld + t dz - sag(|q(t)|^2),
// started on the plane through the sag at the ray's (x, y).  False if missed
// (status bit on non-convergence).
__device__ __forceinline__ bool conformal_hit(const DSurf& S, float x, float y, double zld,
                                              float dx, float dy, float dz, double& t,
                                              unsigned* status) {
    if (S.kind == RW_GAUSS) {
        const double h = S.cd, iw2 = 0.5 / (S.kd * S.kd);
        const double X0 = x, Y0 = y, DX = dx, DY = dy, DZ = dz;
        t = (h * exp(-(X0 * X0 + Y0 * Y0) * iw2) - zld) / DZ;
        for (int it = 0; it < 40; ++it) {
            const double qx = X0 + t * DX, qy = Y0 + t * DY;
            const double e = h * exp(-(qx * qx + qy * qy) * iw2);
            const double gp = DZ + 2.0 * iw2 * e * (qx * DX + qy * DY);
            if (gp == 0.0) break;
            const double step = (zld + t * DZ - e) / gp;
            t -= step;
            if (fabs(step) <= 1e-13 * (1.0 + fabs(t))) return true;
        }
        if (status) atomicOr(status, RW_ST_NOTCONV);
        return false;
    }
    float tf;
    if (!intersect_local(S, x, y, (float)zld, dx, dy, dz, tf, status)) return false;
    t = (double)tf;
    const double c = S.cd;
    for (int it = 0; it < 2; ++it) {
        double qx = (double)x + t * dx, qy = (double)y + t * dy, qz = zld + t * dz;
        double f = c * (qx * qx + qy * qy + qz * qz) - 2.0 * qz;
        double fp = 2.0 * c * (qx * dx + qy * dy + qz * dz) - 2.0 * dz;
        if (fp == 0.0) return false;
        t -= f / fp;
    }
    return true;
}

// conformal_hit from a ray state in double (the FP64 trace before the DOE):
// the sphere's root in closed form in double, the bump as above.
__device__ __forceinline__ bool conformal_hit(const DSurf& S, double x, double y, double zld,
                                              double dx, double dy, double dz, double& t,
                                              unsigned* status) {
    if (S.kind == RW_GAUSS) {
        const double h = S.cd, iw2 = 0.5 / (S.kd * S.kd);
        t = (h * exp(-(x * x + y * y) * iw2) - zld) / dz;
        for (int it = 0; it < 40; ++it) {
            const double qx = x + t * dx, qy = y + t * dy;
            const double e = h * exp(-(qx * qx + qy * qy) * iw2);
            const double gp = dz + 2.0 * iw2 * e * (qx * dx + qy * dy);
            if (gp == 0.0) break;
            const double step = (zld + t * dz - e) / gp;
            t -= step;
            if (fabs(step) <= 1e-13 * (1.0 + fabs(t))) return true;
        }
        if (status) atomicOr(status, RW_ST_NOTCONV);
        return false;
    }
    return intersect_local_d(S, x, y, zld, dx, dy, dz, t, status);
}

// ------------------------------------------------------------------ A1 + A2
// Trace incident ray g (concatenated job order) to the DOE, build the
// tangent frame and everything the patch step needs.  The DOE hit is
// computed in double (planar: one division; conformal: FP32 sphere root
// refined by two FP64 Newton steps on c|Q|^2 - 2 Q_z = 0).
// EXACT = false (the block culling): the run to the DOE in FP32, enough for
// enclosures with a two-pixel margin; a ray the FP32 run loses gets
// alive = 2 ("unknown": the culling keeps all its blocks, the forward's FP64
// run decides).
template <bool EXACT = true>
__device__ __forceinline__ void incident_to_doe(const DSys& sys, const DJob* __restrict__ jobs,
                                                const long long* __restrict__ prefix, int njob,
                                                long long total, const RaysIn& rays,
                                                long long g, RayAtDoe& R, unsigned* status) {
    R.alive = 0;
    R.gid = g;
    if (g >= total) return;
    const int j = find_job(prefix, njob, g);
    const DJob& J = jobs[j];
    const long long ri = J.off + (g - prefix[j]);
    R.rid = ri;
    if constexpr (!EXACT) R.alive = 2;      // every early return below: unknown
    double xd, yd, zd, dxd, dyd, dzd;
    double opl = rays.opl[ri];
    const DSurf& S = sys.s[sys.doe_index];
    if constexpr (EXACT) {
        // the run to the DOE in double (see trace_one_d), from the float ray
        xd = rays.ox[ri]; yd = rays.oy[ri]; zd = rays.oz[ri];
        dxd = rays.dx[ri]; dyd = rays.dy[ri]; dzd = rays.dz[ri];
        for (int s = 0; s < sys.doe_index; ++s)
            if (!trace_one_d(sys.s[s], xd, yd, zd, dxd, dyd, dzd, opl, status)) return;
    } else {
        float x = rays.ox[ri], y = rays.oy[ri], zl = rays.oz[ri];
        float dx = rays.dx[ri], dy = rays.dy[ri], dz = rays.dz[ri];
        const double oz = (double)zl;
        for (int s = 0; s < sys.doe_index; ++s)
            if (!trace_one<true>(sys.s[s], x, y, zl, dx, dy, dz, opl, nullptr)) return;
        xd = x; yd = y; dxd = dx; dyd = dy; dzd = dz;
        zd = (sys.doe_index == 0) ? oz : (double)zl + sys.s[sys.doe_index - 1].z;
    }
    const double zld = zd - S.z;
    if (dzd == 0.0) return;
    double t;
    float nx, ny, nz;
    if (!sys.conformal) {
        t = -zld / dzd;
    } else if (!conformal_hit(S, xd, yd, zld, dxd, dyd, dzd, t, EXACT ? status : nullptr)) {
        return;
    }
    const float dx = (float)dxd, dy = (float)dyd, dz = (float)dzd;
    const double pxd = __dadd_rn(xd, __dmul_rn(t, dxd));
    const double pyd = __dadd_rn(yd, __dmul_rn(t, dyd));
    const double pzl = sys.conformal ? zld + t * dzd : 0.0;   // planar: on the plane
    // the tangent frame in double, rounded once: every secondary direction is
    // built from it, and on an oblique field a float frame's ~1e-7 error moves
    // a ray's whole fan by nanometres at a sensor tens of mm away
    double nxd = 0.0, nyd = 0.0, nzd = 1.0;
    if (S.kind == RW_GAUSS && sys.conformal) {
        // normal grad(z - sag) with -dsag/dx = x h e^{-s/(2 w^2)} / w^2 (same for y)
        const double iw2 = 0.5 / (S.kd * S.kd);
        const double e = S.cd * exp(-(pxd * pxd + pyd * pyd) * iw2);
        const double mx = 2.0 * iw2 * e * pxd, my = 2.0 * iw2 * e * pyd;
        const double inv = 1.0 / sqrt(mx * mx + my * my + 1.0);
        nxd = mx * inv; nyd = my * inv; nzd = inv;
    } else if (sys.conformal) {
        const double c = S.cd;
        const double s2 = pxd * pxd + pyd * pyd;
        const double a = 1.0 - c * c * s2;
        if (a <= 0.0) return;
        nxd = -c * pxd; nyd = -c * pyd; nzd = sqrt(a);
    }
    if (nxd * dxd + nyd * dyd + nzd * dzd < 0.0) { nxd = -nxd; nyd = -nyd; nzd = -nzd; }
    // u = normalise(x - (x.n) n), v = n x u
    double uxd = 1.0 - nxd * nxd, uyd = -nxd * nyd, uzd = -nxd * nzd;
    const double invu = 1.0 / sqrt(uxd * uxd + uyd * uyd + uzd * uzd);
    uxd *= invu; uyd *= invu; uzd *= invu;
    const double vxd = nyd * uzd - nzd * uyd, vyd = nzd * uxd - nxd * uzd,
                 vzd = nxd * uyd - nyd * uxd;
    nx = (float)nxd; ny = (float)nyd; nz = (float)nzd;
    const float ux = (float)uxd, uy = (float)uyd, uz = (float)uzd;
    const float vx = (float)vxd, vy = (float)vyd, vz = (float)vzd;
    R.u[0] = ux; R.u[1] = uy; R.u[2] = uz;
    R.v[0] = vx; R.v[1] = vy; R.v[2] = vz;
    // R.n is the normal the secondary rays leave along: reversed by a mirror
    if (sys.reflective) { nx = -nx; ny = -ny; nz = -nz; }
    R.n[0] = nx; R.n[1] = ny; R.n[2] = nz;
    const float k0 = J.k0;
    R.kin_u = k0 * sys.n_in * (dx * ux + dy * uy + dz * uz);
    R.kin_v = k0 * sys.n_in * (dx * vx + dy * vy + dz * vz);
    R.K = k0 * sys.n_out;
    R.invK = 1.f / R.K;
    {
        const double rn = sys.n_in_d / (double)sys.n_out;
        const double tu = rn * (dxd * ux + dyd * uy + dzd * uz);   // on the float frame
        const double tv = rn * (dxd * vx + dyd * vy + dzd * vz);
        const double ts = J.lambda / ((double)sys.M * sys.pitch * (double)sys.n_out);
        R.tu = (float)tu; R.tu_lo = (float)(tu - (double)R.tu);
        R.tv = (float)tv; R.tv_lo = (float)(tv - (double)R.tv);
        R.tstep = (float)ts; R.tstep_lo = (float)(ts - (double)R.tstep);
    }
    R.px = (float)pxd; R.py = (float)pyd; R.pz = (float)pzl;
    R.pxd = pxd; R.pyd = pyd;
    R.a_re = rays.are[ri]; R.a_im = rays.aim[ri];
    R.opl = opl + sys.n_in_d * t * sqrt(dxd * dxd + dyd * dyd + dzd * dzd);
    R.job = j;
    R.cx = J.cx; R.cy = J.cy;
    {
        const double sx = pxd - J.cxd, sy = pyd - J.cyd;
        const double sl = (sys.sensor_z - S.z) - pzl;
        R.sx = (float)sx; R.sx_lo = (float)(sx - (double)R.sx);
        R.sy = (float)sy; R.sy_lo = (float)(sy - (double)R.sy);
        R.sl = (float)sl; R.sl_lo = (float)(sl - (double)R.sl);
    }
    const double p = sys.pitch;
    if (sys.gather == RW_GATHER_NEAREST) {
        const double cs = floor(pxd / p + (double)sys.W / 2.0);
        const double rs = floor(pyd / p + (double)sys.H / 2.0);
        R.c0 = (int)cs - sys.D / 2;
        R.r0 = (int)rs - sys.D / 2;
        R.s0 = (float)((((double)R.c0 - (double)sys.W / 2.0 + 0.5) * p - pxd) / (sys.M * p));
        R.t0 = (float)((((double)R.r0 - (double)sys.H / 2.0 + 0.5) * p - pyd) / (sys.M * p));
    } else {
        const double uc = pxd / p + (double)sys.W / 2.0 - 0.5;
        const double vc = pyd / p + (double)sys.H / 2.0 - 0.5;
        const double iu = floor(uc), iv = floor(vc);
        R.c0 = (int)iu; R.r0 = (int)iv;
        R.s0 = (float)(uc - iu); R.t0 = (float)(vc - iv);
    }
    R.alive = 1;
}

// ------------------------------------------------------------------ A3
__device__ __forceinline__ float2 tmap(const float2* __restrict__ T, int H, int W, int r, int c) {
    if ((unsigned)r < (unsigned)H && (unsigned)c < (unsigned)W) return __ldg(&T[(long long)r * W + c]);
    return make_float2(0.f, 0.f);
}

// Per-bin phase factors exp(-i k_j s_0), j in [-M/2, M/2), that refer the
// spectrum to the hit point.  Bilinear patches start at s_0 = -(D/2) p, so
// the factor is exp(i pi j D / M).
template <int M>
__device__ __forceinline__ void phase_factors(const DSys& sys, const RayAtDoe& R, float2* phu,
                                              float2* phv) {
    const int t = ltid();
    if (t < M) {
        const float j = (float)(t - M / 2);
        float s, c;
        if (sys.gather == RW_GATHER_NEAREST) {
            sincospif(-2.f * j * R.s0, &s, &c);
            phu[t] = make_float2(c, s);
            sincospif(-2.f * j * R.t0, &s, &c);
            phv[t] = make_float2(c, s);
        } else {
            sincospif(j / (float)(M / sys.D), &s, &c);
            phu[t] = make_float2(c, s);
            phv[t] = make_float2(c, s);
        }
    }
}

// Fill the M x M buffer X (row stride M + 1) with the D x D patch in its
// top-left corner and zeros elsewhere (the padding), and phu/phv with the
// phase factors.
template <int M>
__device__ __forceinline__ void gather_patch(const DSys& sys, const RayAtDoe& R,
                                             const float2* __restrict__ T, float2* X,
                                             float2* phu, float2* phv) {
    constexpr int S = Patch<M>::S;
    const int H = sys.H, W = sys.W, D = sys.D;
    if (sys.gather == RW_GATHER_NEAREST) {
        for (int f = threadIdx.x; f < M * M; f += RW_THREADS) {
            const int b = f / M, a = f - (f / M) * M;
            X[b * S + a] = (a < D && b < D) ? tmap(T, H, W, R.r0 + b, R.c0 + a)
                                            : make_float2(0.f, 0.f);
        }
    } else {
        for (int f = threadIdx.x; f < M * M; f += RW_THREADS) {
            const int b = f / M, a = f - (f / M) * M;
            if (a >= D || b >= D) { X[b * S + a] = make_float2(0.f, 0.f); continue; }
            const float oa = (float)(a - D / 2), ob = (float)(b - D / 2);
            const float fu = R.s0 + oa * R.u[0] + ob * R.v[0];
            const float fv = R.t0 + oa * R.u[1] + ob * R.v[1];
            const float iuf = floorf(fu), ivf = floorf(fv);
            const float wu = fu - iuf, wv = fv - ivf;
            const int i0 = R.c0 + (int)iuf, j0 = R.r0 + (int)ivf;
            float2 t00 = tmap(T, H, W, j0, i0), t10 = tmap(T, H, W, j0, i0 + 1);
            float2 t01 = tmap(T, H, W, j0 + 1, i0), t11 = tmap(T, H, W, j0 + 1, i0 + 1);
            const float w00 = (1.f - wu) * (1.f - wv), w10 = wu * (1.f - wv);
            const float w01 = (1.f - wu) * wv, w11 = wu * wv;
            X[b * S + a] = make_float2(w00 * t00.x + w10 * t10.x + w01 * t01.x + w11 * t11.x,
                                       w00 * t00.y + w10 * t10.y + w01 * t01.y + w11 * t11.y);
        }
    }
    phase_factors<M>(sys, R, phu, phv);
}

// ------------------------------------------------------------------ A3 by bulk copies
// A nearest-pixel patch without padding (D = M = 64) whose rows r0 .. r0+63
// and columns c0 .. c0+63 lie inside a map of even width: row b is fetched
// as the M + 2 samples from column c0 & ~1 (a 16-byte aligned source) by one
// asynchronous bulk copy to stage + b (M + 2); the first FFT stage reads the
// patch at column offset c0 & 1 (fft2d_staged).
#define RW_BULK_WAIT (1ll << 26)   // polls of the copy barrier before giving up

template <int M>
__device__ __forceinline__ bool bulk_patch_ok(const DSys& sys, const RayAtDoe& R) {
    return M == 64 && sys.gather == RW_GATHER_NEAREST && sys.D == M && (sys.W & 1) == 0 &&
           R.r0 >= 0 && R.r0 + M <= sys.H && R.c0 >= 0 && (R.c0 & ~1) + M + 2 <= sys.W;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                 "[%0], [%1], %2, [%3];"
                 :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

// Warp 0 issues the M row copies (lane 0 first posts the byte count).
template <int M>
__device__ __forceinline__ void bulk_patch_issue(const DSys& sys, const RayAtDoe& R,
                                                 const float2* __restrict__ T, float2* stage,
                                                 uint64_t* bar) {
    constexpr uint32_t ROW = (M + 2) * sizeof(float2);
    const int lane = threadIdx.x & 31;
    if (lane == 0) mbar_expect_tx(bar, ROW * M);
    __syncwarp();
    const int ca = R.c0 & ~1;
    for (int b = lane; b < M; b += 32)
        bulk_g2s(stage + b * (M + 2), T + (long long)(R.r0 + b) * sys.W + ca, ROW, bar);
}

// ------------------------------------------------------------------ A6 + A7
// Trace a secondary ray from the DOE hit through the remaining surfaces to
// the sensor; returns false if dropped.  Position is left in (x, y).
// Run from a point at local z = zl (relative to the last surface's vertex)
// to the sensor plane: moves (x, y) there and returns the run t; with OPL
// the run is formed in double (see trace_one) and n_s t |d| is added to opl.
template <bool OPL>
__device__ __forceinline__ bool sensor_segment(const DSys& sys, float& x, float& y, float zl,
                                               float dx, float dy, float dz, double& opl,
                                               float& t) {
    if (dz == 0.f) return false;
    if (OPL) {
        const double td = ((double)sys.sensor_gap - (double)zl) / (double)dz;
        t = (float)td;
        opl += (double)sys.n_sensor * td * dnorm(dx, dy, dz);
    } else {
        t = -(zl - sys.sensor_gap) / dz;
    }
    x = fmaf(t, dx, x);
    y = fmaf(t, dy, y);
    return true;
}

template <bool OPL>
__device__ __forceinline__ bool trace_to_sensor(const DSys& sys, float& x, float& y, float& zl,
                                                float& dx, float& dy, float& dz, double& opl,
                                                unsigned* status) {
    for (int s = sys.doe_index + 1; s < sys.nsurf; ++s)
        if (!trace_one<OPL>(sys.s[s], x, y, zl, dx, dy, dz, opl, status)) return false;
    float t;
    return sensor_segment<OPL>(sys, x, y, zl, dx, dy, dz, opl, t);
}

// Bilinear |a|^2 deposit.  The image is accumulated in double: a focal
// pixel can receive ~1e6 deposits, and float accumulation there would drop
// small contributions.
// Where a secondary ray leaving the DOE along (dx, dy, dz) meets the sensor
// plane, relative to the job's window centre, when the DOE is the last
// surface: (p - c) + L (dx, dy) / dz with p - c and L from the incident ray
// in double (RayAtDoe::sx, sy, sl).  Evaluated in float pairs: the run is
// tens of mm and the window centre of an oblique field tens of mm off axis,
// where a float coordinate is only good to ~2 nm (1e-3 of a 2 um pixel).
__device__ __forceinline__ void sensor_offset(const RayAtDoe& R, float dx, float dy, float dz,
                                              float& ox, float& oy) {
    const float iz = __frcp_rn(dz);
    const float d2[2] = {dx, dy};
    const float p_hi[2] = {R.sx, R.sy}, p_lo[2] = {R.sx_lo, R.sy_lo};
    float o[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        // q = d / dz as hi + lo
        const float q = d2[c] * iz;
        const float ql = fmaf(-q, dz, d2[c]) * iz;
        // L q as hi + lo
        const float m = R.sl * q;
        const float ml = fmaf(R.sl, ql, fmaf(R.sl_lo, q, fmaf(R.sl, q, -m)));
        // (p_hi + m) + (p_lo + ml), the first sum exactly (two-sum)
        const float s = p_hi[c] + m;
        const float bb = s - p_hi[c];
        const float err = (p_hi[c] - (s - bb)) + (m - bb);
        o[c] = s + (err + (p_lo[c] + ml));
    }
    ox = o[0];
    oy = o[1];
}

__device__ __forceinline__ bool splat_bilinear(const DSys& sys, float cx, float cy, float x,
                                               float y, float w, double* __restrict__ img) {
    const float u = (x - cx) * sys.inv_spitch + 0.5f * sys.nx - 0.5f;
    const float v = (y - cy) * sys.inv_spitch + 0.5f * sys.ny - 0.5f;
    if (!(u > -1.f && v > -1.f && u < (float)sys.nx && v < (float)sys.ny)) return false;
    const float fi = floorf(u), fj = floorf(v);
    const int i0 = (int)fi, j0 = (int)fj;
    const float fu = u - fi, fv = v - fj;
    const int nx = sys.nx, ny = sys.ny;
    if (j0 >= 0) {
        if (i0 >= 0) atomicAdd(img + j0 * nx + i0, (double)(w * (1.f - fu) * (1.f - fv)));
        if (i0 + 1 < nx) atomicAdd(img + j0 * nx + i0 + 1, (double)(w * fu * (1.f - fv)));
    }
    if (j0 + 1 < ny) {
        if (i0 >= 0) atomicAdd(img + (j0 + 1) * nx + i0, (double)(w * (1.f - fu) * fv));
        if (i0 + 1 < nx) atomicAdd(img + (j0 + 1) * nx + i0 + 1, (double)(w * fu * fv));
    }
    return true;
}

// Pixel range [i_lo, i_hi] x [j_lo, j_hi] of the Eq. 2 sum of a ray that
// meets the sensor plane at (x, y): the whole sensor, or +-window pixels
// around the nearest pixel.  False if the range is empty.  Also returns
// the wavelet's phase at the hit, k OPL reduced to [-pi, pi] in double.
__device__ __forceinline__ bool coherent_range(const DSys& sys, float k0, float cx, float cy,
                                               float x, float y, double opl, int& i_lo,
                                               int& i_hi, int& j_lo, int& j_hi, float& phb) {
    const double TWO_PI = 6.283185307179586;
    double ph0 = (double)k0 * opl;
    ph0 -= TWO_PI * rint(ph0 / TWO_PI);
    phb = (float)ph0;
    const float u = (x - cx) * sys.inv_spitch + 0.5f * sys.nx - 0.5f;
    const float v = (y - cy) * sys.inv_spitch + 0.5f * sys.ny - 0.5f;
    if (!(u == u) || !(v == v)) return false;
    i_lo = 0; i_hi = sys.nx - 1; j_lo = 0; j_hi = sys.ny - 1;
    if (sys.window > 0) {
        const float ic = rintf(u), jc = rintf(v);
        if (ic < -(float)sys.window - 1.f || ic > (float)(sys.nx + sys.window)) return false;
        if (jc < -(float)sys.window - 1.f || jc > (float)(sys.ny + sys.window)) return false;
        i_lo = max(i_lo, (int)ic - sys.window); i_hi = min(i_hi, (int)ic + sys.window);
        j_lo = max(j_lo, (int)jc - sys.window); j_hi = min(j_hi, (int)jc + sys.window);
    }
    return i_lo <= i_hi && j_lo <= j_hi;
}

// Eq. 2: add a exp(i k (OPL + n_s d_t.((X,Y) - r))) d_z over the window.
__device__ __forceinline__ void splat_coherent(const DSys& sys, float k0, float cx, float cy,
                                               float x, float y, double opl, float dx,
                                               float dy, float dz, float2 a,
                                               float2* __restrict__ fld) {
    int i_lo, i_hi, j_lo, j_hi;
    float phb;
    if (!coherent_range(sys, k0, cx, cy, x, y, opl, i_lo, i_hi, j_lo, j_hi, phb)) return;
    const float kx = k0 * sys.n_sensor * dx, ky = k0 * sys.n_sensor * dy;
    const float2 ad = make_float2(a.x * dz, a.y * dz);
    // one sincos every 8 pixels of a row, rotations by the step kx * pitch between
    float st_s, st_c;
    sincosf(kx * sys.spitch, &st_s, &st_c);
    for (int j = j_lo; j <= j_hi; ++j) {
        const float Y = cy + ((float)j - 0.5f * sys.ny + 0.5f) * sys.spitch;
        float s = 0.f, c = 1.f;
        for (int i = i_lo; i <= i_hi; ++i) {
            if (((i - i_lo) & 7) == 0) {
                const float X = cx + ((float)i - 0.5f * sys.nx + 0.5f) * sys.spitch;
                sincosf(phb + kx * (X - x) + ky * (Y - y), &s, &c);
            } else {
                const float t = c * st_c - s * st_s;
                s = s * st_c + c * st_s;
                c = t;
            }
            float2* p = fld + j * sys.nx + i;
            atomicAdd(&p->x, ad.x * c - ad.y * s);
            atomicAdd(&p->y, ad.x * s + ad.y * c);
        }
    }
}

// Eq. 2 over the whole sensor (window 0) for the 32 secondary rays of a warp
// at once.  Every lane evaluates its wavelet (amplitude zero if `ok` is
// false) on the same group of 8 pixels; a transpose-reduction across the warp
// (9 shuffles per component) leaves the group's 8 sums in 8 lanes, which add
// them to the field: 8 atomics per group instead of 32 per pixel on one
// address.  Must be called by all 32 lanes of the warp together.
__device__ __forceinline__ void splat_coherent_warp(const DSys& sys, float k0, float cx, float cy,
                                                    bool ok, float x, float y, double opl,
                                                    float dx, float dy, float dz, float2 a,
                                                    float2* __restrict__ fld) {
    const int lane = threadIdx.x & 31;
    int i_lo, i_hi, j_lo, j_hi;
    float phb = 0.f;
    if (ok) ok = coherent_range(sys, k0, cx, cy, x, y, opl, i_lo, i_hi, j_lo, j_hi, phb);
    const float kx = ok ? k0 * sys.n_sensor * dx : 0.f;
    const float ky = ok ? k0 * sys.n_sensor * dy : 0.f;
    const float2 ad = ok ? make_float2(a.x * dz, a.y * dz) : make_float2(0.f, 0.f);
    if (!ok) { x = 0.f; y = 0.f; }
    const int nx = sys.nx, npx = sys.nx * sys.ny;
    // the pixel this lane adds after the reduction
    const int q_out = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    // along a row the phase grows by kx * pitch per pixel: a group of 8 pixels
    // in one row takes one sincos and 7 rotations by that step
    float st_s, st_c;
    sincosf(kx * sys.spitch, &st_s, &st_c);
    // the step to the power 4: pixels 4..7 of a group run as a second chain
    const float s2c = st_c * st_c - st_s * st_s, s2s = 2.f * st_c * st_s;
    const float s4c = s2c * s2c - s2s * s2s, s4s = 2.f * s2c * s2s;
    const bool rows8 = (nx & 7) == 0;
    for (int p0 = 0; p0 < npx; p0 += 8) {
        float re[8], im[8];
        if (rows8) {
            const int j = p0 / nx, i = p0 - j * nx;
            const float X = cx + ((float)i - 0.5f * sys.nx + 0.5f) * sys.spitch;
            const float Y = cy + ((float)j - 0.5f * sys.ny + 0.5f) * sys.spitch;
            float sn, cs;
            sincosf(phb + kx * (X - x) + ky * (Y - y), &sn, &cs);
            float er = ad.x * cs - ad.y * sn, ei = ad.x * sn + ad.y * cs;
            float fr = er * s4c - ei * s4s, fi = er * s4s + ei * s4c;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                re[q] = er;
                im[q] = ei;
                re[q + 4] = fr;
                im[q + 4] = fi;
                const float t = er * st_c - ei * st_s;
                ei = er * st_s + ei * st_c;
                er = t;
                const float u = fr * st_c - fi * st_s;
                fi = fr * st_s + fi * st_c;
                fr = u;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int p = p0 + q;
                re[q] = 0.f;
                im[q] = 0.f;
                if (p < npx) {
                    const int j = p / nx, i = p - j * nx;
                    const float X = cx + ((float)i - 0.5f * sys.nx + 0.5f) * sys.spitch;
                    const float Y = cy + ((float)j - 0.5f * sys.ny + 0.5f) * sys.spitch;
                    const float ph = phb + kx * (X - x) + ky * (Y - y);
                    float sn, cs;
                    sincosf(ph, &sn, &cs);
                    re[q] = ad.x * cs - ad.y * sn;
                    im[q] = ad.x * sn + ad.y * cs;
                }
            }
        }
        // 8 -> 4 (lanes xor 16), 4 -> 2 (xor 8), 2 -> 1 (xor 4): each lane keeps
        // the half of its pixels selected by its lane bit and receives the
        // partner's share of them
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool hi = lane & 16;
            const float sr = hi ? re[k] : re[k + 4], si = hi ? im[k] : im[k + 4];
            const float rr = __shfl_xor_sync(0xffffffffu, sr, 16);
            const float ri = __shfl_xor_sync(0xffffffffu, si, 16);
            re[k] = (hi ? re[k + 4] : re[k]) + rr;
            im[k] = (hi ? im[k + 4] : im[k]) + ri;
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const bool hi = lane & 8;
            const float sr = hi ? re[k] : re[k + 2], si = hi ? im[k] : im[k + 2];
            const float rr = __shfl_xor_sync(0xffffffffu, sr, 8);
            const float ri = __shfl_xor_sync(0xffffffffu, si, 8);
            re[k] = (hi ? re[k + 2] : re[k]) + rr;
            im[k] = (hi ? im[k + 2] : im[k]) + ri;
        }
        {
            const bool hi = lane & 4;
            const float sr = hi ? re[0] : re[1], si = hi ? im[0] : im[1];
            const float rr = __shfl_xor_sync(0xffffffffu, sr, 4);
            const float ri = __shfl_xor_sync(0xffffffffu, si, 4);
            re[0] = (hi ? re[1] : re[0]) + rr;
            im[0] = (hi ? im[1] : im[0]) + ri;
        }
        re[0] += __shfl_xor_sync(0xffffffffu, re[0], 2);
        im[0] += __shfl_xor_sync(0xffffffffu, im[0], 2);
        re[0] += __shfl_xor_sync(0xffffffffu, re[0], 1);
        im[0] += __shfl_xor_sync(0xffffffffu, im[0], 1);
        const int p = p0 + q_out;
        if ((lane & 3) == 0 && p < npx && (re[0] != 0.f || im[0] != 0.f)) {
            atomicAdd(&fld[p].x, re[0]);
            atomicAdd(&fld[p].y, im[0]);
        }
    }
}

// Direction of spectral bin (ju, jv) for the incident state R; false if
// evanescent.  In units of K = k0 n_out: (a_u, a_v) = (tu, tv) + tstep (ju, jv)
// (one rounding each), a_n = sqrt(1 - a_u^2 - a_v^2) correctly rounded (the
// run to the next surface divides by it), d = a_u u + a_v v + a_n n.  Near
// grazing (a_n^2 < 1e-2) the float rounding of a_u, a_v would be amplified
// by 1 / a_n, so a_n^2 is formed in double from the double-float (tu, tv,
// tstep).
template <bool FAST = false>
__device__ __forceinline__ bool bin_direction(const DSys& sys, const RayAtDoe& R, int ju, int jv,
                                              float& dx, float& dy, float& dz) {
    const float au = fmaf(R.tstep, (float)ju, R.tu);
    const float av = fmaf(R.tstep, (float)jv, R.tv);
    float an2 = fmaf(-av, av, fmaf(-au, au, 1.f));
    if (an2 < 1e-2f) {
        const double aud = ((double)R.tstep + (double)R.tstep_lo) * ju + ((double)R.tu + (double)R.tu_lo);
        const double avd = ((double)R.tstep + (double)R.tstep_lo) * jv + ((double)R.tv + (double)R.tv_lo);
        an2 = (float)fma(-avd, avd, fma(-aud, aud, 1.0));
    }
    if (!(an2 > 0.f)) return false;
    const float an = sqrtf(an2);
    if (FAST && !sys.conformal) {
        // planar DOE: u = x, v = (0, s, 0), outgoing normal (0, 0, +-s), s = +-1
        dx = au;
        dy = av * R.v[1];
        dz = an * R.n[2];
        return true;
    }
    dx = fmaf(au, R.u[0], fmaf(av, R.v[0], an * R.n[0]));
    dy = fmaf(au, R.u[1], fmaf(av, R.v[1], an * R.n[1]));
    dz = fmaf(au, R.u[2], fmaf(av, R.v[2], an * R.n[2]));
    return true;
}

// U~ of bin (jui - M/2, jvi - M/2) from the FFT output X (row stride S).
template <int M, int S = Patch<M>::S>
__device__ __forceinline__ float2 spectrum_at(const float2* X, const float2* phu, const float2* phv,
                                              int jui, int jvi, float norm) {
    int mu = jui + M / 2; if (mu >= M) mu -= M;
    int mv = jvi + M / 2; if (mv >= M) mv -= M;
    return cscale(cmul(cmul(X[mv * S + mu], phu[jui]), phv[jvi]), norm);
}

// Trace one secondary ray and deposit it; returns true if it reached the
// sensor plane with any bilinear tap on the sensor (incoherent mode).
// Incoherent: deposits w = |a|^2; coherent: sums the complex amplitude a.
template <int MODE, int NS>
__device__ __forceinline__ bool deposit(const DSys& sys, const DJob& J, const RayAtDoe& R,
                                        float dx, float dy, float dz, float2 a, float w,
                                        double* __restrict__ psf, float2* __restrict__ field,
                                        unsigned* status) {
    float x = R.px, y = R.py, zl = R.pz;
    double opl = R.opl;
    const long long npx = (long long)sys.nx * sys.ny;
    if (MODE == MODE_SPLAT && NS == 0) {
        float ox, oy;
        sensor_offset(R, dx, dy, dz, ox, oy);
        return splat_bilinear(sys, 0.f, 0.f, ox, oy, w, psf + (long long)J.out * npx);
    } else if (MODE == MODE_SPLAT && NS > 0) {
        if (!fast_to_sensor<NS>(sys, x, y, zl, dx, dy, dz)) return false;
        return splat_bilinear(sys, R.cx, R.cy, x, y, w, psf + (long long)J.out * npx);
    } else if (MODE == MODE_SPLAT) {
        if (!trace_to_sensor<false>(sys, x, y, zl, dx, dy, dz, opl, status)) return false;
        return splat_bilinear(sys, R.cx, R.cy, x, y, w, psf + (long long)J.out * npx);
    } else {
        if (!trace_to_sensor<true>(sys, x, y, zl, dx, dy, dz, opl, status)) return false;
        splat_coherent(sys, J.k0, R.cx, R.cy, x, y, opl, dx, dy, dz, a,
                       field + (long long)J.out * npx);
        return true;
    }
}

template <int M>
__device__ __forceinline__ void emit_dead(const DSys& sys, long long g, long long total,
                                          const EmitOut& eo) {
    if (g >= total) return;
    const long long S = (sys.emit == RW_EMIT_EXHAUSTIVE) ? (long long)M * M : sys.n_ssr;
    for (long long b = threadIdx.x; b < S; b += RW_THREADS) {
        const long long s = g * S + b;
        eo.dx[s] = 0.f; eo.dy[s] = 0.f; eo.dz[s] = 0.f; eo.are[s] = 0.f; eo.aim[s] = 0.f;
        if (eo.bin) eo.bin[s] = -1;
    }
    if (threadIdx.x == 0) { eo.hx[g] = 0.f; eo.hy[g] = 0.f; eo.hz[g] = 0.f; eo.opl[g] = 0.0; }
}

// ------------------------------------------------------------------ A5 exhaustive
// Ray phase: trace only the bins of kept blocks, packed over the CTA's
// threads (converged warps).  Dropped bins cannot deposit, so the image and
// the visibility mask equal those of tracing every bin.
//
// With a tape (tape.iray != null, needs vis), the secondary rays that
// reached the sensor are also appended to the adjoint's work list: one
// allocation per incident ray, items (ray, bin, U~) in bin order, so the
// adjoint need not recompute the patch and its spectrum.  An allocation past
// tape.cap writes nothing; the counter still grows, which tells the host.
template <int M, int NS>
__device__ __forceinline__ void emit_culled(const DSys& sys, const DJob& J, const RayAtDoe& R,
                                            const float2* X, const float2* phu,
                                            const float2* phv, double* psf, long long g,
                                            unsigned* status, unsigned* __restrict__ vis,
                                            const unsigned* keepw, unsigned* vw,
                                            const SplitBufs& tape) {
    // keepw: this ray's kept-block words (shared); vw: its visibility words,
    // zero on entry and left zero on return (each word is read and cleared by
    // the thread that owns it)
    constexpr int S = Patch<M>::S;
    constexpr int NW = M * M / 32, B8 = M / 8, KW = cull_keep_words(M);
    static_assert(NW <= RW_THREADS, "one visibility word per thread at most");
    unsigned keep[KW];
    int nkept = 0;
#pragma unroll
    for (int w = 0; w < KW; ++w) {
        keep[w] = keepw[w];
        nkept += __popc(keep[w]);
    }
    const float2 ain = make_float2(R.a_re, R.a_im);
    const float norm = sys.norm;
    const float ain2 = (ain.x * ain.x + ain.y * ain.y) * norm * norm;
    for (int i = ltid(); i < 64 * nkept; i += RW_THREADS) {
        // block of the (i / 64)-th set bit, bin i % 64 inside it
        int k = i >> 6, bi = 0;
#pragma unroll
        for (int w = 0; w < KW; ++w) {
            const int c = __popc(keep[w]);
            if (k >= 0 && k < c) bi = w * 32 + (int)__fns(keep[w], 0u, k + 1);
            k -= c;
        }
        const int q = i & 63;
        const int jui = (bi % B8) * 8 + (q & 7), jvi = (bi / B8) * 8 + (q >> 3);
        float dx, dy, dz;
        if (!bin_direction<true>(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz)) continue;
        int mu = jui + M / 2; if (mu >= M) mu -= M;
        int mv = jvi + M / 2; if (mv >= M) mv -= M;
        const float2 xm = X[mv * S + mu];
        const float w2 = ain2 * (xm.x * xm.x + xm.y * xm.y);
        if (deposit<MODE_SPLAT, NS>(sys, J, R, dx, dy, dz, make_float2(0.f, 0.f), w2, psf,
                                    nullptr, status) && vis) {
            const int f = jvi * M + jui;
            atomicOr(&vw[f >> 5], 1u << (f & 31));
        }
    }
    if (vis) {
        main_sync();
        for (int i = ltid(); i < NW; i += RW_THREADS) vis[g * (long long)NW + i] = vw[i];
        if (!tape.iray)
            for (int i = ltid(); i < NW; i += RW_THREADS) vw[i] = 0u;
    }
    if (vis && tape.iray) {
        constexpr int KV = (NW + RW_THREADS - 1) / RW_THREADS;   // words per thread
        constexpr int NWARP = RW_THREADS / 32;
        int* wsum = reinterpret_cast<int*>(vw + NW);
        const int lane = ltid() & 31, warp = ltid() >> 5;
        unsigned word[KV];
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < KV; ++k) {
            const int wi = ltid() * KV + k;
            word[k] = wi < NW ? vw[wi] : 0u;
            if (wi < NW) vw[wi] = 0u;
            cnt += __popc(word[k]);
        }
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[warp] = incl;
        main_sync();
        if (ltid() == 0) {
            int t = 0;
            for (int w = 0; w < NWARP; ++w) { const int v = wsum[w]; wsum[w] = t; t += v; }
            long long base = 0;
            if (t > 0) base = (long long)atomicAdd(tape.counter, (unsigned long long)t);
            if (base + t > tape.cap) t = 0;
            tape.voff[g] = base;
            tape.vcnt[g] = t;
            wsum[NWARP] = (int)(base & 0x7fffffff);
            wsum[NWARP + 1] = (int)(base >> 31);
            wsum[NWARP + 2] = t;
        }
        main_sync();
        if (wsum[NWARP + 2] > 0) {
            long long pos = (long long)wsum[NWARP] + ((long long)wsum[NWARP + 1] << 31) +
                            wsum[warp] + (incl - cnt);
            const float norm = sys.norm;
#pragma unroll
            for (int k = 0; k < KV; ++k) {
                unsigned wk = word[k];
                while (wk) {
                    const int b = __ffs(wk) - 1;
                    wk &= wk - 1u;
                    const int f = (ltid() * KV + k) * 32 + b;
                    const int jvi = f / M, jui = f - (f / M) * M;
                    tape.iray[pos] = (int)g;
                    tape.ibin[pos] = f;
                    tape.iU[pos] = spectrum_at<M>(X, phu, phv, jui, jvi, norm);
                    ++pos;
                }
            }
        }
    }
}

template <int M, int MODE, int NS>
__device__ __forceinline__ void emit_exhaustive(const DSys& sys, const DJob& J, const RayAtDoe& R,
                                                const float2* X, const float2* phu,
                                                const float2* phv, double* psf, float2* field,
                                                const EmitOut& eo, long long g, unsigned* status,
                                                unsigned* __restrict__ vis,
                                                const unsigned* keepw, unsigned* vw,
                                                const SplitBufs& tape, int f0 = 0,
                                                int f1 = M * M) {
    // bins f0 .. f1-1 of the ray (a slice in coherent launches; both multiples
    // of RW_THREADS or M * M, so every warp runs the loop the same number of times)
    if constexpr (MODE == MODE_SPLAT && NS >= 0 && M <= 64) {
        if (keepw) {
            emit_culled<M, NS>(sys, J, R, X, phu, phv, psf, g, status, vis, keepw, vw, tape);
            return;
        }
    }
    constexpr int S = Patch<M>::S;
    const float2 ain = make_float2(R.a_re, R.a_im);
    const float norm = sys.norm;
    const float ain2 = (ain.x * ain.x + ain.y * ain.y) * norm * norm;
    if (MODE == MODE_EMIT && ltid() == 0) {
        eo.hx[g] = R.px; eo.hy[g] = R.py; eo.hz[g] = (float)((double)R.pz + sys.s[sys.doe_index].z);
        eo.opl[g] = R.opl;
    }
    for (int f = f0 + ltid(); f < f1; f += RW_THREADS) {
        const int jvi = f / M, jui = f - (f / M) * M;
        float dx, dy, dz;
        const bool prop = bin_direction<(NS >= 0)>(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz);
        if (MODE == MODE_EMIT) {
            const long long s = g * (long long)(M * M) + f;
            if (!prop) {
                eo.dx[s] = 0.f; eo.dy[s] = 0.f; eo.dz[s] = 0.f; eo.are[s] = 0.f; eo.aim[s] = 0.f;
            } else {
                const float2 a = cmul(ain, spectrum_at<M>(X, phu, phv, jui, jvi, norm));
                eo.dx[s] = dx; eo.dy[s] = dy; eo.dz[s] = dz; eo.are[s] = a.x; eo.aim[s] = a.y;
            }
            if (eo.bin) eo.bin[s] = f;
            continue;
        }
        if (MODE == MODE_COHERENT && sys.window == 0) {
            // whole-sensor sum: each lane traces its ray, the warp sums its 32 wavelets
            float x = R.px, y = R.py, zl = R.pz;
            double opl = R.opl;
            float2 a = make_float2(0.f, 0.f);
            bool ok = false;
            if (prop) {
                a = cmul(ain, spectrum_at<M>(X, phu, phv, jui, jvi, norm));
                ok = trace_to_sensor<true>(sys, x, y, zl, dx, dy, dz, opl, status);
            }
            __syncwarp();
            splat_coherent_warp(sys, J.k0, R.cx, R.cy, ok, x, y, opl, dx, dy, dz, a,
                                field + (long long)J.out * sys.nx * sys.ny);
            continue;
        }
        bool landed = false;
        if (prop) {
            float2 a = make_float2(0.f, 0.f);
            float w = 0.f;
            if (MODE == MODE_SPLAT) {
                // the incoherent deposit |a|^2 = |a_in|^2 |X_m|^2 norm^2 needs no phase factor
                int mu = jui + M / 2; if (mu >= M) mu -= M;
                int mv = jvi + M / 2; if (mv >= M) mv -= M;
                const float2 xm = X[mv * S + mu];
                w = ain2 * (xm.x * xm.x + xm.y * xm.y);
            } else {
                a = cmul(ain, spectrum_at<M>(X, phu, phv, jui, jvi, norm));
            }
            landed = deposit<MODE, NS>(sys, J, R, dx, dy, dz, a, w, psf, field, status);
        }
        if (MODE == MODE_SPLAT && vis) {
            // one visibility bit per secondary ray: bin f -> word g * M^2/32 + f/32
            const unsigned word = __ballot_sync(0xffffffffu, landed);
            if ((ltid() & 31) == 0) vis[g * (long long)(M * M / 32) + (f >> 5)] = word;
        }
    }
}

// ------------------------------------------------------------------ A5 sampled
// Gumbel-max: draw i picks argmax_j (log p_j + g_ij) over propagating bins,
// g = -log(-log u), u from Philox (counter (j>>2, i, ray, offset), word j&3),
// ray = the incident ray's index in the caller's ray arrays.
// Coherent sensor: p ~ |U~|, a = a_in U~ / (N p).  Incoherent: p ~ |U~|^2,
// a = a_in U~ / sqrt(N p) so that |a|^2 is the unbiased power weight.
//
// Screening (exact).  Bin j scores above -log(tau) only if E_j = -log u_j <
// tau p_j, i.e. u_j > exp(-tau p_j): its 23-bit uniform exceeds a per-bin
// threshold that is fixed for the whole patch.  A draw compares every
// Philox word with that threshold (integer compares, no logarithm) and
// evaluates the score, with the same float expression as a full scan, only
// for the few candidates (tau of them on average).  The thresholds are
// rounded towards more candidates, and a candidate is accepted only when its
// score clears -log(tau) by a margin far above float rounding; otherwise the
// draw rescans every bin.  The chosen bin is therefore always the full
// scan's (ties: the lowest bin).
#define RW_GUMBEL_TAU 12.0f
#define RW_GUMBEL_FLOOR (-2.4849066497880004f + 1e-3f)   // -log(tau) + margin

// score of bin j with probability p > 0 and Philox word w: the decision rule
__device__ __forceinline__ float gumbel_score(float p, uint32_t w) {
    return logf(p) - logf(-logf(u01(w)));
}

// Smallest Philox word with which a bin of probability p can score above
// -log(tau): u > exp(-tau p) implies (w >> 9) >= tm (tm rounded down).
__device__ __forceinline__ uint32_t gumbel_screen_word(float p) {
    if (!(p > 0.f)) return 0xffffffffu;
    const float e = expf(-RW_GUMBEL_TAU * p);
    const float tm = floorf(e * 8388608.f * (1.f - 1e-6f)) - 1.f;
    return tm <= 0.f ? 0u : ((uint32_t)tm << 9);
}

// E = -log u of the uniform of word w, to 1e-5 relative (it weighs the soft
// Gumbel-softmax terms of the adjoint, never a draw): near u = 1 (v = 1 - u
// < 1/32, where a logarithm of u loses relative accuracy) the series
// -log(1 - v) = v + v^2/2 + v^3/3 (truncation < v^3/4 = 8e-6 relative),
// elsewhere the hardware base-2 logarithm (absolute error ~2^-22.6 in log2,
// at most 4e-6 relative for u <= 31/32).
__device__ __forceinline__ float gumbel_E_fast(uint32_t w) {
    const float m = (float)(w >> 9);
    const float v = (8388607.5f - m) * 1.1920928955078125e-7f;            // 1 - u, exact
    const float series = v * (1.f + v * (0.5f + v * 0.33333334f));
    float lg;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"((m + 0.5f) * 1.1920928955078125e-7f));
    return v < 0.03125f ? series : -0.69314718f * lg;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void gumbel_keep(float sc, int jb, float& best, int& bj) {
    if (sc > best || (sc == best && jb < bj)) { best = sc; bj = jb; }
}

// Full scan of draw i (every propagating bin scored): the fallback when no
// screened candidate clears the floor.  p[j] = 0 marks bins that cannot be drawn.
template <int M, int STRIDE = 1>
__device__ __forceinline__ void gumbel_full_scan(const float* p, uint32_t i, uint32_t ray,
                                                 uint32_t off, uint32_t k0, uint32_t k1,
                                                 float& best, int& bj) {
    for (int G = 0; G < M * M / 4; ++G) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)G, i, ray, off), k0, k1);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float pj = p[(4 * G + q) * STRIDE];
            if (pj > 0.f) gumbel_keep(gumbel_score(pj, ws[q]), 4 * G + q, best, bj);
        }
    }
}

// Order-preserving map of a float to 32 bits (for packed atomic maxima).
__device__ __forceinline__ uint32_t float_order(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_unorder(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}


// Draws d0 .. d1-1 of one incident ray into sel[] (-1: no bin can be
// drawn).  The 32 lanes of a warp make 32 draws together, walking the bins in
// step so that the thresholds are broadcast reads; eight independent Philox
// blocks per step keep the integer pipes busy.  The rare screening
// candidates are only queued in the loop; the warp scores them together
// afterwards (or when the queue fills) and keeps each draw's best with a
// packed atomic maximum, so the scoring never diverges inside the loop.  A
// draw whose queue share overflowed, or whose best candidate does not clear
// the floor, rescans every bin.  Not inlined: the hot loop gets registers of
// its own, apart from the rest of the fused kernel.
template <int M, int GQ = RW_GQ>
__device__ __noinline__ void gumbel_draws(const float* __restrict__ p,
                                          const uint4* __restrict__ thr4, int* __restrict__ sel,
                                          int d0, int d1, uint32_t ray, uint32_t off,
                                          uint32_t k0, uint32_t k1, unsigned char* qmem) {
    constexpr int NG = M * M / 4, CH = 8;
    static_assert(NG % CH == 0, "bin groups in blocks of eight");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* wm = qmem + (size_t)warp * gumbel_warp_queue_bytes(GQ);
    uint2* wq = reinterpret_cast<uint2*>(wm);
    unsigned long long* wk = reinterpret_cast<unsigned long long*>(wm + GQ * 8);
    int* qn = reinterpret_cast<int*>(wm + GQ * 8 + 32 * 8);
    auto flush = [&]() {
        __syncwarp();
        const int n = min(*qn, GQ);
        for (int t = lane; t < n; t += 32) {
            const uint2 e = wq[t];
            const int jb = (int)(e.y & 0xffffu), il = (int)(e.y >> 16);
            const float sc = gumbel_score(p[jb], e.x);
            atomicMax(&wk[il], ((unsigned long long)float_order(sc) << 32) |
                                   (unsigned long long)(0xffffffffu - (uint32_t)jb));
        }
        __syncwarp();
        if (lane == 0) *qn = 0;
        __syncwarp();
    };
    for (int i0 = d0 + warp * 32; i0 < d1; i0 += (int)blockDim.x) {
        const uint32_t i = (uint32_t)(i0 + lane);
        wk[lane] = 0ull;
        if (lane == 0) *qn = 0;
        bool ovf = false;
        __syncwarp();
        for (int G = 0; G < NG; G += CH) {
            uint4 w[CH];
#pragma unroll
            for (int k = 0; k < CH; ++k)
                w[k] = philox4x32_10(make_uint4((uint32_t)(G + k), i, ray, off), k0, k1);
            unsigned mask = 0u;
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                const uint4 t = thr4[G + k];
                mask |= ((unsigned)(w[k].x >= t.x) | ((unsigned)(w[k].y >= t.y) << 1) |
                         ((unsigned)(w[k].z >= t.z) << 2) | ((unsigned)(w[k].w >= t.w) << 3))
                        << (4 * k);
            }
            if (mask) {
                const int n = __popc(mask);
                int c = atomicAdd(qn, n);
                if (c + n > GQ) {
                    ovf = true;
                } else {
#pragma unroll
                    for (int k = 0; k < CH; ++k) {
                        const uint32_t ws[4] = {w[k].x, w[k].y, w[k].z, w[k].w};
#pragma unroll
                        for (int r = 0; r < 4; ++r)
                            if ((mask >> (4 * k + r)) & 1u)
                                wq[c++] = make_uint2(ws[r], ((uint32_t)lane << 16) |
                                                                (uint32_t)(4 * (G + k) + r));
                    }
                }
            }
            __syncwarp();
            if (*qn > GQ / 2) flush();
        }
        flush();
        if ((int)i < d1) {
            const unsigned long long kk = wk[lane];
            float best = kk ? float_unorder((uint32_t)(kk >> 32)) : -INFINITY;
            int bj = kk ? (int)(0xffffffffu - (uint32_t)(kk & 0xffffffffull)) : 0x7fffffff;
            if (ovf || !(best > RW_GUMBEL_FLOOR)) {
                best = -INFINITY;
                bj = 0x7fffffff;
                gumbel_full_scan<M>(p, i, ray, off, k0, k1, best, bj);
            }
            sel[i] = (best > -INFINITY) ? bj : -1;
        }
        __syncwarp();
    }
}

// Probabilities of the patch's bins, shared by the forward and the adjoint so
// that both make the same draws: m_j = |U~_j|^2 (incoherent), |U~_j|
// (coherent) or 1 (uniform density) over propagating bins, p_j = m_j / S.
// Writes p[f * STRIDE] (0 for bins that cannot be drawn) and returns S;
// `red` holds >= 8 floats.  Ends with a barrier.
template <int M, int STRIDE = 1>
__device__ __forceinline__ float sampled_probs(const DSys& sys, const RayAtDoe& R,
                                               const float2* X, const float2* phu,
                                               const float2* phv, float* p, float* red) {
    const bool coh = sys.coherent != 0;
    float part = 0.f;
    for (int f = threadIdx.x; f < M * M; f += RW_THREADS) {
        const int jvi = f / M, jui = f - (f / M) * M;
        float dx, dy, dz;
        float m = 0.f;
        if (bin_direction(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz)) {
            const float2 U = spectrum_at<M>(X, phu, phv, jui, jvi, sys.norm);
            const float p2 = U.x * U.x + U.y * U.y;
            m = sys.uniform ? 1.f : (coh ? sqrtf(p2) : p2);
        }
        p[f * STRIDE] = m;
        part += m;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    main_sync();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    main_sync();
    float tot = 0.f;
    for (int w = 0; w < RW_THREADS / 32; ++w) tot += red[w];
    const float inv_tot = tot > 0.f ? 1.f / tot : 0.f;
    for (int f = threadIdx.x; f < M * M; f += RW_THREADS) p[f * STRIDE] *= inv_tot;
    main_sync();
    return tot;
}

// Shared scratch after the patch: p[M*M] floats, thr[M*M] words, sel[n_ssr]
// ints, red[32].
template <int M, int MODE, int NS, int GQ = RW_GQ>
__device__ __forceinline__ void emit_sampled(const DSys& sys, const DJob& J, const RayAtDoe& R,
                                             const float2* X, const float2* phu, const float2* phv,
                                             double* psf, float2* field, const EmitOut& eo,
                                             long long g, unsigned* status,
                                             unsigned char* scratch, int d0 = 0, int d1 = -1) {
    // draws d0 .. d1-1 (a slice in coherent launches; d0 a multiple of RW_THREADS)
    if (d1 < 0) d1 = sys.n_ssr;
    constexpr int NG = M * M / 4;
    float* p = reinterpret_cast<float*>(scratch);
    uint4* thr4 = reinterpret_cast<uint4*>(p + M * M);
    uint32_t* thr = reinterpret_cast<uint32_t*>(thr4);
    int* sel = reinterpret_cast<int*>(thr + M * M);
    float* red = reinterpret_cast<float*>(sel + sys.n_ssr);
    const bool coh = sys.coherent != 0;
    const float norm = sys.norm;
    sampled_probs<M>(sys, R, X, phu, phv, p, red);
    for (int f = threadIdx.x; f < M * M; f += RW_THREADS) thr[f] = gumbel_screen_word(p[f]);
    __syncthreads();           // CTA: helper warps (k_forward) join the draws
    gumbel_draws<M, GQ>(p, thr4, sel, d0, d1, (uint32_t)R.rid, (uint32_t)sys.rng_offset,
                        (uint32_t)(sys.seed & 0xffffffffull), (uint32_t)(sys.seed >> 32),
                        scratch + sampled_queue_offset(M, sys.n_ssr));
    __syncthreads();           // CTA
    const float2 ain = make_float2(R.a_re, R.a_im);
    if (MODE == MODE_EMIT && threadIdx.x == 0) {
        eo.hx[g] = R.px; eo.hy[g] = R.py; eo.hz[g] = (float)((double)R.pz + sys.s[sys.doe_index].z);
        eo.opl[g] = R.opl;
    }
    const float N = (float)sys.n_ssr;
    if (MODE == MODE_COHERENT && sys.window == 0) {
        // whole-sensor sum, a warp's 32 draws at a time (warps past n_ssr skip)
        for (int i0 = d0; i0 < d1; i0 += RW_THREADS) {
            if (i0 + (int)(threadIdx.x & ~31u) >= d1) continue;
            const int i = i0 + threadIdx.x;
            const int jb = i < d1 ? sel[i] : -1;
            float dx = 0.f, dy = 0.f, dz = 0.f;
            float x = R.px, y = R.py, zl = R.pz;
            double opl = R.opl;
            float2 a = make_float2(0.f, 0.f);
            bool ok = false;
            if (jb >= 0) {
                const int jvi = jb / M, jui = jb - (jb / M) * M;
                ok = bin_direction(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz);
                const float2 U = spectrum_at<M>(X, phu, phv, jui, jvi, norm);
                a = cscale(cmul(ain, U), 1.f / (N * p[jb]));
                if (ok) ok = trace_to_sensor<true>(sys, x, y, zl, dx, dy, dz, opl, status);
            }
            __syncwarp();
            splat_coherent_warp(sys, J.k0, R.cx, R.cy, ok, x, y, opl, dx, dy, dz, a,
                                field + (long long)J.out * sys.nx * sys.ny);
        }
        return;
    }
    for (int i = d0 + threadIdx.x; i < d1; i += RW_THREADS) {
        const int jb = sel[i];
        float dx = 0.f, dy = 0.f, dz = 0.f;
        float2 a = make_float2(0.f, 0.f);
        bool ok = false;
        if (jb >= 0) {
            const int jvi = jb / M, jui = jb - (jb / M) * M;
            ok = bin_direction<(NS >= 0)>(sys, R, jui - M / 2, jvi - M / 2, dx, dy, dz);
            const float2 U = spectrum_at<M>(X, phu, phv, jui, jvi, norm);
            const float pj = p[jb];
            const float sc = coh ? 1.f / (N * pj) : rsqrtf(N * pj);
            a = cscale(cmul(ain, U), sc);
        }
        if (MODE == MODE_EMIT) {
            const long long s = g * (long long)sys.n_ssr + i;
            eo.dx[s] = ok ? dx : 0.f; eo.dy[s] = ok ? dy : 0.f; eo.dz[s] = ok ? dz : 0.f;
            eo.are[s] = ok ? a.x : 0.f; eo.aim[s] = ok ? a.y : 0.f;
            if (eo.bin) eo.bin[s] = jb;
            continue;
        }
        if (ok) deposit<MODE, NS>(sys, J, R, dx, dy, dz, a, a.x * a.x + a.y * a.y, psf, field,
                                  status);
    }
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_prep_maps(const LaunchCtx& L, const float* phi, const float* phi2,
                             const float* amp, int64_t npix, const float* scales_dev, int nslot,
                             float2* T);
cudaError_t launch_generate_rays(const LaunchCtx& L, const GenJob* jobs, const long long* prefix,
                                 int njob, long long total, double z_start, double n_object,
                                 const RaysOut& out);
// Block culling applies (exhaustive incoherent splat over plane/sphere
// surfaces without RW_DOE_TRACE_ALL); `keep` then needs cull_keep_words(M)
// words per incident ray.
bool forward_culls(const DSys& sys);
// k_cull alone (M <= 64, plane/sphere surfaces behind the DOE).
cudaError_t launch_cull(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                        const long long* prefix, int njob, long long total, const RaysIn& rays,
                        unsigned* keep, unsigned* status);
// The fused forward with the tensor-core patch transform (D = M = 64,
// exhaustive emission, incoherent sensor; culling when `keep` is given).
cudaError_t launch_forward_tc(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                              const long long* prefix, int njob, long long total,
                              const RaysIn& rays, const float2* T, double* psf, unsigned* status,
                              unsigned* vis, unsigned* keep, const SplitBufs* tape);
cudaError_t launch_forward(const LaunchCtx& L, int mode, const DSys& sys, const DJob* jobs,
                           const long long* prefix, int njob, long long total,
                           const RaysIn& rays, const float2* T, double* psf, float2* field,
                           const EmitOut& eo, unsigned* status, unsigned* vis = nullptr,
                           unsigned* keep = nullptr, const SplitBufs* tape = nullptr);
cudaError_t launch_psf_finalize(const LaunchCtx& L, const double* acc, float* psf, long long n);
cudaError_t launch_coherent_finalize(const LaunchCtx& L, const float2* field, float* psf,
                                     long long n);
// field <- 2 g field (dL/dU of I = |U|^2 from dL/dI = g)
cudaError_t launch_coherent_grad(const LaunchCtx& L, float2* field, const float* g, long long n);
