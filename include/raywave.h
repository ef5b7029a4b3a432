/*
 * raywave.h -- C ABI of the GB300 ray-wave DOE library (librw.so).
 *
 * The library evaluates the ray -> wave -> ray step of the differentiable
 * ray-wave model for hybrid refractive-diffractive optics (Cheng, Gao, Shao,
 * Mao, Milster, Fan) and the refractive tracing around it, on one GPU:
 *
 *   A0  collimated ray bundles per (wavelength, field) job
 *   A1  sequential refraction (Snell; sphere in closed form; even asphere by
 *       Newton's method) up to the DOE
 *   A2  DOE intersection and tangent frame (u, v, n)   [section "Ray-Wave
 *       Simulator Formalism", second paragraph]
 *   A3  D x D patch of the transmission U = A exp(i phi) centred on the hit
 *   A4  angular spectrum U~(k_u, k_v) of the patch (Fourier transform), on
 *       the grid of M = P D points when the patch is zero-padded by P
 *       (section "Benchmark and Inverse Design Demonstrations")
 *   A5  secondary rays along the propagating wavevectors, weight U~ / p (Eq. 1);
 *       sampled mode draws wavevectors by Gumbel-max (same section, third
 *       paragraph)
 *   A6  refraction of the secondary rays through the remaining surfaces
 *   A7  sensor: incoherent bilinear splat of |a|^2, or the coherent sum of
 *       plane wavelets of Eq. 2
 *   A8  normalised least-squares loss of Eq. 3
 *   A9  adjoint of A1..A7: gradients w.r.t. DOE phase/amplitude pixels and
 *       surface parameters (section "Benchmark and Inverse Design
 *       Demonstrations", end-to-end optimisation)
 *
 * Conventions
 *   - Units: millimetres; wavelengths are vacuum wavelengths in mm.  +z is
 *     the optical axis, light travels towards +z.
 *   - Small descriptors (rw_system, rw_surface, rw_job arrays) are HOST
 *     memory read during the call.  Every array inside rw_rays, rw_emitted,
 *     the DOE maps, PSFs and gradients is DEVICE memory owned by the caller;
 *     the library never frees or retains it after the call returns.
 *   - Every call is enqueued on the context's CUDA stream and returns before
 *     the GPU work finishes; synchronise that stream before reading outputs.
 *   - Every call returns rw_status.  On a non-OK status no GPU work of that
 *     call was enqueued (validation runs on the host first) unless the status
 *     is RW_ECUDA; outputs are then unspecified and rw_last_error() holds a
 *     one-line message.  Device-side conditions (Newton non-convergence,
 *     capacity overflow) are counted in a status word that
 *     rw_device_status() reads.
 *   - The library keeps per-context scratch (the complex transmission map per
 *     wavelength, job tables, reduction buffers) and grows it on demand.
 */
#ifndef RAYWAVE_H
#define RAYWAVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rw_ctx rw_ctx;

typedef enum {
    RW_OK = 0,
    RW_EINVAL = 1,     /* bad argument (null pointer, size, unsupported mode) */
    RW_ENOMEM = 2,     /* scratch allocation failed */
    RW_ECUDA = 3,      /* a CUDA runtime call failed */
    RW_ECAPACITY = 4,  /* output capacity too small */
    RW_ETIMEOUT = 5,   /* a bounded device wait gave up */
    RW_ENOTCONV = 6    /* Newton iteration did not converge for some rays */
} rw_status;

/* surface kinds (RW_GAUSS only as the substrate of a conformal DOE) */
enum { RW_PLANE = 0, RW_SPHERE = 1, RW_ASPHERE = 2, RW_GAUSS = 3 };
/* DOE patch gather: nearest pixel window (planar) / bilinear (conformal) */
enum { RW_GATHER_NEAREST = 0, RW_GATHER_BILINEAR = 1 };
/* secondary-ray emission: every propagating bin; n_ssr Gumbel-max draws from
 * p ~ |U~| (coherent sensor) or |U~|^2 (incoherent); or n_ssr draws from the
 * uniform density over the propagating bins (the paper's p_uni, for
 * comparison).  Sampled weights: a = a_in U~ / (N p) (coherent) or
 * a_in U~ / sqrt(N p) (incoherent). */
enum { RW_EMIT_EXHAUSTIVE = 0, RW_EMIT_SAMPLED = 1, RW_EMIT_SAMPLED_UNIFORM = 2 };
/* phase at wavelength lambda: phi * lambda0 / lambda (HEIGHT) or phi (FIXED) */
enum { RW_PHASE_HEIGHT = 0, RW_PHASE_FIXED = 1 };
/* patch transform implementation */
enum { RW_DFT_FFT32 = 0, RW_DFT_TC = 1 };
/* rw_doe.flags:
 *   RW_DOE_TRACE_ALL: trace every secondary ray (no block culling; the
 *     results are the same, only slower -- for verification);
 *   RW_DOE_REFLECTIVE: the DOE reflects (the reflective conformal DOE of the
 *     paper's inverse-design section): secondary rays leave with the normal
 *     component of their wavevector reversed, d = (kappa_u u + kappa_v v -
 *     kn n) / (k0 n_in), back into the incident medium (index n_in; the DOE
 *     surface's n_after is unused).  The DOE must be the last surface and the
 *     sensor must lie in front of it (sensor z < DOE vertex z); incident rays
 *     cross the sensor plane without interacting. */
enum { RW_DOE_TRACE_ALL = 1, RW_DOE_REFLECTIVE = 2 };

#define RW_MAX_SURFACES 16

/* One rotationally symmetric surface in vertex form:
 *   z - z_vertex = c s / (1 + sqrt(1 - (1 + k) c^2 s)) + A4 s^2 + A6 s^3 + A8 s^4 + A10 s^5,
 *   s = x^2 + y^2.
 * PLANE ignores c, k, A; SPHERE ignores k, A.  RW_GAUSS (DOE substrate only)
 * is the Gaussian bump z - z_vertex = c exp(-s / (2 k^2)): height c (mm,
 * either sign), width k > 0 (mm); its apex radius of curvature is k^2 / |c|.
 * n_after is the index of the medium behind the surface.  r_ap > 0 drops
 * rays hitting at radius > r_ap. */
typedef struct {
    int32_t kind;
    int32_t reserved;
    double z;
    double c;
    double k;
    double A4, A6, A8, A10;
    double n_after;
    double r_ap;
    double sellmeier[6];   /* B1, B2, B3, C1, C2, C3 (C in um^2); all zero: the medium
                            * behind has the constant index n_after.  Otherwise its
                            * index at a job's vacuum wavelength L (um) is
                            * sqrt(1 + sum_i B_i L^2 / (L^2 - C_i)) and n_after is
                            * unused: rw_forward and rw_backward run one launch per
                            * distinct wavelength (not rw_doe_emit, rw_patch_spectra
                            * or the visibility mask: RW_EINVAL), and dsurf's n_after
                            * slot is dL/dn for a shift common to all wavelengths. */
} rw_surface;

/* The DOE: its transmission map and the ray-wave parameters.  The geometry
 * is surfaces[doe_index] of the system (PLANE = planar DOE, SPHERE or GAUSS =
 * conformal DOE; a conformal hit is refined in double precision by Newton's
 * method, RW_ENOTCONV if it fails).  Pixel (r, c) is centred at
 * x = (c - W/2 + 1/2) pitch, y = (r - H/2 + 1/2) pitch. */
typedef struct {
    int32_t H, W;
    double pitch;          /* mm */
    double lambda0;        /* design wavelength of phi (HEIGHT model), mm */
    const float* phi;      /* device, [H][W] radians */
    const float* amp;      /* device, [H][W], or NULL for amplitude 1 */
    int32_t D;             /* patch side in pixels: 16, 32, 64 or 96 */
    int32_t gather;        /* RW_GATHER_* */
    int32_t emit;          /* RW_EMIT_* */
    int32_t n_ssr;         /* draws per incident ray in sampled mode */
    int32_t phase_model;   /* RW_PHASE_* */
    int32_t dft;           /* RW_DFT_*: patch transform (see rw_forward, rw_patch_spectra) */
    uint64_t seed;         /* Philox key for sampled mode */
    uint64_t rng_offset;   /* Philox counter word 3 for sampled mode: draw i of the
                            * incident ray stored at index r of the ray arrays
                            * perturbs bin j with word j & 3 of Philox4x32-10 at
                            * counter (j >> 2, i, r, rng_offset), so a ray's draws do
                            * not depend on how the job table groups the rays */
    int32_t pad;           /* zero-padding factor P (0 or 1: none): the D x D patch is
                            * transformed on M = P D points, M in {16, 32, 64, 96, 128};
                            * bins are k_j = 2 pi j / (M pitch), and U~ is scaled by
                            * 1/M^2 (coherent sensor) or 1/(D M) (incoherent) */
    int32_t flags;         /* RW_DOE_* bits, 0 by default.  Without RW_DOE_TRACE_ALL
                            * the exhaustive incoherent forward over plane/sphere
                            * surfaces skips blocks of bins whose affine-arithmetic
                            * enclosure of the sensor hit lies two pixels or more
                            * outside the sensor window (they cannot deposit) */
    const float* phi2;     /* device, [H][W] radians, or NULL: with a second phase
                            * profile the field is U = A (exp(i phi) + exp(i phi2))
                            * (the complex-amplitude DOE of the paper's conformal
                            * beam-splitting demonstration); both profiles follow
                            * phase_model */
} rw_doe;

/* Sensor plane z = const.  Pixel (i, j) of job J is centred at
 * x = sensor_cx_J + (i - nx/2 + 1/2) pitch, y = sensor_cy_J + (j - ny/2 + 1/2) pitch. */
typedef struct {
    double z;
    int32_t nx, ny;
    double pitch;
    int32_t coherent;      /* 0: bilinear |a|^2 splat; 1: Eq. 2 wavelet sum */
    int32_t window;        /* coherent: +-window pixels around each hit (0 = all) */
} rw_sensor;

typedef struct {
    const rw_surface* surfaces;   /* host, nsurf entries, sorted by z */
    int32_t nsurf;                /* 1 .. RW_MAX_SURFACES */
    int32_t doe_index;            /* which surface carries the DOE */
    double n_object;              /* index of the medium before surface 0 */
    rw_doe doe;
    rw_sensor sensor;
} rw_system;

/* One (wavelength, field) job: its rays are rays[ray_offset .. ray_offset+ray_count).
 * grid_n, spacing, x0, y0, theta_x, theta_y and z_start describe the
 * collimated bundle rw_generate_rays writes; the other calls only use
 * lambda, ray_offset, ray_count and the sensor window centre. */
typedef struct {
    double lambda;
    double theta_x, theta_y;
    int64_t ray_offset;
    int64_t ray_count;
    double sensor_cx, sensor_cy;
    int64_t grid_n;
    double spacing, x0, y0;
} rw_job;

/* Incident rays, structure of arrays on the device, n entries each. */
typedef struct {
    int64_t n;
    float* ox; float* oy; float* oz;
    float* dx; float* dy; float* dz;
    float* a_re; float* a_im;
    double* opl;
} rw_rays;

/* Secondary rays written by rw_doe_emit.  Slot s = i * S + b for incident
 * ray i and bin/draw b, S = M*M with M = pad * D (exhaustive;
 * b = (j_v + M/2) * M + (j_u + M/2)) or n_ssr (sampled).  Dropped rays (evanescent, missed DOE) have a = 0 and
 * d = 0.  hit/opl are per incident ray. */
typedef struct {
    int64_t capacity;                /* slots available: >= n_incident * S */
    float* dx; float* dy; float* dz; /* [capacity] */
    float* a_re; float* a_im;        /* [capacity] */
    int32_t* bin;                    /* [capacity] chosen bin (sampled), may be NULL */
    float* hx; float* hy; float* hz; /* [n_incident] DOE hit point */
    double* opl;                     /* [n_incident] optical path at the hit */
} rw_emitted;

/* ---- context ---------------------------------------------------------- */

/* Create a context on CUDA device `device`, enqueuing on `cuda_stream`
 * (a cudaStream_t, NULL = legacy default stream).  Errors: RW_EINVAL, RW_ECUDA. */
rw_status rw_create(rw_ctx** out, int device, void* cuda_stream);
rw_status rw_destroy(rw_ctx* ctx);
rw_status rw_set_stream(rw_ctx* ctx, void* cuda_stream);
/* Last error message of this context ("" if none); valid until the next call. */
const char* rw_last_error(const rw_ctx* ctx);
/* Synchronise the stream and return the device status word accumulated
 * since the last call of this function (bit 0: Newton non-convergence,
 * bit 1: capacity overflow, bit 2: bounded wait timeout), then clear it. */
rw_status rw_device_status(rw_ctx* ctx, uint32_t* status_out);
const char* rw_version(void);
/* Number of kernels this context has launched so far (for benchmarks). */
int64_t rw_launch_count(const rw_ctx* ctx);
/* Per-launch timing (library extension for benchmarks; the paper has no
 * counterpart).  rw_profile(ctx, 1) synchronises the stream, clears the
 * totals and from then on records a CUDA event on the context's stream just
 * before and just after every kernel launch (not while the stream is being
 * captured into a graph); rw_profile(ctx, 0) stops recording.
 * rw_profile_read synchronises the stream, folds the recorded launches into
 * per-kernel totals (since the last rw_profile call) and returns how many
 * kernels there are; rw_profile_entry(i) gives kernel i's name (owned by the
 * context, valid until the next rw_profile / rw_profile_read), its summed
 * launch durations in ms and its launch count.  Errors: RW_EINVAL (null
 * argument, index out of range), RW_ECUDA. */
rw_status rw_profile(rw_ctx* ctx, int32_t enable);
rw_status rw_profile_read(rw_ctx* ctx, int32_t* n_kernels);
rw_status rw_profile_entry(rw_ctx* ctx, int32_t i, const char** kernel, double* total_ms,
                           int64_t* launches);
/* Block-culling statistics of the most recent forward call on this context
 * that culled (library extension; the paper has no counterpart): the number
 * of 8 x 8 bin blocks (n_rays * (M/8)^2) and how many of them were kept and
 * traced (64 bins each).  Synchronises the stream; (0, 0) if no forward has
 * culled yet.  Errors: RW_EINVAL, RW_ECUDA. */
rw_status rw_cull_stats(rw_ctx* ctx, int64_t* blocks, int64_t* kept);

/* ---- A10: launch tuning ------------------------------------------------- */

/* Kernels whose persistent grid (CTAs of the launch) can be tuned; indices of
 * the grids arrays below. */
enum { RW_K_FORWARD = 0, RW_K_CULL, RW_K_BS_SPECTRA, RW_K_BS_TRACE, RW_K_BS_SCATTER,
       RW_K_BACKWARD, RW_K_SPECTRA, RW_NK };

/* Tune the persistent grid of every kernel on this workload (batching and
 * scheduling of the method's per-ray work; the paper names no GPU and has no
 * counterpart): runs one warm-up step, then one step -- rw_forward_vis (or
 * rw_forward when vis is NULL) and, when dl_dpsf is not NULL, the adjoint
 * with the same mask -- for each candidate grid (the occupancy default and
 * 1, 2, 3, 4, 6, 8 CTAs per SM), times every launch with CUDA events and
 * keeps, per kernel, the fastest.  The context then launches with those
 * grids; grids_out receives them (RW_NK entries, 0 = occupancy default).
 * psf, dphi, dsurf are used as scratch: their contents afterwards are
 * unspecified.  Synchronises the stream; not during graph capture.
 * Errors: as rw_forward / rw_backward_vis, RW_EINVAL. */
rw_status rw_autotune(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs, int32_t njob,
                      const rw_rays* rays, float* psf, const float* dl_dpsf, uint32_t* vis,
                      int64_t vis_words, float* dphi, double* dsurf, int64_t* grids_out);
/* Set the per-kernel grids directly (RW_NK entries, <= 0 = occupancy default),
 * e.g. to reuse an earlier rw_autotune result.  Errors: RW_EINVAL. */
rw_status rw_set_grids(rw_ctx* ctx, const int64_t* grids);

/* Measurement aid (no paper counterpart): enqueue win * win * nwin float
 * atomic adds (results unused) onto map (device float [H][W], modified),
 * in nwin windows of win x win pixels at pseudo-random offsets, a warp on
 * adjacent pixels of a row -- the pattern of the adjoint's map scatter.
 * Timing it gives the reduction ceiling the scatter's roofline is read
 * against.  Errors: RW_EINVAL (NULL map, win outside [1, min(H, W)],
 * nwin < 0). */
rw_status rw_probe_red(rw_ctx* ctx, float* map, int32_t H, int32_t W, int32_t win,
                       int64_t nwin);

/* ---- A0: ray generation ------------------------------------------------ */

/* Fill rays[ray_offset ..) of every job with its collimated grid launched
 * from z = z_start: direction normalise(tan theta_x, tan theta_y, 1), ray
 * (ix, iy) -> index iy*grid_n + ix at x0 + (ix - (grid_n-1)/2) spacing,
 * y0 + (iy - (grid_n-1)/2) spacing; a = 1; opl = n_object (d . o).
 * Positions are computed in double and rounded once to float.
 * Errors: RW_EINVAL (ray_count != grid_n^2, out of range, null pointer). */
rw_status rw_generate_rays(rw_ctx* ctx, double z_start, double n_object,
                           const rw_job* jobs, int32_t njob, rw_rays* rays);

/* ---- A1..A5: emit secondary rays at the DOE ---------------------------- */

/* Trace every job's rays to the DOE and write its secondary rays.
 * Errors: RW_EINVAL, RW_ECAPACITY (out->capacity < n_rays * S). */
rw_status rw_doe_emit(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs,
                      int32_t njob, const rw_rays* rays, rw_emitted* out);

/* ---- A1..A7: forward to the sensor ------------------------------------- */

/* psf: device float [njob][ny][nx], overwritten (zeroed then accumulated).
 * Incoherent: sum of bilinear |a|^2 deposits; coherent: |Eq. 2|^2.
 * doe.dft = RW_DFT_TC forms each patch spectrum by the tensor-core
 * contraction of rw_patch_spectra inside the fused kernel (D = 64 without
 * padding, exhaustive emission, incoherent sensor; otherwise RW_EINVAL);
 * RW_DFT_FFT32 uses the FP32 shared-memory FFT. */
rw_status rw_forward(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs,
                     int32_t njob, const rw_rays* rays, float* psf);

/* rw_forward that also records which secondary rays reached the sensor:
 * bit (f & 31) of vis[i * M*M/32 + f/32] is set when bin f of incident ray i
 * (job order) hit the sensor plane with a bilinear tap on the sensor.  One
 * bit per secondary ray (M = 64: 512 bytes per incident ray).  Needs the
 * incoherent sensor and exhaustive emission.
 * Errors: as rw_forward, RW_ECAPACITY (vis_words < n_rays * M*M / 32). */
rw_status rw_forward_vis(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs, int32_t njob,
                         const rw_rays* rays, float* psf, uint32_t* vis, int64_t vis_words);

/* ---- A3..A4: patch spectra only ----------------------------------------- */

/* Trace every job's rays to the DOE and write the angular spectrum of each
 * patch, U~[j_v][j_u] referred to the hit point with the normalisation of
 * doe.pad (1/D^2 without padding; section "Ray-Wave Simulator Formalism",
 * second paragraph), as complex float pairs:
 * spectra[(i * M + (j_v + M/2)) * M + (j_u + M/2)], M = pad * D, for incident
 * ray i in job order; rays that miss the DOE give zeros.  doe.dft selects the
 * implementation: RW_DFT_FFT32 (FP32 shared-memory FFT, any supported M) or
 * RW_DFT_TC (tensor-core contraction F X F^T with a BF16x3 split and FP32
 * accumulation, D = 64 without padding only).  capacity counts complex entries.
 * Errors: RW_EINVAL, RW_ECAPACITY (capacity < n_rays * M * M). */
rw_status rw_patch_spectra(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs, int32_t njob,
                           const rw_rays* rays, float* spectra, int64_t capacity);

/* ---- A8: Eq. 3 loss ---------------------------------------------------- */

/* L = || alpha I - T ||^2 with alpha = <I,T>/<I,I> over all n entries.
 * loss_out: device double[3] = {L, alpha, <I,I>}; dl_dpsf (device float[n],
 * may be NULL) receives 2 alpha (alpha I - T). */
rw_status rw_loss_eq3(rw_ctx* ctx, const float* psf, const float* target, int64_t n,
                      double* loss_out, float* dl_dpsf);

/* ---- A9: adjoint -------------------------------------------------------- */

/* Given dL/dpsf (device float [njob][ny][nx]), ACCUMULATE (+=) into
 *   dphi  device float [H][W]   (may be NULL); with doe.phi2 set,
 *         [2][H][W]: dL/dphi, then dL/dphi2
 *   damp  device float [H][W]   (may be NULL; needs doe.amp)
 *   dsurf device double [nsurf][8] = d/d(z, c, k, A4, A6, A8, A10, n_after)
 *         (may be NULL).
 * Patches and spectra are recomputed, not stored, with the FP32 FFT whatever
 * doe.dft selects (a mask or tape from a RW_DFT_TC forward is accepted).
 * Supported: incoherent
 * and coherent sensor, exhaustive or sampled emission (straight-through
 * Gumbel-softmax with temperature 1), M = pad * D <= 96 (M = 128 only
 * through rw_backward_vis with exhaustive emission and the incoherent
 * sensor).  Coherent sensor (Eq. 2, psf = |U|^2): the call first recomputes
 * the complex field U of the same inputs (one forward pass; the phase is not
 * in psf), forms dL/dU = 2 (dL/dpsf) U and reverses every secondary ray's
 * window sum, optical path included; surface gradients then carry the
 * optical-path terms of every segment.  With a conformal DOE (sphere or
 * Gaussian bump) the hit point, the tangent frame (u, v, n) and the
 * tangent-plane patch samples depend on the incident ray and on the
 * substrate: their reverse gives the substrate's z and c (sphere) or z,
 * height (c slot) and width (k slot) of the bump, and carries dL/d(ray)
 * on to the surfaces before the DOE. */
rw_status rw_backward(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs,
                      int32_t njob, const rw_rays* rays, const float* dl_dpsf,
                      float* dphi, float* damp, double* dsurf);

/* ---- allocation-free ray generation ------------------------------------ */

/* Same result as rw_generate_rays, for callers that cannot call cudaMalloc:
 * a plugin inside a host application that owns all device memory through
 * its own allocator, or a real-time loop that cannot afford the implicit
 * device synchronisation of cudaMalloc.  (The paper has no counterpart;
 * this is a deployment interface.)
 *
 * Needs no context and allocates nothing: the job table is built in a
 * static host buffer (under a mutex; no large stack frame) and copied into a
 * file-scope device array of the library sized for at most 1024 jobs (about
 * 64 KiB, held by every GPU that loads the library until the process
 * exits).  njob > 1024 returns RW_ECAPACITY before anything is written; bad
 * arguments return RW_EINVAL; a failing CUDA call returns RW_ECUDA.  Work is
 * enqueued on `cuda_stream` (a cudaStream_t, NULL = legacy default stream)
 * of the CURRENT device; the array's device address is looked up on every
 * call with that device current.  A call while `cuda_stream` is being
 * captured into a graph returns RW_EINVAL: the upload reads a host buffer
 * that later calls overwrite.  Every call shares the device array and
 * rewrites the part it uses, so nothing needs clearing, but calls that
 * overlap on the GPU (different streams, no ordering) race on it. */
rw_status rw_generate_rays_static(double z_start, double n_object, const rw_job* jobs,
                                  int32_t njob, rw_rays* rays, void* cuda_stream);

/* rw_backward with the visibility mask written by rw_forward_vis for the
 * SAME inputs: a secondary ray that deposited nothing on the sensor has zero
 * gradient, so only the visible ones are re-traced and reversed (exact).
 * Exhaustive emission and the incoherent sensor; patch sizes above 64
 * ignore the mask. */
rw_status rw_backward_vis(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs, int32_t njob,
                          const rw_rays* rays, const float* dl_dpsf, const uint32_t* vis,
                          int64_t vis_words, float* dphi, float* damp, double* dsurf);

#ifdef __cplusplus
}
#endif
#endif /* RAYWAVE_H */
