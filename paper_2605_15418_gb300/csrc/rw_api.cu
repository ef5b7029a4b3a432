// Host side of the C ABI declared in include/raywave.h: argument checks,
// packing of the host descriptors into device-side structs, per-context
// scratch, and kernel launches on the context's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "rw_kernels.cuh"

cudaError_t launch_loss_eq3(const LaunchCtx& L, const float* I, const float* T, long long n,
                            double* acc, double* out, float* g);
cudaError_t launch_probe_red(const LaunchCtx& L, float* map, int H, int W, int win,
                             long long nwin);
cudaError_t launch_backward(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                            const long long* prefix, int njob, long long total,
                            const RaysIn& rays, const float2* T, const float* amp,
                            const float* dl_dpsf, const float2* gfield, float* coh_rsum,
                            double* coh_jsum, float* dphi, float* damp, double* dsurf,
                            const unsigned* vis, unsigned* status, int* launches);
size_t backward_smem_needed(const DSys& sys);
cudaError_t launch_bs_count(const LaunchCtx& L, const unsigned* vis, long long nwords,
                            unsigned long long* total);
cudaError_t launch_backward_split(const LaunchCtx& L, const DSys& sys, const DJob* jobs,
                                  const long long* prefix, int njob, long long total,
                                  const RaysIn& rays, const float2* T, const float* amp,
                                  const float* gpsf, const unsigned* vis, const SplitBufs& B,
                                  long long nitems, int have_list, float* dphi, float* damp,
                                  double* dsurf, unsigned* status);
cudaError_t launch_spectra(const LaunchCtx& L, const DSys& sys, int tc, const DJob* jobs,
                           const long long* prefix, int njob, long long total, const RaysIn& rays,
                           const float2* T, float2* out, unsigned* status);

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t need) {
        if (need <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, need);
        if (e == cudaSuccess) bytes = need;
        return e;
    }
    void release() { if (p) cudaFree(p); p = nullptr; bytes = 0; }
};

}  // namespace

struct rw_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    std::string err;
    DevBuf tmaps;       // complex transmission per wavelength slot
    DevBuf tables;      // job tables, prefix sums, map scales
    DevBuf field;       // coherent field accumulator
    DevBuf coh_rsum;    // coherent adjoint: per-ray emission gradient sums (7 floats)
    DevBuf coh_jsum;    // coherent adjoint: per-job sum of dL/dOPL and ray count
    DevBuf acc;         // double PSF accumulator
    DevBuf split_rays;  // split adjoint: per-ray state, offsets, sums
    DevBuf split_items; // split adjoint: work list of visible secondary rays
    DevBuf keep;        // block culling: kept 8 x 8 bin blocks per incident ray
    long long keep_words = 0, keep_blocks = 0;   // of the last culled forward
    // tape of the last rw_forward_vis: its visible secondary rays already in
    // split_rays / split_items, valid for the adjoint with the same mask
    bool tape_valid = false;
    const void* tape_vis = nullptr;
    long long tape_total = 0, tape_cap = 0, tape_hint = 0;
    int tape_M = 0;
    unsigned long long* count_host = nullptr;   // pinned
    DevBuf misc;        // status word + loss sums
    void* staging = nullptr;       // pinned host copy source of `tables`
    size_t staging_bytes = 0;
    cudaEvent_t staging_done = nullptr;
    // tables uploaded while the stream is being captured into a CUDA graph:
    // bump-allocated, never reused, so every captured copy node keeps its data
    void* cap_host = nullptr;
    DevBuf cap_dev;
    size_t cap_used = 0;
    int64_t launches = 0;
    long long grid_override = 0;
    long long grid[RW_NK] = {0, 0, 0, 0, 0, 0, 0};    // tuned persistent grids (rw_autotune)
    // per-launch timing (rw_profile): events around every kernel launch
    bool prof_on = false;
    ProfHook prof_hook{};
    std::vector<cudaEvent_t> prof_pool;       // created on demand, reused
    std::vector<const char*> prof_names;      // name per recorded event (null: end)
    size_t prof_used = 0;
    std::vector<std::string> prof_kernels;    // results of the last rw_profile_read
    std::vector<double> prof_ms;
    std::vector<int64_t> prof_count;
};

static rw_status fail(rw_ctx* c, rw_status s, const std::string& m) {
    if (c) c->err = m;
    return s;
}
static rw_status cuda_fail(rw_ctx* c, cudaError_t e, const char* where) {
    return fail(c, RW_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define RW_CUDA(call, where)                                  \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

static unsigned* status_word(rw_ctx* ctx) { return reinterpret_cast<unsigned*>(ctx->misc.p); }
static double* loss_acc(rw_ctx* ctx) {
    return reinterpret_cast<double*>(reinterpret_cast<char*>(ctx->misc.p) + 64);
}

#define RW_CAPTURE_ARENA (4u << 20)

static bool capturing(rw_ctx* ctx) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess) return false;
    return cs == cudaStreamCaptureStatusActive;
}

// Grow a scratch buffer; refused while the stream is being captured (run the
// same call once eagerly first so the scratch is already large enough).
static rw_status ensure_buf(rw_ctx* ctx, DevBuf& b, size_t need, const char* what) {
    if (need <= b.bytes) return RW_OK;
    if (capturing(ctx))
        return fail(ctx, RW_EINVAL, std::string(what) +
                                        ": scratch must grow during graph capture; run the call "
                                        "once outside the capture first");
    if (b.ensure(need) != cudaSuccess) return fail(ctx, RW_ENOMEM, what);
    return RW_OK;
}

// Copy small host tables to the device through the pinned staging buffer.
// The previous copy out of the staging buffer is waited for first.  During
// stream capture the tables go through the capture arenas instead.
static rw_status upload(rw_ctx* ctx, const std::vector<std::pair<const void*, size_t>>& parts,
                        std::vector<void*>& dev_ptrs) {
    size_t total = 0;
    std::vector<size_t> offs;
    for (auto& p : parts) { offs.push_back(total); total += align16(p.second); }
    if (total == 0) total = 16;
    RW_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (capturing(ctx)) {
        if (!ctx->cap_host || ctx->cap_used + total > RW_CAPTURE_ARENA)
            return fail(ctx, RW_ENOMEM, "graph-capture table arena exhausted (4 MiB per context)");
        char* h = (char*)ctx->cap_host + ctx->cap_used;
        char* dv = (char*)ctx->cap_dev.p + ctx->cap_used;
        ctx->cap_used += total;
        for (size_t i = 0; i < parts.size(); ++i)
            if (parts[i].second) std::memcpy(h + offs[i], parts[i].first, parts[i].second);
        RW_CUDA(cudaMemcpyAsync(dv, h, total, cudaMemcpyHostToDevice, ctx->stream),
                "captured table upload");
        dev_ptrs.clear();
        for (size_t i = 0; i < parts.size(); ++i) dev_ptrs.push_back(dv + offs[i]);
        return RW_OK;
    }
    if (ctx->staging_done) RW_CUDA(cudaEventSynchronize(ctx->staging_done), "staging wait");
    if (total > ctx->staging_bytes) {
        if (ctx->staging) cudaFreeHost(ctx->staging);
        ctx->staging = nullptr;
        ctx->staging_bytes = 0;
        RW_CUDA(cudaMallocHost(&ctx->staging, total), "cudaMallocHost");
        ctx->staging_bytes = total;
    }
    {
        rw_status st = ensure_buf(ctx, ctx->tables, total, "table scratch");
        if (st != RW_OK) return st;
    }
    for (size_t i = 0; i < parts.size(); ++i)
        if (parts[i].second) std::memcpy((char*)ctx->staging + offs[i], parts[i].first, parts[i].second);
    RW_CUDA(cudaMemcpyAsync(ctx->tables.p, ctx->staging, total, cudaMemcpyHostToDevice, ctx->stream),
            "table upload");
    RW_CUDA(cudaEventRecord(ctx->staging_done, ctx->stream), "event record");
    dev_ptrs.clear();
    for (size_t i = 0; i < parts.size(); ++i) dev_ptrs.push_back((char*)ctx->tables.p + offs[i]);
    return RW_OK;
}

static bool capturing(rw_ctx* ctx);

static void prof_mark(void* user, const char* kernel) {
    rw_ctx* ctx = static_cast<rw_ctx*>(user);
    if (ctx->prof_used == ctx->prof_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        ctx->prof_pool.push_back(e);
        ctx->prof_names.push_back(nullptr);
    }
    if (cudaEventRecord(ctx->prof_pool[ctx->prof_used], ctx->stream) != cudaSuccess) return;
    ctx->prof_names[ctx->prof_used++] = kernel;
}

static LaunchCtx lctx(rw_ctx* ctx) {
    LaunchCtx L;
    L.stream = ctx->stream;
    L.num_sms = ctx->num_sms;
    L.grid_override = ctx->grid_override;
    for (int k = 0; k < RW_NK; ++k) L.grid[k] = ctx->grid[k];
    L.prof = nullptr;
    if (ctx->prof_on && !capturing(ctx)) {
        ctx->prof_hook.user = ctx;
        ctx->prof_hook.mark = prof_mark;
        L.prof = &ctx->prof_hook;
    }
    return L;
}

// ---------------------------------------------------------------- validation + packing
struct Packed {
    DSys sys;
    std::vector<DJob> jobs;
    std::vector<long long> prefix;
    std::vector<float> scales;
    long long total = 0;
};

static bool supported_D(int D) { return D == 16 || D == 32 || D == 64 || D == 96; }
// transform sizes with a compiled FFT plan (M = pad * D)
static bool supported_M(int M) { return M == 16 || M == 32 || M == 64 || M == 96 || M == 128; }

// Split-adjoint buffers for n incident rays and cap work items (the forward's
// tape uses the same layout).
static rw_status split_buffers(rw_ctx* ctx, long long n, long long cap, int nrs, SplitBufs& B) {
    const size_t per_ray = sizeof(RayAtDoe) + sizeof(long long) + sizeof(int) + nrs * sizeof(float);
    rw_status st = ensure_buf(ctx, ctx->split_rays, n * per_ray + 256, "split adjoint rays");
    if (st != RW_OK) return st;
    if (cap < 1) cap = 1;
    const size_t per_item = 2 * sizeof(int) + 2 * sizeof(float2);
    st = ensure_buf(ctx, ctx->split_items, (size_t)cap * per_item + 256, "split adjoint list");
    if (st != RW_OK) return st;
    char* rp = (char*)ctx->split_rays.p;
    B.rinfo = (RayAtDoe*)rp;                    rp += align16(n * sizeof(RayAtDoe));
    B.voff = (long long*)rp;                    rp += align16(n * sizeof(long long));
    B.vcnt = (int*)rp;                          rp += align16(n * sizeof(int));
    B.rsum = (float*)rp;
    char* ip = (char*)ctx->split_items.p;
    B.igU = (float2*)ip;                        ip += (size_t)cap * sizeof(float2);
    B.iU = (float2*)ip;                         ip += (size_t)cap * sizeof(float2);
    B.iray = (int*)ip;                          ip += (size_t)cap * sizeof(int);
    B.ibin = (int*)ip;
    B.cap = cap;
    return RW_OK;
}
// tape counter, forward-with-mask epoch, epoch of the tape: three adjacent words
static unsigned long long* tape_counter(rw_ctx* ctx) {
    return reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(ctx->misc.p) + 192);
}

// ---------------------------------------------------------------- dispersion
// A surface with Sellmeier coefficients makes the medium behind it
// dispersive.  Such systems run one launch per distinct wavelength, each with
// that wavelength's indices; the job table of a launch carries every job's
// image index and ray-id offset, so the results equal one launch over all jobs.
static bool is_dispersive(const rw_system* sys) {
    if (!sys || !sys->surfaces || sys->nsurf < 1 || sys->nsurf > RW_MAX_SURFACES) return false;
    for (int i = 0; i < sys->nsurf; ++i)
        for (int k = 0; k < 6; ++k)
            if (sys->surfaces[i].sellmeier[k] != 0.0) return true;
    return false;
}

// n^2 = 1 + sum_i B_i L^2 / (L^2 - C_i), L the vacuum wavelength in micrometres
static double sellmeier_index(const double* c, double lambda_mm) {
    const double L2 = (lambda_mm * 1e3) * (lambda_mm * 1e3);
    double n2 = 1.0;
    for (int i = 0; i < 3; ++i) n2 += c[i] * L2 / (L2 - c[3 + i]);
    return n2 > 0.0 ? std::sqrt(n2) : std::nan("");
}

struct WaveGroups {
    std::vector<double> lambda;
    std::vector<std::vector<rw_job>> jobs;
    std::vector<std::vector<int>> out;        // job index in the caller's table
};

static rw_status group_by_wavelength(rw_ctx* ctx, const rw_job* jobs, int njob, WaveGroups& G) {
    if (njob < 1) return fail(ctx, RW_EINVAL, "njob must be >= 1");
    if (!jobs) return fail(ctx, RW_EINVAL, "jobs is NULL");
    std::map<double, int> index;
    for (int i = 0; i < njob; ++i) {
        auto it = index.find(jobs[i].lambda);
        int g;
        if (it == index.end()) {
            g = (int)G.lambda.size();
            index[jobs[i].lambda] = g;
            G.lambda.push_back(jobs[i].lambda);
            G.jobs.emplace_back();
            G.out.emplace_back();
        } else {
            g = it->second;
        }
        G.jobs[g].push_back(jobs[i]);
        G.out[g].push_back(i);
    }
    return RW_OK;
}

// The system at one wavelength: every Sellmeier medium gets its index there.
static rw_status system_at(rw_ctx* ctx, const rw_system* sys, double lambda, rw_system& out,
                           std::vector<rw_surface>& surf) {
    surf.assign(sys->surfaces, sys->surfaces + sys->nsurf);
    for (auto& s : surf) {
        bool disp = false;
        for (int k = 0; k < 6; ++k) disp = disp || s.sellmeier[k] != 0.0;
        if (!disp) continue;
        s.n_after = sellmeier_index(s.sellmeier, lambda);
        if (!(s.n_after > 0.0) || !std::isfinite(s.n_after))
            return fail(ctx, RW_EINVAL, "Sellmeier index not real and positive at a job wavelength");
    }
    out = *sys;
    out.surfaces = surf.data();
    return RW_OK;
}

static rw_status pack_system(rw_ctx* ctx, const rw_system* sys, Packed& P) {
    if (!sys) return fail(ctx, RW_EINVAL, "sys is NULL");
    if (sys->nsurf < 1 || sys->nsurf > RW_MAX_SURFACES)
        return fail(ctx, RW_EINVAL, "nsurf must be in 1..16");
    if (!sys->surfaces) return fail(ctx, RW_EINVAL, "surfaces is NULL");
    if (sys->doe_index < 0 || sys->doe_index >= sys->nsurf)
        return fail(ctx, RW_EINVAL, "doe_index out of range");
    if (!(sys->n_object > 0)) return fail(ctx, RW_EINVAL, "n_object must be > 0");
    const rw_doe& doe = sys->doe;
    if (!doe.phi) return fail(ctx, RW_EINVAL, "doe.phi is NULL");
    if (doe.H < 1 || doe.W < 1) return fail(ctx, RW_EINVAL, "doe map size must be positive");
    if (!(doe.pitch > 0)) return fail(ctx, RW_EINVAL, "doe.pitch must be > 0");
    if (!supported_D(doe.D)) return fail(ctx, RW_EINVAL, "doe.D must be 16, 32, 64 or 96");
    const int pad = doe.pad > 0 ? doe.pad : 1;
    if (pad > 8 || !supported_M(pad * doe.D))
        return fail(ctx, RW_EINVAL, "doe.pad * doe.D must be 16, 32, 64, 96 or 128");
    if (doe.gather != RW_GATHER_NEAREST && doe.gather != RW_GATHER_BILINEAR)
        return fail(ctx, RW_EINVAL, "doe.gather invalid");
    if (doe.emit != RW_EMIT_EXHAUSTIVE && doe.emit != RW_EMIT_SAMPLED &&
        doe.emit != RW_EMIT_SAMPLED_UNIFORM)
        return fail(ctx, RW_EINVAL, "doe.emit invalid");
    if (doe.emit != RW_EMIT_EXHAUSTIVE && (doe.n_ssr < 1 || doe.n_ssr > 16384))
        return fail(ctx, RW_EINVAL, "doe.n_ssr must be in 1..16384 for sampled emission");
    if (doe.phase_model != RW_PHASE_HEIGHT && doe.phase_model != RW_PHASE_FIXED)
        return fail(ctx, RW_EINVAL, "doe.phase_model invalid");
    if (doe.phase_model == RW_PHASE_HEIGHT && !(doe.lambda0 > 0))
        return fail(ctx, RW_EINVAL, "doe.lambda0 must be > 0 for the height model");
    if (doe.dft != RW_DFT_FFT32 && doe.dft != RW_DFT_TC)
        return fail(ctx, RW_EINVAL, "doe.dft invalid");
    if (doe.flags & ~(RW_DOE_TRACE_ALL | RW_DOE_REFLECTIVE))
        return fail(ctx, RW_EINVAL, "doe.flags has unknown bits");
    const bool reflective = (doe.flags & RW_DOE_REFLECTIVE) != 0;
    const rw_sensor& sen = sys->sensor;
    if (sen.nx < 1 || sen.ny < 1 || !(sen.pitch > 0))
        return fail(ctx, RW_EINVAL, "sensor size and pitch must be positive");
    if (sen.window < 0) return fail(ctx, RW_EINVAL, "sensor.window must be >= 0");
    DSys& d = P.sys;
    std::memset(&d, 0, sizeof(d));
    d.nsurf = sys->nsurf;
    d.doe_index = sys->doe_index;
    d.n_object = sys->n_object;
    double prev_z = 0.0, n_prev = sys->n_object;
    for (int i = 0; i < sys->nsurf; ++i) {
        const rw_surface& s = sys->surfaces[i];
        if (s.kind != RW_PLANE && s.kind != RW_SPHERE && s.kind != RW_ASPHERE &&
            s.kind != RW_GAUSS)
            return fail(ctx, RW_EINVAL, "surface kind invalid");
        if (s.kind == RW_GAUSS && i != sys->doe_index)
            return fail(ctx, RW_EINVAL, "RW_GAUSS is only a DOE substrate");
        if (s.kind == RW_GAUSS && !(s.k > 0) )
            return fail(ctx, RW_EINVAL, "RW_GAUSS width k must be > 0");
        if (i > 0 && s.z < sys->surfaces[i - 1].z)
            return fail(ctx, RW_EINVAL, "surfaces must be sorted by z");
        if (!(s.n_after > 0)) return fail(ctx, RW_EINVAL, "surface n_after must be > 0");
        if (!std::isfinite(s.z) || !std::isfinite(s.c)) return fail(ctx, RW_EINVAL, "surface not finite");
        DSurf& o = d.s[i];
        o.kind = s.kind;
        o.c = (float)(s.kind == RW_PLANE ? 0.0 : s.c);
        o.cd = (s.kind == RW_PLANE ? 0.0 : s.c);
        o.kd = s.k;
        o.k = (float)s.k;
        o.A4 = (float)s.A4; o.A6 = (float)s.A6; o.A8 = (float)s.A8; o.A10 = (float)s.A10;
        o.n_before = (float)n_prev;
        o.n_after = (float)s.n_after;
        o.r_ap2 = s.r_ap > 0 ? (float)(s.r_ap * s.r_ap) : 0.f;
        o.gap = (float)(s.z - prev_z);
        o.z = s.z;
        o.A4d = s.A4; o.A6d = s.A6; o.A8d = s.A8; o.A10d = s.A10;
        o.nbd = n_prev;
        o.nad = s.n_after;
        o.r_ap2d = s.r_ap > 0 ? s.r_ap * s.r_ap : 0.0;
        if (i == sys->doe_index) {
            if (s.kind == RW_ASPHERE)
                return fail(ctx, RW_EINVAL, "DOE surface must be PLANE, SPHERE or GAUSS");
            d.n_in = (float)n_prev;
            d.n_in_d = n_prev;
            // a reflective DOE sends the secondary rays back into the incident medium
            d.n_out = reflective ? (float)n_prev : (float)s.n_after;
            d.conformal = (s.kind == RW_SPHERE || s.kind == RW_GAUSS) ? 1 : 0;
        }
        prev_z = s.z;
        // behind a reflective DOE (the last surface) the rays travel in n_in
        if (!(reflective && i == sys->doe_index)) n_prev = s.n_after;
    }
    if (reflective) {
        if (sys->doe_index != sys->nsurf - 1)
            return fail(ctx, RW_EINVAL, "a reflective DOE must be the last surface");
        if (!(sen.z < sys->surfaces[sys->doe_index].z))
            return fail(ctx, RW_EINVAL, "the sensor must lie in front of a reflective DOE");
        if (sys->surfaces[sys->doe_index].kind == RW_GAUSS &&
            sen.z > sys->surfaces[sys->doe_index].z + std::min(0.0, sys->surfaces[sys->doe_index].c))
            return fail(ctx, RW_EINVAL, "the sensor must lie in front of a reflective DOE");
    } else if (sen.z < prev_z) {
        return fail(ctx, RW_EINVAL, "sensor must lie behind the last surface");
    }
    d.reflective = reflective ? 1 : 0;
    // surface whose n_after is the index the secondary rays enter / the
    // sensor medium (-1: the object space index, no gradient slot)
    d.nout_slot = reflective ? sys->doe_index - 1 : sys->doe_index;
    d.nsen_slot = reflective ? sys->doe_index - 1 : sys->nsurf - 1;
    d.two_phase = doe.phi2 ? 1 : 0;
    d.phi = doe.phi;
    d.phi2 = doe.phi2;
    // surfaces behind the DOE for the specialised plane/sphere trace
    d.n_post = sys->nsurf - sys->doe_index - 1;
    d.fast_ok = d.n_post <= 8 ? 1 : 0;
    for (int i = 0; i < d.n_post && d.fast_ok; ++i) {
        const int si = sys->doe_index + 1 + i;
        const rw_surface& s = sys->surfaces[si];
        if (s.kind == RW_ASPHERE) { d.fast_ok = 0; break; }
        PSurf& q = d.post[i];
        q.kind = s.kind;
        q.c = (s.kind == RW_PLANE) ? 0.f : (float)s.c;
        q.gap = d.s[si].gap;
        q.r_ap2 = d.s[si].r_ap2;
        const double nb = (si == 0) ? sys->n_object : sys->surfaces[si - 1].n_after;
        q.eta = (float)(nb / s.n_after);
        q.inv_n_after = (float)(1.0 / s.n_after);
    }
    d.H = doe.H; d.W = doe.W; d.D = doe.D;
    d.M = pad * doe.D;
    // coherent: Fourier-series coefficient of the padded patch; incoherent:
    // keeps sum |U~|^2 = mean |T|^2 (both 1/D^2 without padding)
    d.norm = sen.coherent ? (float)(1.0 / ((double)d.M * d.M)) : (float)(1.0 / ((double)d.D * d.M));
    d.gather = doe.gather;
    // kernels see two modes; uniform sampling is the sampled mode with p = 1/n_prop
    d.emit = doe.emit == RW_EMIT_EXHAUSTIVE ? RW_EMIT_EXHAUSTIVE : RW_EMIT_SAMPLED;
    d.uniform = doe.emit == RW_EMIT_SAMPLED_UNIFORM ? 1 : 0;
    d.n_ssr = doe.n_ssr;
    d.phase_model = doe.phase_model;
    d.pitch = doe.pitch;
    d.pitchf = (float)doe.pitch;
    d.inv_pitch = (float)(1.0 / doe.pitch);
    d.seed = doe.seed;
    d.rng_offset = doe.rng_offset;
    d.kstep = (float)(2.0 * M_PI / (d.M * doe.pitch));
    d.cull = (doe.flags & RW_DOE_TRACE_ALL) ? 0 : 1;
    d.sensor_z = sen.z;
    d.sensor_gap = (float)(sen.z - prev_z);
    d.nx = sen.nx; d.ny = sen.ny;
    d.spitch = (float)sen.pitch;
    d.inv_spitch = (float)(1.0 / sen.pitch);
    d.coherent = sen.coherent ? 1 : 0;
    // per-ray adjoint sums: the conformal frame and patch gather add theirs
    d.nrs = d.conformal ? RW_RS : (d.coherent ? 7 : 6);
    d.window = sen.window;
    d.n_sensor = (float)n_prev;
    return RW_OK;
}

// outs[i]: image of job i in the psf / dL/dpsf arrays (default i)
static rw_status pack_jobs(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs, int njob,
                           int64_t n_rays, Packed& P, const int* outs = nullptr) {
    if (njob < 1) return fail(ctx, RW_EINVAL, "njob must be >= 1");
    if (!jobs) return fail(ctx, RW_EINVAL, "jobs is NULL");
    std::map<double, int> slot_of;
    P.jobs.resize(njob);
    P.prefix.resize(njob + 1);
    P.prefix[0] = 0;
    for (int i = 0; i < njob; ++i) {
        const rw_job& j = jobs[i];
        if (!(j.lambda > 0)) return fail(ctx, RW_EINVAL, "job lambda must be > 0");
        if (j.ray_count < 0 || j.ray_offset < 0 || j.ray_offset + j.ray_count > n_rays)
            return fail(ctx, RW_EINVAL, "job ray range outside the ray arrays");
        auto it = slot_of.find(j.lambda);
        int slot;
        if (it == slot_of.end()) {
            slot = (int)P.scales.size();
            slot_of[j.lambda] = slot;
            P.scales.push_back(sys->doe.phase_model == RW_PHASE_HEIGHT
                                   ? (float)(sys->doe.lambda0 / j.lambda) : 1.f);
        } else {
            slot = it->second;
        }
        DJob& d = P.jobs[i];
        d.lambda = j.lambda;
        d.k0 = (float)(2.0 * M_PI / j.lambda);
        d.phase_scale = P.scales[slot];
        d.off = j.ray_offset;
        d.cnt = j.ray_count;
        d.cx = (float)j.sensor_cx;
        d.cy = (float)j.sensor_cy;
        d.cxd = j.sensor_cx;
        d.cyd = j.sensor_cy;
        d.slot = slot;
        d.out = outs ? outs[i] : i;
        P.prefix[i + 1] = P.prefix[i] + j.ray_count;
    }
    P.total = P.prefix[njob];
    return RW_OK;
}

static rw_status check_rays(rw_ctx* ctx, const rw_rays* r) {
    if (!r) return fail(ctx, RW_EINVAL, "rays is NULL");
    if (r->n < 0) return fail(ctx, RW_EINVAL, "rays.n < 0");
    if (r->n > 0 && (!r->ox || !r->oy || !r->oz || !r->dx || !r->dy || !r->dz || !r->a_re ||
                     !r->a_im || !r->opl))
        return fail(ctx, RW_EINVAL, "a ray array is NULL");
    return RW_OK;
}

static RaysIn rays_in(const rw_rays* r) {
    RaysIn x;
    x.ox = r->ox; x.oy = r->oy; x.oz = r->oz; x.dx = r->dx; x.dy = r->dy; x.dz = r->dz;
    x.are = r->a_re; x.aim = r->a_im; x.opl = r->opl;
    return x;
}

static size_t shared_limit_ok(rw_ctx* ctx, const DSys& d) {
    int lim = 0;
    cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    return forward_smem_bytes(d.M, d.emit, d.n_ssr) <= (size_t)lim;
}

// Prepare the transmission maps and device tables.  Returns device pointers.
static rw_status prepare(rw_ctx* ctx, const rw_system* sys, const Packed& P, float2** T,
                         DJob** djobs, long long** dprefix) {
    if (!shared_limit_ok(ctx, P.sys))
        return fail(ctx, RW_EINVAL, "patch size / n_ssr too large for the forward's shared memory "
                                    "(sampled emission: M <= 96)");
    std::vector<void*> ptrs;
    rw_status st = upload(ctx, {{P.jobs.data(), P.jobs.size() * sizeof(DJob)},
                                {P.prefix.data(), P.prefix.size() * sizeof(long long)},
                                {P.scales.data(), P.scales.size() * sizeof(float)}},
                          ptrs);
    if (st != RW_OK) return st;
    *djobs = (DJob*)ptrs[0];
    *dprefix = (long long*)ptrs[1];
    const int64_t npix = (int64_t)sys->doe.H * sys->doe.W;
    const int nslot = (int)P.scales.size();
    st = ensure_buf(ctx, ctx->tmaps, (size_t)npix * nslot * sizeof(float2),
                    "transmission-map scratch");
    if (st != RW_OK) return st;
    *T = (float2*)ctx->tmaps.p;
    RW_CUDA(launch_prep_maps(lctx(ctx), sys->doe.phi, sys->doe.phi2, sys->doe.amp, npix,
                             (const float*)ptrs[2], nslot, *T),
            "prep maps");
    ctx->launches++;
    return RW_OK;
}

// ---------------------------------------------------------------- API
extern "C" {

const char* rw_version(void) { return "raywave-gb300 0.1 (sm_103a)"; }

rw_status rw_create(rw_ctx** out, int device, void* cuda_stream) {
    if (!out) return RW_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return RW_EINVAL;
    rw_ctx* ctx = new rw_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return RW_ECUDA; }
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaEventCreateWithFlags(&ctx->staging_done, cudaEventDisableTiming) != cudaSuccess ||
        ctx->misc.ensure(256) != cudaSuccess ||
        cudaMemset(ctx->misc.p, 0, 256) != cudaSuccess ||
        cudaMallocHost(&ctx->cap_host, RW_CAPTURE_ARENA) != cudaSuccess ||
        cudaMallocHost((void**)&ctx->count_host, 64) != cudaSuccess ||
        ctx->cap_dev.ensure(RW_CAPTURE_ARENA) != cudaSuccess) {
        delete ctx;
        return RW_ECUDA;
    }
    const char* g = std::getenv("RW_GRID");
    if (g) ctx->grid_override = std::atoll(g);
    *out = ctx;
    return RW_OK;
}

rw_status rw_destroy(rw_ctx* ctx) {
    if (!ctx) return RW_EINVAL;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream); else cudaDeviceSynchronize();
    ctx->tmaps.release();
    ctx->tables.release();
    ctx->field.release();
    ctx->coh_rsum.release();
    ctx->coh_jsum.release();
    ctx->acc.release();
    ctx->misc.release();
    ctx->cap_dev.release();
    ctx->split_rays.release();
    ctx->split_items.release();
    ctx->keep.release();
    if (ctx->cap_host) cudaFreeHost(ctx->cap_host);
    if (ctx->count_host) cudaFreeHost(ctx->count_host);
    if (ctx->staging) cudaFreeHost(ctx->staging);
    if (ctx->staging_done) cudaEventDestroy(ctx->staging_done);
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    delete ctx;
    return RW_OK;
}

rw_status rw_profile(rw_ctx* ctx, int32_t enable) {
    if (!ctx) return RW_EINVAL;
    ctx->err.clear();
    RW_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    RW_CUDA(cudaStreamSynchronize(ctx->stream), "profile sync");
    ctx->prof_on = enable != 0;
    ctx->prof_used = 0;
    ctx->prof_kernels.clear();
    ctx->prof_ms.clear();
    ctx->prof_count.clear();
    return RW_OK;
}

rw_status rw_profile_read(rw_ctx* ctx, int32_t* n_kernels) {
    if (!ctx || !n_kernels) return fail(ctx, RW_EINVAL, "null argument");
    ctx->err.clear();
    RW_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    RW_CUDA(cudaStreamSynchronize(ctx->stream), "profile sync");
    for (size_t i = 0; i + 1 < ctx->prof_used; ++i) {
        const char* name = ctx->prof_names[i];
        if (!name || ctx->prof_names[i + 1]) continue;     // a start mark followed by its end
        float ms = 0.f;
        RW_CUDA(cudaEventElapsedTime(&ms, ctx->prof_pool[i], ctx->prof_pool[i + 1]), "elapsed");
        size_t k = 0;
        while (k < ctx->prof_kernels.size() && ctx->prof_kernels[k] != name) ++k;
        if (k == ctx->prof_kernels.size()) {
            ctx->prof_kernels.push_back(name);
            ctx->prof_ms.push_back(0.0);
            ctx->prof_count.push_back(0);
        }
        ctx->prof_ms[k] += ms;
        ctx->prof_count[k] += 1;
    }
    ctx->prof_used = 0;
    *n_kernels = (int32_t)ctx->prof_kernels.size();
    return RW_OK;
}

rw_status rw_profile_entry(rw_ctx* ctx, int32_t i, const char** kernel, double* total_ms,
                           int64_t* launches) {
    if (!ctx || !kernel || !total_ms || !launches) return fail(ctx, RW_EINVAL, "null argument");
    if (i < 0 || i >= (int32_t)ctx->prof_kernels.size())
        return fail(ctx, RW_EINVAL, "profile entry out of range");
    *kernel = ctx->prof_kernels[i].c_str();
    *total_ms = ctx->prof_ms[i];
    *launches = ctx->prof_count[i];
    return RW_OK;
}

rw_status rw_cull_stats(rw_ctx* ctx, int64_t* blocks, int64_t* kept) {
    if (!ctx || !blocks || !kept) return fail(ctx, RW_EINVAL, "null argument");
    ctx->err.clear();
    *blocks = ctx->keep_blocks;
    *kept = 0;
    if (ctx->keep_words == 0) return RW_OK;
    RW_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    unsigned long long* dcount = reinterpret_cast<unsigned long long*>(
        reinterpret_cast<char*>(ctx->misc.p) + 128);
    RW_CUDA(launch_bs_count(lctx(ctx), (const unsigned*)ctx->keep.p, ctx->keep_words, dcount),
            "kept-block count");
    ctx->launches++;
    RW_CUDA(cudaMemcpyAsync(ctx->count_host, dcount, sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, ctx->stream), "count read");
    RW_CUDA(cudaStreamSynchronize(ctx->stream), "count sync");
    *kept = (int64_t)*ctx->count_host;
    return RW_OK;
}

rw_status rw_set_stream(rw_ctx* ctx, void* cuda_stream) {
    if (!ctx) return RW_EINVAL;
    ctx->stream = (cudaStream_t)cuda_stream;
    return RW_OK;
}

const char* rw_last_error(const rw_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t rw_launch_count(const rw_ctx* ctx) { return ctx ? ctx->launches : 0; }

rw_status rw_device_status(rw_ctx* ctx, uint32_t* status_out) {
    if (!ctx || !status_out) return fail(ctx, RW_EINVAL, "null argument");
    RW_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    unsigned v = 0;
    RW_CUDA(cudaMemcpyAsync(&v, status_word(ctx), sizeof(unsigned), cudaMemcpyDeviceToHost,
                            ctx->stream), "status read");
    RW_CUDA(cudaStreamSynchronize(ctx->stream), "status sync");
    RW_CUDA(cudaMemsetAsync(status_word(ctx), 0, sizeof(unsigned), ctx->stream), "status clear");
    *status_out = v;
    return RW_OK;
}

rw_status rw_generate_rays(rw_ctx* ctx, double z_start, double n_object, const rw_job* jobs,
                           int32_t njob, rw_rays* rays) {
    if (!ctx) return RW_EINVAL;
    ctx->err.clear();
    rw_status st = check_rays(ctx, rays);
    if (st != RW_OK) return st;
    if (njob < 1 || !jobs) return fail(ctx, RW_EINVAL, "jobs missing");
    if (!(n_object > 0)) return fail(ctx, RW_EINVAL, "n_object must be > 0");
    std::vector<GenJob> g(njob);
    std::vector<long long> prefix(njob + 1, 0);
    if (const char* why = gen_table_fill(jobs, njob, rays->n, g.data(), prefix.data()))
        return fail(ctx, RW_EINVAL, why);
    if (prefix[njob] == 0) return RW_OK;
    std::vector<void*> ptrs;
    st = upload(ctx, {{g.data(), g.size() * sizeof(GenJob)},
                      {prefix.data(), prefix.size() * sizeof(long long)}}, ptrs);
    if (st != RW_OK) return st;
    RaysOut o;
    o.ox = rays->ox; o.oy = rays->oy; o.oz = rays->oz; o.dx = rays->dx; o.dy = rays->dy;
    o.dz = rays->dz; o.are = rays->a_re; o.aim = rays->a_im; o.opl = rays->opl;
    RW_CUDA(launch_generate_rays(lctx(ctx), (GenJob*)ptrs[0], (long long*)ptrs[1], njob,
                                 prefix[njob], z_start, n_object, o), "generate rays");
    ctx->launches++;
    return RW_OK;
}

rw_status rw_doe_emit(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs, int32_t njob,
                      const rw_rays* rays, rw_emitted* out) {
    if (!ctx) return RW_EINVAL;
    ctx->err.clear();
    if (is_dispersive(sys))
        return fail(ctx, RW_EINVAL, "dispersive surfaces: rw_forward and rw_backward only");
    Packed P;
    rw_status st = pack_system(ctx, sys, P);
    if (st != RW_OK) return st;
    if (sys->doe.dft == RW_DFT_TC)
        return fail(ctx, RW_EINVAL, "the fused kernels use the FP32 FFT; the tensor-core "
                                    "transform is available through rw_patch_spectra");
    if ((st = check_rays(ctx, rays)) != RW_OK) return st;
    if ((st = pack_jobs(ctx, sys, jobs, njob, rays->n, P)) != RW_OK) return st;
    if (!out || !out->dx || !out->dy || !out->dz || !out->a_re || !out->a_im || !out->hx ||
        !out->hy || !out->hz || !out->opl)
        return fail(ctx, RW_EINVAL, "an emitted-ray array is NULL");
    const long long S = (P.sys.emit == RW_EMIT_EXHAUSTIVE) ? (long long)P.sys.M * P.sys.M
                                                           : (long long)P.sys.n_ssr;
    if (out->capacity < P.total * S)
        return fail(ctx, RW_ECAPACITY, "emitted capacity < n_rays * slots per ray");
    if (P.total == 0) return RW_OK;
    float2* T; DJob* dj; long long* dp;
    if ((st = prepare(ctx, sys, P, &T, &dj, &dp)) != RW_OK) return st;
    EmitOut eo;
    eo.dx = out->dx; eo.dy = out->dy; eo.dz = out->dz; eo.are = out->a_re; eo.aim = out->a_im;
    eo.bin = out->bin; eo.hx = out->hx; eo.hy = out->hy; eo.hz = out->hz; eo.opl = out->opl;
    RW_CUDA(launch_forward(lctx(ctx), MODE_EMIT, P.sys, dj, dp, njob, P.total, rays_in(rays), T,
                           nullptr, nullptr, eo, status_word(ctx)), "emit kernel");
    ctx->launches++;
    return RW_OK;
}

static rw_status forward_dispersive(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs,
                                    int32_t njob, const rw_rays* rays, float* psf);
static rw_status backward_dispersive(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs,
                                     int32_t njob, const rw_rays* rays, const float* dl_dpsf,
                                     float* dphi, float* damp, double* dsurf);

static rw_status forward_impl(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs,
                              int32_t njob, const rw_rays* rays, float* psf, uint32_t* vis,
                              int64_t vis_words) {
    if (!ctx) return RW_EINVAL;
    ctx->err.clear();
    if (is_dispersive(sys)) {
        if (vis) return fail(ctx, RW_EINVAL, "the visibility mask needs non-dispersive media");
        return forward_dispersive(ctx, sys, jobs, njob, rays, psf);
    }
    Packed P;
    rw_status st = pack_system(ctx, sys, P);
    if (st != RW_OK) return st;
    const bool tc = sys->doe.dft == RW_DFT_TC;
    if (tc && (P.sys.D != 64 || P.sys.M != 64 || P.sys.emit != RW_EMIT_EXHAUSTIVE ||
               P.sys.coherent))
        return fail(ctx, RW_EINVAL, "the fused tensor-core patch transform needs D = 64 without "
                                    "padding, exhaustive emission and the incoherent sensor");
    if ((st = check_rays(ctx, rays)) != RW_OK) return st;
    if ((st = pack_jobs(ctx, sys, jobs, njob, rays->n, P)) != RW_OK) return st;
    if (!psf) return fail(ctx, RW_EINVAL, "psf is NULL");
    if (vis) {
        if (P.sys.coherent || P.sys.emit != RW_EMIT_EXHAUSTIVE)
            return fail(ctx, RW_EINVAL, "the visibility mask needs the incoherent sensor and "
                                        "exhaustive emission");
        if (vis_words < P.total * (int64_t)P.sys.M * P.sys.M / 32)
            return fail(ctx, RW_ECAPACITY, "vis_words < n_rays * M * M / 32");
    }
    const long long npx = (long long)P.sys.nx * P.sys.ny * njob;
    RW_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    RW_CUDA(cudaMemsetAsync(psf, 0, npx * sizeof(float), ctx->stream), "psf clear");
    if (P.total == 0) return RW_OK;
    float2* T; DJob* dj; long long* dp;
    if ((st = prepare(ctx, sys, P, &T, &dj, &dp)) != RW_OK) return st;
    EmitOut eo;
    std::memset(&eo, 0, sizeof(eo));
    if (P.sys.coherent) {
        if ((st = ensure_buf(ctx, ctx->field, npx * sizeof(float2), "coherent field scratch")) !=
            RW_OK)
            return st;
        RW_CUDA(cudaMemsetAsync(ctx->field.p, 0, npx * sizeof(float2), ctx->stream), "field clear");
        RW_CUDA(launch_forward(lctx(ctx), MODE_COHERENT, P.sys, dj, dp, njob, P.total,
                               rays_in(rays), T, nullptr, (float2*)ctx->field.p, eo,
                               status_word(ctx)), "coherent forward");
        ctx->launches++;
        RW_CUDA(launch_coherent_finalize(lctx(ctx), (float2*)ctx->field.p, psf, npx), "finalize");
        ctx->launches++;
    } else {
        if ((st = ensure_buf(ctx, ctx->acc, npx * sizeof(double), "PSF accumulator scratch")) !=
            RW_OK)
            return st;
        RW_CUDA(cudaMemsetAsync(ctx->acc.p, 0, npx * sizeof(double), ctx->stream), "acc clear");
        unsigned* keep = nullptr;
        SplitBufs tape;
        std::memset(&tape, 0, sizeof(tape));
        if (vis) {
            ctx->tape_valid = false;
            tape.epoch = tape_counter(ctx) + 1;
        }
        if (forward_culls(P.sys)) {
            const size_t kb = (size_t)P.total * cull_keep_words(P.sys.M) * sizeof(unsigned);
            if ((st = ensure_buf(ctx, ctx->keep, kb, "block-culling scratch")) != RW_OK) return st;
            keep = (unsigned*)ctx->keep.p;
            ctx->keep_words = (long long)P.total * cull_keep_words(P.sys.M);
            ctx->keep_blocks = (long long)P.total * (P.sys.M / 8) * (P.sys.M / 8);
            ctx->launches++;          // k_cull
            if (vis && !capturing(ctx)) {
                // tape the visible secondary rays for the adjoint
                long long cap = ctx->tape_hint;
                if (cap <= 0) cap = std::max<long long>(1 << 20, P.total * P.sys.M * P.sys.M / 64);
                if ((st = split_buffers(ctx, P.total, cap, P.sys.nrs, tape)) != RW_OK) return st;
                tape.counter = tape_counter(ctx);
                RW_CUDA(cudaMemsetAsync(tape.counter, 0, sizeof(unsigned long long), ctx->stream),
                        "tape counter");
                ctx->tape_valid = true;
                ctx->tape_vis = vis;
                ctx->tape_total = P.total;
                ctx->tape_M = P.sys.M;
                ctx->tape_cap = cap;
            }
        }
        if (tc) {
            RW_CUDA(launch_forward_tc(lctx(ctx), P.sys, dj, dp, njob, P.total, rays_in(rays), T,
                                      (double*)ctx->acc.p, status_word(ctx), vis, keep,
                                      vis ? &tape : nullptr),
                    "tensor-core forward kernel");
        } else {
            RW_CUDA(launch_forward(lctx(ctx), MODE_SPLAT, P.sys, dj, dp, njob, P.total,
                                   rays_in(rays), T, (double*)ctx->acc.p, nullptr, eo,
                                   status_word(ctx), vis, keep, vis ? &tape : nullptr),
                    "forward kernel");
        }
        ctx->launches++;
        RW_CUDA(launch_psf_finalize(lctx(ctx), (const double*)ctx->acc.p, psf, npx), "psf finalize");
        ctx->launches++;
    }
    return RW_OK;
}

rw_status rw_forward(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs, int32_t njob,
                     const rw_rays* rays, float* psf) {
    return forward_impl(ctx, sys, jobs, njob, rays, psf, nullptr, 0);
}

rw_status rw_forward_vis(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs, int32_t njob,
                         const rw_rays* rays, float* psf, uint32_t* vis, int64_t vis_words) {
    if (!vis) return fail(ctx, RW_EINVAL, "vis is NULL");
    return forward_impl(ctx, sys, jobs, njob, rays, psf, vis, vis_words);
}

rw_status rw_loss_eq3(rw_ctx* ctx, const float* psf, const float* target, int64_t n,
                      double* loss_out, float* dl_dpsf) {
    if (!ctx) return RW_EINVAL;
    ctx->err.clear();
    if (!psf || !target || !loss_out) return fail(ctx, RW_EINVAL, "null argument");
    if (n < 1) return fail(ctx, RW_EINVAL, "n must be >= 1");
    RW_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    RW_CUDA(launch_loss_eq3(lctx(ctx), psf, target, n, loss_acc(ctx), loss_out, dl_dpsf), "loss");
    ctx->launches += 2;
    return RW_OK;
}

static rw_status backward_impl(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs,
                               int32_t njob, const rw_rays* rays, const float* dl_dpsf,
                               const uint32_t* vis, int64_t vis_words, float* dphi, float* damp,
                               double* dsurf) {
    if (!ctx) return RW_EINVAL;
    ctx->err.clear();
    if (is_dispersive(sys)) {
        if (vis) return fail(ctx, RW_EINVAL, "the visibility mask needs non-dispersive media");
        return backward_dispersive(ctx, sys, jobs, njob, rays, dl_dpsf, dphi, damp, dsurf);
    }
    Packed P;
    rw_status st = pack_system(ctx, sys, P);
    if (st != RW_OK) return st;
    // the adjoint re-forms the patch spectra with the FP32 FFT whatever
    // doe.dft selects (see rw_backward)
    if ((st = check_rays(ctx, rays)) != RW_OK) return st;
    if ((st = pack_jobs(ctx, sys, jobs, njob, rays->n, P)) != RW_OK) return st;
    if (!dl_dpsf) return fail(ctx, RW_EINVAL, "dl_dpsf is NULL");
    if (P.sys.coherent && vis)
        return fail(ctx, RW_EINVAL, "the visibility mask needs the incoherent sensor");
    // the split adjoint (three kernels) needs the mask and a host read-back of
    // its count, so it runs eagerly; otherwise the fused kernel
    const bool split = vis && P.sys.emit == RW_EMIT_EXHAUSTIVE && !capturing(ctx);
    if (!split) {
        int lim = 0;
        cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
        if (P.sys.M > 96 || backward_smem_needed(P.sys) > (size_t)lim)
            return fail(ctx, RW_EINVAL, "patch size / n_ssr too large for the fused adjoint's "
                                        "shared memory (M = 128 needs exhaustive emission with "
                                        "a visibility mask, outside graph capture)");
    }
    if (damp && !sys->doe.amp) return fail(ctx, RW_EINVAL, "damp requires doe.amp");
    if (vis) {
        if (P.sys.emit != RW_EMIT_EXHAUSTIVE)
            return fail(ctx, RW_EINVAL, "the visibility mask needs exhaustive emission");
        if (vis_words < P.total * (int64_t)P.sys.M * P.sys.M / 32)
            return fail(ctx, RW_ECAPACITY, "vis_words < n_rays * M * M / 32");
    }
    if (P.total == 0 || (!dphi && !damp && !dsurf)) return RW_OK;
    float2* T; DJob* dj; long long* dp;
    if ((st = prepare(ctx, sys, P, &T, &dj, &dp)) != RW_OK) return st;
    if (split) {
        // Split adjoint over the mask's visible secondary rays: with the
        // forward's tape for this mask, trace+reverse / conjugate FFT+scatter
        // of the taped work list; otherwise count them (one host sync), size the
        // work list and run spectra+list / trace+reverse / conjugate FFT+scatter.
        SplitBufs B;
        std::memset(&B, 0, sizeof(B));
        long long nitems = 0;
        bool taped = ctx->tape_valid && ctx->tape_vis == (const void*)vis &&
                     ctx->tape_total == P.total && ctx->tape_M == P.sys.M;
        if (taped) {
            // counter, epoch, tape epoch: a forward with a mask replayed from a
            // graph since the tape was written has moved the epoch on
            RW_CUDA(cudaMemcpyAsync(ctx->count_host, tape_counter(ctx),
                                    3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                    ctx->stream), "tape count read");
            RW_CUDA(cudaStreamSynchronize(ctx->stream), "tape count sync");
            nitems = (long long)ctx->count_host[0];
            if (ctx->count_host[1] != ctx->count_host[2]) {
                taped = false;
            } else if (nitems > ctx->tape_cap) {
                // the tape overflowed: size the next one, recompute this time
                ctx->tape_hint = nitems + nitems / 8 + 1024;
                taped = false;
            } else {
                if ((st = split_buffers(ctx, P.total, ctx->tape_cap, P.sys.nrs, B)) != RW_OK) return st;
                B.counter = tape_counter(ctx);
            }
        }
        if (!taped) {
            ctx->tape_valid = false;          // the buffers are reused below
            const long long nwords = P.total * (long long)P.sys.M * P.sys.M / 32;
            unsigned long long* dcount = reinterpret_cast<unsigned long long*>(
                reinterpret_cast<char*>(ctx->misc.p) + 128);
            RW_CUDA(launch_bs_count(lctx(ctx), vis, nwords, dcount), "visible count");
            ctx->launches++;
            RW_CUDA(cudaMemcpyAsync(ctx->count_host, dcount, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, ctx->stream), "count read");
            RW_CUDA(cudaStreamSynchronize(ctx->stream), "count sync");
            nitems = (long long)*ctx->count_host;
            if ((st = split_buffers(ctx, P.total, nitems, P.sys.nrs, B)) != RW_OK) return st;
            B.counter = dcount;
            RW_CUDA(cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), ctx->stream), "counter");
        }
        RW_CUDA(cudaMemsetAsync(B.rsum, 0, P.total * P.sys.nrs * sizeof(float), ctx->stream),
                "sums");
        RW_CUDA(launch_backward_split(lctx(ctx), P.sys, dj, dp, njob, P.total, rays_in(rays), T,
                                      sys->doe.amp, dl_dpsf, vis, B, nitems, taped ? 1 : 0, dphi,
                                      damp, dsurf, status_word(ctx)),
                "split adjoint");
        ctx->launches += (taped ? 1 : 2) + (nitems > 0 ? 1 : 0);
        return RW_OK;
    }
    float2* gfield = nullptr;
    float* coh_rsum = nullptr;
    double* coh_jsum = nullptr;
    if (P.sys.coherent) {
        if ((st = ensure_buf(ctx, ctx->coh_rsum, (size_t)P.total * P.sys.nrs * sizeof(float),
                             "coherent adjoint scratch")) != RW_OK)
            return st;
        if ((st = ensure_buf(ctx, ctx->coh_jsum, (size_t)njob * 2 * sizeof(double),
                             "coherent adjoint scratch")) != RW_OK)
            return st;
        coh_rsum = (float*)ctx->coh_rsum.p;
        coh_jsum = (double*)ctx->coh_jsum.p;
        RW_CUDA(cudaMemsetAsync(coh_jsum, 0, (size_t)njob * 2 * sizeof(double), ctx->stream),
                "job sums clear");
        // per-ray sums: bin slices of one ray add into them
        RW_CUDA(cudaMemsetAsync(coh_rsum, 0, (size_t)P.total * P.sys.nrs * sizeof(float), ctx->stream),
                "ray sums clear");
        // I = |U|^2 loses the phase of U: recompute the field, then
        // dL/dU = 2 (dL/dI) U in place
        const long long npx = (long long)P.sys.nx * P.sys.ny * njob;
        if ((st = ensure_buf(ctx, ctx->field, npx * sizeof(float2), "coherent field scratch")) !=
            RW_OK)
            return st;
        gfield = (float2*)ctx->field.p;
        EmitOut eo;
        std::memset(&eo, 0, sizeof(eo));
        RW_CUDA(cudaMemsetAsync(gfield, 0, npx * sizeof(float2), ctx->stream), "field clear");
        RW_CUDA(launch_forward(lctx(ctx), MODE_COHERENT, P.sys, dj, dp, njob, P.total,
                               rays_in(rays), T, nullptr, gfield, eo, status_word(ctx)),
                "coherent field");
        RW_CUDA(launch_coherent_grad(lctx(ctx), gfield, dl_dpsf, npx), "field gradient");
        ctx->launches += 2;
    }
    int nl = 0;
    RW_CUDA(launch_backward(lctx(ctx), P.sys, dj, dp, njob, P.total, rays_in(rays), T,
                            sys->doe.amp, dl_dpsf, gfield, coh_rsum, coh_jsum, dphi, damp,
                            dsurf, vis, status_word(ctx), &nl),
            "backward kernel");
    ctx->launches += nl;
    return RW_OK;
}

// One launch per wavelength group into shared outputs (see is_dispersive).
static rw_status forward_dispersive(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs,
                                    int32_t njob, const rw_rays* rays, float* psf) {
    WaveGroups G;
    rw_status st = group_by_wavelength(ctx, jobs, njob, G);
    if (st != RW_OK) return st;
    if (sys->doe.dft == RW_DFT_TC)
        return fail(ctx, RW_EINVAL, "the fused kernels use the FP32 FFT; the tensor-core "
                                    "transform is available through rw_patch_spectra");
    if ((st = check_rays(ctx, rays)) != RW_OK) return st;
    if (!psf) return fail(ctx, RW_EINVAL, "psf is NULL");
    std::vector<rw_system> sg(G.lambda.size());
    std::vector<std::vector<rw_surface>> surf(G.lambda.size());
    std::vector<Packed> P(G.lambda.size());
    long long total = 0;
    for (size_t g = 0; g < G.lambda.size(); ++g) {
        if ((st = system_at(ctx, sys, G.lambda[g], sg[g], surf[g])) != RW_OK) return st;
        if ((st = pack_system(ctx, &sg[g], P[g])) != RW_OK) return st;
        if ((st = pack_jobs(ctx, &sg[g], G.jobs[g].data(), (int)G.jobs[g].size(), rays->n, P[g],
                            G.out[g].data())) != RW_OK)
            return st;
        total += P[g].total;
    }
    const bool coherent = P[0].sys.coherent != 0;
    const long long npx = (long long)P[0].sys.nx * P[0].sys.ny * njob;
    RW_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    RW_CUDA(cudaMemsetAsync(psf, 0, npx * sizeof(float), ctx->stream), "psf clear");
    if (total == 0) return RW_OK;
    DevBuf& acc = coherent ? ctx->field : ctx->acc;
    const size_t bytes = npx * (coherent ? sizeof(float2) : sizeof(double));
    if ((st = ensure_buf(ctx, acc, bytes, "image accumulator scratch")) != RW_OK) return st;
    RW_CUDA(cudaMemsetAsync(acc.p, 0, bytes, ctx->stream), "accumulator clear");
    EmitOut eo;
    std::memset(&eo, 0, sizeof(eo));
    for (size_t g = 0; g < G.lambda.size(); ++g) {
        if (P[g].total == 0) continue;
        float2* T; DJob* dj; long long* dp;
        if ((st = prepare(ctx, &sg[g], P[g], &T, &dj, &dp)) != RW_OK) return st;
        const int nj = (int)G.jobs[g].size();
        if (coherent) {
            RW_CUDA(launch_forward(lctx(ctx), MODE_COHERENT, P[g].sys, dj, dp, nj, P[g].total,
                                   rays_in(rays), T, nullptr, (float2*)acc.p, eo,
                                   status_word(ctx)), "coherent forward");
        } else {
            unsigned* keep = nullptr;
            if (forward_culls(P[g].sys)) {
                const size_t kb = (size_t)P[g].total * cull_keep_words(P[g].sys.M) * sizeof(unsigned);
                if ((st = ensure_buf(ctx, ctx->keep, kb, "block-culling scratch")) != RW_OK)
                    return st;
                keep = (unsigned*)ctx->keep.p;
                ctx->launches++;      // k_cull
            }
            RW_CUDA(launch_forward(lctx(ctx), MODE_SPLAT, P[g].sys, dj, dp, nj, P[g].total,
                                   rays_in(rays), T, (double*)acc.p, nullptr, eo,
                                   status_word(ctx), nullptr, keep, nullptr), "forward kernel");
        }
        ctx->launches++;
    }
    if (coherent)
        RW_CUDA(launch_coherent_finalize(lctx(ctx), (float2*)acc.p, psf, npx), "finalize");
    else
        RW_CUDA(launch_psf_finalize(lctx(ctx), (const double*)acc.p, psf, npx), "psf finalize");
    ctx->launches++;
    return RW_OK;
}

static rw_status backward_dispersive(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs,
                                     int32_t njob, const rw_rays* rays, const float* dl_dpsf,
                                     float* dphi, float* damp, double* dsurf) {
    WaveGroups G;
    rw_status st = group_by_wavelength(ctx, jobs, njob, G);
    if (st != RW_OK) return st;
    if (sys->doe.dft == RW_DFT_TC)
        return fail(ctx, RW_EINVAL, "the fused kernels use the FP32 FFT; the tensor-core "
                                    "transform is available through rw_patch_spectra");
    if ((st = check_rays(ctx, rays)) != RW_OK) return st;
    if (!dl_dpsf) return fail(ctx, RW_EINVAL, "dl_dpsf is NULL");
    if (damp && !sys->doe.amp) return fail(ctx, RW_EINVAL, "damp requires doe.amp");
    std::vector<rw_system> sg(G.lambda.size());
    std::vector<std::vector<rw_surface>> surf(G.lambda.size());
    std::vector<Packed> P(G.lambda.size());
    long long total = 0;
    int lim = 0;
    cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    for (size_t g = 0; g < G.lambda.size(); ++g) {
        if ((st = system_at(ctx, sys, G.lambda[g], sg[g], surf[g])) != RW_OK) return st;
        if ((st = pack_system(ctx, &sg[g], P[g])) != RW_OK) return st;
        if ((st = pack_jobs(ctx, &sg[g], G.jobs[g].data(), (int)G.jobs[g].size(), rays->n, P[g],
                            G.out[g].data())) != RW_OK)
            return st;
        if (P[g].sys.M > 96 || backward_smem_needed(P[g].sys) > (size_t)lim)
            return fail(ctx, RW_EINVAL, "patch size / n_ssr too large for the fused adjoint's "
                                        "shared memory");
        total += P[g].total;
    }
    if (total == 0 || (!dphi && !damp && !dsurf)) return RW_OK;
    RW_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    const bool coherent = P[0].sys.coherent != 0;
    const long long npx = (long long)P[0].sys.nx * P[0].sys.ny * njob;
    float2* gfield = nullptr;
    EmitOut eo;
    std::memset(&eo, 0, sizeof(eo));
    if (coherent) {
        // the whole field of every job first, then dL/dU = 2 (dL/dI) U
        if ((st = ensure_buf(ctx, ctx->field, npx * sizeof(float2), "coherent field scratch")) !=
            RW_OK)
            return st;
        gfield = (float2*)ctx->field.p;
        RW_CUDA(cudaMemsetAsync(gfield, 0, npx * sizeof(float2), ctx->stream), "field clear");
        for (size_t g = 0; g < G.lambda.size(); ++g) {
            if (P[g].total == 0) continue;
            float2* T; DJob* dj; long long* dp;
            if ((st = prepare(ctx, &sg[g], P[g], &T, &dj, &dp)) != RW_OK) return st;
            RW_CUDA(launch_forward(lctx(ctx), MODE_COHERENT, P[g].sys, dj, dp,
                                   (int)G.jobs[g].size(), P[g].total, rays_in(rays), T, nullptr,
                                   gfield, eo, status_word(ctx)), "coherent field");
            ctx->launches++;
        }
        RW_CUDA(launch_coherent_grad(lctx(ctx), gfield, dl_dpsf, npx), "field gradient");
        ctx->launches++;
    }
    for (size_t g = 0; g < G.lambda.size(); ++g) {
        if (P[g].total == 0) continue;
        float2* T; DJob* dj; long long* dp;
        if ((st = prepare(ctx, &sg[g], P[g], &T, &dj, &dp)) != RW_OK) return st;
        const int nj = (int)G.jobs[g].size();
        float* coh_rsum = nullptr;
        double* coh_jsum = nullptr;
        if (coherent) {
            if ((st = ensure_buf(ctx, ctx->coh_rsum, (size_t)P[g].total * P[g].sys.nrs * sizeof(float),
                                 "coherent adjoint scratch")) != RW_OK)
                return st;
            if ((st = ensure_buf(ctx, ctx->coh_jsum, (size_t)nj * 2 * sizeof(double),
                                 "coherent adjoint scratch")) != RW_OK)
                return st;
            coh_rsum = (float*)ctx->coh_rsum.p;
            coh_jsum = (double*)ctx->coh_jsum.p;
            RW_CUDA(cudaMemsetAsync(coh_jsum, 0, (size_t)nj * 2 * sizeof(double), ctx->stream),
                    "job sums clear");
            RW_CUDA(cudaMemsetAsync(coh_rsum, 0, (size_t)P[g].total * P[g].sys.nrs * sizeof(float),
                                    ctx->stream), "ray sums clear");
        }
        int nl = 0;
        RW_CUDA(launch_backward(lctx(ctx), P[g].sys, dj, dp, nj, P[g].total, rays_in(rays), T,
                                sys->doe.amp, dl_dpsf, gfield, coh_rsum, coh_jsum, dphi, damp,
                                dsurf, nullptr, status_word(ctx), &nl),
                "backward kernel");
        ctx->launches += nl;
    }
    return RW_OK;
}

rw_status rw_backward(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs, int32_t njob,
                      const rw_rays* rays, const float* dl_dpsf, float* dphi, float* damp,
                      double* dsurf) {
    return backward_impl(ctx, sys, jobs, njob, rays, dl_dpsf, nullptr, 0, dphi, damp, dsurf);
}

rw_status rw_backward_vis(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs, int32_t njob,
                          const rw_rays* rays, const float* dl_dpsf, const uint32_t* vis,
                          int64_t vis_words, float* dphi, float* damp, double* dsurf) {
    if (!vis) return fail(ctx, RW_EINVAL, "vis is NULL");
    return backward_impl(ctx, sys, jobs, njob, rays, dl_dpsf, vis, vis_words, dphi, damp, dsurf);
}

// ---------------------------------------------------------------- autotuning (A10)
static int kernel_kind(const std::string& name) {
    if (name == "k_forward") return RW_K_FORWARD;
    if (name == "k_cull") return RW_K_CULL;
    if (name == "k_bs_spectra") return RW_K_BS_SPECTRA;
    if (name == "k_bs_trace") return RW_K_BS_TRACE;
    if (name == "k_bs_scatter") return RW_K_BS_SCATTER;
    if (name == "k_backward") return RW_K_BACKWARD;
    if (name == "k_spectra_fft" || name == "k_spectra_tc") return RW_K_SPECTRA;
    return -1;
}

rw_status rw_autotune(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs, int32_t njob,
                      const rw_rays* rays, float* psf, const float* dl_dpsf, uint32_t* vis,
                      int64_t vis_words, float* dphi, double* dsurf, int64_t* grids_out) {
    if (!ctx) return RW_EINVAL;
    if (!grids_out) return fail(ctx, RW_EINVAL, "grids_out is NULL");
    if (capturing(ctx)) return fail(ctx, RW_EINVAL, "rw_autotune cannot run during capture");
    const bool prof_was = ctx->prof_on;
    auto step = [&]() -> rw_status {
        rw_status st = forward_impl(ctx, sys, jobs, njob, rays, psf, vis, vis_words);
        if (st != RW_OK || !dl_dpsf) return st;
        return backward_impl(ctx, sys, jobs, njob, rays, dl_dpsf, vis, vis_words, dphi, nullptr,
                             dsurf);
    };
    for (int k = 0; k < RW_NK; ++k) ctx->grid[k] = 0;
    rw_status st = step();                                   // warm-up: sizes every buffer
    if (st != RW_OK) return st;
    // candidates: the occupancy default (0), then 1, 2, 3, 4, 6, 8 CTAs per SM
    const int mult[7] = {0, 1, 2, 3, 4, 6, 8};
    double best_ms[RW_NK];
    long long best[RW_NK];
    for (int k = 0; k < RW_NK; ++k) { best_ms[k] = -1.0; best[k] = 0; }
    for (int c = 0; c < 7; ++c) {
        for (int k = 0; k < RW_NK; ++k) ctx->grid[k] = (long long)mult[c] * ctx->num_sms;
        if ((st = rw_profile(ctx, 1)) != RW_OK) break;
        if ((st = step()) != RW_OK) break;
        int32_t n = 0;
        if ((st = rw_profile_read(ctx, &n)) != RW_OK) break;
        for (int i = 0; i < n; ++i) {
            const int k = kernel_kind(ctx->prof_kernels[i]);
            if (k < 0 || ctx->prof_count[i] == 0) continue;
            const double ms = ctx->prof_ms[i] / (double)ctx->prof_count[i];
            if (best_ms[k] < 0.0 || ms < best_ms[k]) { best_ms[k] = ms; best[k] = ctx->grid[k]; }
        }
    }
    ctx->prof_on = prof_was;
    ctx->prof_used = 0;
    for (int k = 0; k < RW_NK; ++k) {
        ctx->grid[k] = (st == RW_OK) ? best[k] : 0;
        grids_out[k] = ctx->grid[k];
    }
    return st;
}

rw_status rw_probe_red(rw_ctx* ctx, float* map, int32_t H, int32_t W, int32_t win,
                       int64_t nwin) {
    if (!ctx) return RW_EINVAL;
    ctx->err.clear();
    if (!map) return fail(ctx, RW_EINVAL, "map is NULL");
    if (H < 1 || W < 1 || win < 1 || win > H || win > W || nwin < 0)
        return fail(ctx, RW_EINVAL, "need 1 <= win <= H, W and nwin >= 0");
    if (nwin == 0) return RW_OK;
    RW_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    RW_CUDA(launch_probe_red(lctx(ctx), map, H, W, win, nwin), "reduction probe");
    ctx->launches++;
    return RW_OK;
}

rw_status rw_set_grids(rw_ctx* ctx, const int64_t* grids) {
    if (!ctx || !grids) return fail(ctx, RW_EINVAL, "null argument");
    for (int k = 0; k < RW_NK; ++k) ctx->grid[k] = grids[k] > 0 ? grids[k] : 0;
    return RW_OK;
}

rw_status rw_patch_spectra(rw_ctx* ctx, const rw_system* sys, const rw_job* jobs, int32_t njob,
                           const rw_rays* rays, float* spectra, int64_t capacity) {
    if (!ctx) return RW_EINVAL;
    ctx->err.clear();
    if (is_dispersive(sys))
        return fail(ctx, RW_EINVAL, "dispersive surfaces: rw_forward and rw_backward only");
    Packed P;
    rw_status st = pack_system(ctx, sys, P);
    if (st != RW_OK) return st;
    if ((st = check_rays(ctx, rays)) != RW_OK) return st;
    if ((st = pack_jobs(ctx, sys, jobs, njob, rays->n, P)) != RW_OK) return st;
    if (!spectra) return fail(ctx, RW_EINVAL, "spectra is NULL");
    const int tc = sys->doe.dft == RW_DFT_TC;
    if (tc && (P.sys.D != 64 || P.sys.M != 64))
        return fail(ctx, RW_EINVAL, "the tensor-core patch transform supports D = 64 without padding");
    if (capacity < P.total * (int64_t)P.sys.M * P.sys.M)
        return fail(ctx, RW_ECAPACITY, "spectra capacity < n_rays * M * M");
    if (P.total == 0) return RW_OK;
    float2* T; DJob* dj; long long* dp;
    if ((st = prepare(ctx, sys, P, &T, &dj, &dp)) != RW_OK) return st;
    RW_CUDA(launch_spectra(lctx(ctx), P.sys, tc, dj, dp, njob, P.total, rays_in(rays), T,
                           (float2*)spectra, status_word(ctx)),
            "spectra kernel");
    ctx->launches++;
    return RW_OK;
}

}  // extern "C"
