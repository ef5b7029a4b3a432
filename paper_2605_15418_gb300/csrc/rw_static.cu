// Allocation-free variant of ray generation (A0).
//
// rw_generate_rays() keeps its job table in per-context device scratch,
// which rw_create() allocates.  Callers that cannot call cudaMalloc -- a
// plugin whose host application owns all device memory through its own
// allocator, or a real-time loop that cannot afford cudaMalloc's implicit
// device synchronisation -- use rw_generate_rays_static() instead: its job
// table lives in the file-scope device array below, so the call needs no
// context and allocates nothing.
#include <cmath>
#include <cstring>
#include <mutex>

#include "rw_kernels.cuh"

#define RW_STATIC_MAX_JOBS 1024

// Job table + prefix sums for at most RW_STATIC_MAX_JOBS jobs.  Every GPU
// that loads the library holds this array until the process exits.
#define RW_STATIC_TABLE_BYTES \
    (sizeof(GenJob) * RW_STATIC_MAX_JOBS + sizeof(long long) * (RW_STATIC_MAX_JOBS + 1))
static __device__ __align__(256) unsigned char g_static_gen_table[RW_STATIC_TABLE_BYTES];

#define RW_STATIC_MAX_DEVICES 64
static void* g_table_addr[RW_STATIC_MAX_DEVICES];   // device address per device
static std::mutex g_table_mu;

// Device address of g_static_gen_table on the current device.  In host code
// the symbol names a host-side stand-in, so the kernel is given the address
// that cudaGetSymbolAddress returns (looked up once per device, with that
// device current).
static cudaError_t table_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= RW_STATIC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_table_mu);
    if (!g_table_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_gen_table);
        if (e != cudaSuccess) return e;
        g_table_addr[dev] = p;
    }
    *out = g_table_addr[dev];
    return cudaSuccess;
}

extern "C" rw_status rw_generate_rays_static(double z_start, double n_object,
                                             const rw_job* jobs, int32_t njob,
                                             rw_rays* rays, void* cuda_stream) {
    if (!jobs || !rays || njob < 1) return RW_EINVAL;
    if (njob > RW_STATIC_MAX_JOBS) return RW_ECAPACITY;
    if (!(n_object > 0) || rays->n < 0) return RW_EINVAL;
    if (rays->n > 0 && (!rays->ox || !rays->oy || !rays->oz || !rays->dx || !rays->dy ||
                        !rays->dz || !rays->a_re || !rays->a_im || !rays->opl))
        return RW_EINVAL;
    // host copy of the table (stack, no allocation), then one async copy
    unsigned char host[RW_STATIC_TABLE_BYTES];
    GenJob* g = reinterpret_cast<GenJob*>(host);
    long long* prefix = reinterpret_cast<long long*>(host + sizeof(GenJob) * RW_STATIC_MAX_JOBS);
    prefix[0] = 0;
    for (int i = 0; i < njob; ++i) {
        const rw_job& j = jobs[i];
        if (j.grid_n < 0 || j.ray_count != j.grid_n * j.grid_n) return RW_EINVAL;
        if (j.ray_offset < 0 || j.ray_offset + j.ray_count > rays->n) return RW_EINVAL;
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
    if (prefix[njob] == 0) return RW_OK;
    void* dev_table = nullptr;
    if (table_address(&dev_table) != cudaSuccess) return RW_ECUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // Every call rewrites the whole table it uses; nothing has to start at zero.
    if (cudaMemcpyAsync(dev_table, host, sizeof(GenJob) * njob, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return RW_ECUDA;
    char* dprefix = (char*)dev_table + sizeof(GenJob) * RW_STATIC_MAX_JOBS;
    if (cudaMemcpyAsync(dprefix, prefix, sizeof(long long) * (njob + 1), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
        return RW_ECUDA;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    LaunchCtx L;
    L.stream = st;
    L.num_sms = sms > 0 ? sms : 1;
    L.grid_override = 0;
    for (int k = 0; k < RW_NK; ++k) L.grid[k] = 0;
    L.prof = nullptr;
    RaysOut o;
    o.ox = rays->ox; o.oy = rays->oy; o.oz = rays->oz; o.dx = rays->dx; o.dy = rays->dy;
    o.dz = rays->dz; o.are = rays->a_re; o.aim = rays->a_im; o.opl = rays->opl;
    if (launch_generate_rays(L, (const GenJob*)dev_table, (const long long*)dprefix, njob,
                             prefix[njob], z_start, n_object, o) != cudaSuccess)
        return RW_ECUDA;
    return RW_OK;
}
