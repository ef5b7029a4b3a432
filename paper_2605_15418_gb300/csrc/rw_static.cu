// Allocation-free variant of ray generation (A0).
//
// rw_generate_rays() keeps its job table in per-context device scratch,
// which rw_create() allocates.  Callers that cannot call cudaMalloc -- a
// plugin whose host application owns all device memory through its own
// allocator, or a real-time loop that cannot afford cudaMalloc's implicit
// device synchronisation -- use rw_generate_rays_static() instead: its job
// table lives in the file-scope device array below, so the call needs no
// context and allocates nothing.
#include <cstring>
#include <mutex>

#include "rw_kernels.cuh"

#define RW_STATIC_MAX_JOBS 1024

// Job table + prefix sums for at most RW_STATIC_MAX_JOBS jobs.  Every GPU
// that loads the library holds this array until the process exits.
#define RW_STATIC_PREFIX_OFF (sizeof(GenJob) * RW_STATIC_MAX_JOBS)
#define RW_STATIC_TABLE_BYTES (RW_STATIC_PREFIX_OFF + sizeof(long long) * (RW_STATIC_MAX_JOBS + 1))
static __device__ __align__(256) unsigned char g_static_gen_table[RW_STATIC_TABLE_BYTES];

// Host copy of the table, built under the mutex and copied from while it is
// held (a copy from pageable memory has read its source when the call
// returns).  A static buffer rather than a stack array: the callers this
// entry point serves often run on threads with small stacks.
static unsigned char g_host_table[RW_STATIC_TABLE_BYTES];
static std::mutex g_table_mu;

extern "C" rw_status rw_generate_rays_static(double z_start, double n_object,
                                             const rw_job* jobs, int32_t njob,
                                             rw_rays* rays, void* cuda_stream) {
    if (!jobs || !rays || njob < 1) return RW_EINVAL;
    if (njob > RW_STATIC_MAX_JOBS) return RW_ECAPACITY;
    if (!(n_object > 0) || rays->n < 0) return RW_EINVAL;
    if (rays->n > 0 && (!rays->ox || !rays->oy || !rays->oz || !rays->dx || !rays->dy ||
                        !rays->dz || !rays->a_re || !rays->a_im || !rays->opl))
        return RW_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // A captured graph would replay the upload from the host buffer, whose
    // contents belong to whichever call came last: refuse capture.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return RW_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) return RW_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RW_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RW_ECUDA;
    // In host code the array's name is a host-side stand-in: the kernel gets
    // the device address, looked up on every call with the device current
    // (cheap, and never stale after a device reset).
    void* dev_table = nullptr;
    if (cudaGetSymbolAddress(&dev_table, g_static_gen_table) != cudaSuccess) return RW_ECUDA;

    std::lock_guard<std::mutex> lock(g_table_mu);
    GenJob* g = reinterpret_cast<GenJob*>(g_host_table);
    long long* prefix = reinterpret_cast<long long*>(g_host_table + RW_STATIC_PREFIX_OFF);
    if (gen_table_fill(jobs, njob, rays->n, g, prefix)) return RW_EINVAL;
    if (prefix[njob] == 0) return RW_OK;
    // Every call rewrites the part of the table it uses; nothing has to start at zero.
    if (cudaMemcpyAsync(dev_table, g, sizeof(GenJob) * njob, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return RW_ECUDA;
    char* dprefix = (char*)dev_table + RW_STATIC_PREFIX_OFF;
    if (cudaMemcpyAsync(dprefix, prefix, sizeof(long long) * (njob + 1), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
        return RW_ECUDA;
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
