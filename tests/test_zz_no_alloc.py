"""rw_generate_rays_static: ray generation for callers that cannot allocate
device memory (e.g. a plugin whose host application owns the device memory,
or a real-time loop that cannot take cudaMalloc's implicit synchronisation).

It must produce exactly what rw_generate_rays produces, call after call,
while using only the library's fixed device array for its job table.  This
file is collected last so that a failure here leaves every other test run.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import rwinputs as R

pytestmark = pytest.mark.gpu


def _compare(RW, lib, ctx, w, stream):
    jobs = RW.jobs_struct(w.jobs)
    ref = RW.alloc_rays(w.n_rays, "cuda")
    got = RW.alloc_rays(w.n_rays, "cuda")
    for t in got.values():
        t.fill_(float("nan"))
    RW.rw_generate_rays(ctx, w.z_start, w.system.n_object, jobs, ref)
    rs = RW.rays_struct(got)
    st = lib.rw_generate_rays_static(float(w.z_start), float(w.system.n_object), jobs,
                                     len(jobs), C.byref(rs), C.c_void_p(stream))
    assert st == 0
    torch.cuda.synchronize()
    for k in ref:
        # bit-exact: same kernel arithmetic, only the job table's home differs
        assert torch.equal(ref[k], got[k]), k


def test_static_generation_matches_context_version_on_consecutive_calls():
    from paper_2605_15418_gb300 import _capi, raywave as RW
    lib = _capi.load()
    ctx = RW.Context(0)
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row with different job tables (the second shrinks the table)
    _compare(RW, lib, ctx, R.configs.c4(n_side=33, D=16, n_fields=5, map_side=64), stream)
    _compare(RW, lib, ctx, R.configs.c5(n_lams=3, n_fields=4, count_lo=100, count_hi=3000,
                                        map_side=64), stream)
    ctx.close()


def test_static_generation_rejects_too_many_jobs():
    from paper_2605_15418_gb300 import _capi, raywave as RW
    lib = _capi.load()
    jobs = (_capi.rw_job * 1025)()
    for j in jobs:
        j.lambda_ = 550e-6
        j.grid_n = 1
        j.ray_count = 1
    rays = RW.alloc_rays(4, "cuda")
    rays["ox"].fill_(7.0)
    rs = RW.rays_struct(rays)
    st = lib.rw_generate_rays_static(-1.0, 1.0, jobs, 1025, C.byref(rs), None)
    assert st == _capi.RW_ECAPACITY
    torch.cuda.synchronize()
    assert (rays["ox"] == 7.0).all()


def _many_jobs(n, side=2):
    """n small jobs of side x side rays with distinct angles and centres."""
    jobs = []
    for i in range(n):
        jobs.append(R.systems.Job(lam=550e-6, theta_x=1e-4 * (i % 37), theta_y=-2e-4 * (i % 11),
                                  grid_n=side, spacing=1e-3 * (1 + i % 5), x0=1e-3 * i,
                                  y0=-2e-3 * (i % 13)))
    return jobs


def test_static_generation_at_the_job_limit():
    # exactly 1024 jobs: the whole fixed table is used
    from paper_2605_15418_gb300 import _capi, raywave as RW
    lib = _capi.load()
    ctx = RW.Context(0)
    stream = torch.cuda.current_stream().cuda_stream
    sysm = R.configs.c3(n_side=4).system
    w = R.systems.Workload("1024 jobs", sysm, _many_jobs(1024), z_start=-1.0)
    _compare(RW, lib, ctx, w, stream)
    ctx.close()


def test_static_generation_refuses_stream_capture():
    # a captured call would replay an upload from a host buffer that later
    # calls overwrite, so the call is refused while its stream is captured
    from paper_2605_15418_gb300 import _capi, raywave as RW
    lib = _capi.load()
    w = R.configs.c3(n_side=4)
    jobs = RW.jobs_struct(w.jobs)
    rays = RW.alloc_rays(w.n_rays, "cuda")
    rays["ox"].fill_(7.0)
    rs = RW.rays_struct(rays)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    marker = torch.zeros(1, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        marker.add_(1.0)
        st = lib.rw_generate_rays_static(float(w.z_start), 1.0, jobs, len(jobs), C.byref(rs),
                                         C.c_void_p(s.cuda_stream))
    assert st == _capi.RW_EINVAL
    g.replay()
    torch.cuda.synchronize()
    assert float(marker.item()) == 1.0
    assert (rays["ox"] == 7.0).all()
    # and the next eager call on the same stream works
    st = lib.rw_generate_rays_static(float(w.z_start), 1.0, jobs, len(jobs), C.byref(rs),
                                     C.c_void_p(s.cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    assert not (rays["ox"] == 7.0).all()
