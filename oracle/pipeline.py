"""End-to-end oracle: rays -> pre-DOE trace -> DOE step -> post-DOE trace
-> sensor, per job, float64, chunked over incident rays.

Chunking only bounds memory: every incident ray's contribution is computed
independently and the per-chunk images are added.
"""
import math

import numpy as np
import torch

from . import geometry as G
from . import doe as DO
from . import sensor as S


def job_rays(job, z_start, n_object=1.0, idx=None):
    """Collimated grid of one job (see rwinputs.Job).  Ray inputs are float32
    quantities: positions are formed in double, x0 + (ix - (n-1)/2) spacing,
    and rounded once to float32, the direction normalise(tan tx, tan ty, 1)
    likewise; everything after that is float64.  a = 1, OPL = n_object (d . o).
    `idx` selects a subset of ray indices."""
    n = job.grid_n
    if idx is None:
        idx = np.arange(n * n)
    idx = torch.as_tensor(np.asarray(idx, dtype=np.int64))
    ix = (idx % n).to(torch.float64)
    iy = (idx // n).to(torch.float64)
    half = (n - 1) * 0.5
    x = (job.x0 + (ix - half) * job.spacing).to(torch.float32).to(torch.float64)
    y = (job.y0 + (iy - half) * job.spacing).to(torch.float32).to(torch.float64)
    z = torch.full_like(x, float(np.float32(z_start)))
    tx, ty = math.tan(job.theta_x), math.tan(job.theta_y)
    nrm = math.sqrt(tx * tx + ty * ty + 1.0)
    dv = torch.tensor([float(np.float32(tx / nrm)), float(np.float32(ty / nrm)),
                       float(np.float32(1.0 / nrm))], dtype=torch.float64)
    o = torch.stack([x, y, z], -1)
    d = dv[None, :].expand_as(o).clone()
    N = o.shape[0]
    return {"o": o, "d": d, "a": torch.ones(N, dtype=torch.complex128),
            "opl": n_object * (o * d).sum(-1), "alive": torch.ones(N, dtype=torch.bool)}


def params_of(system, requires_grad=False):
    return [G.surface_params(s, requires_grad) for s in system.surfaces]


def map_tensors(system, phi=None, amp=None):
    doe = system.doe
    if phi is None:
        phi = torch.from_numpy(np.asarray(doe.phi, dtype=np.float64))
    if amp is None and doe.amp is not None:
        amp = torch.from_numpy(np.asarray(doe.amp, dtype=np.float64))
    return phi, amp


def phi2_tensor(system, phi2=None):
    """The second phase map (float64) or None."""
    if phi2 is None and getattr(system.doe, "phi2", None) is not None:
        phi2 = torch.from_numpy(np.asarray(system.doe.phi2, dtype=np.float64))
    return phi2


def emit_job(system, job, z_start, params, phi, amp, idx=None, ray_base=0, phi2=None,
             rays=None):
    """Pre-DOE trace + DOE step for (a subset of) one job's rays.  Returns
    the DOE step and the index of the medium the secondary rays enter.
    `rays` (dict of o, d, a, opl, alive) replaces the job's collimated grid,
    e.g. the secondary rays of another DOE."""
    di = system.doe_index
    if rays is None:
        ray = job_rays(job, z_start, system.n_object, idx)
    else:
        sel = np.arange(rays["o"].shape[0]) if idx is None else np.asarray(idx)
        ray = {k: v[sel] for k, v in rays.items()}
    ray, n_in = G.trace(ray, params[:di], torch.tensor(system.n_object, dtype=torch.float64))
    # a reflective DOE sends the secondary rays back into the incident medium
    n_out = n_in if getattr(system.doe, "reflective", False) else params[di]["n_after"]
    ids = (np.arange(job.n_rays) if idx is None else np.asarray(idx)) + ray_base
    return DO.doe_step(ray, params[di], system.doe, phi, amp, job.lam, n_in, n_out,
                       ray_ids=ids, coherent=system.sensor.coherent, phi2=phi2), n_out


def psf_job(system, job, z_start, params, phi, amp, idx=None, ray_base=0, chunk=256,
            phi2=None, rays=None):
    """Sensor image [ny, nx] of one job (intensity); `rays` as in emit_job."""
    sen = system.sensor
    di = system.doe_index
    nx, ny = sen.nx, sen.ny
    n_all = job.n_rays if rays is None else int(rays["o"].shape[0])
    n_rays = n_all if idx is None else len(idx)
    all_idx = np.arange(n_all) if idx is None else np.asarray(idx)
    img = torch.zeros(nx * ny, dtype=torch.float64)
    field = torch.zeros(nx * ny, dtype=torch.complex128)
    for c0 in range(0, n_rays, chunk):
        sub = all_idx[c0:c0 + chunk]
        em, n_out = emit_job(system, job, z_start, params, phi, amp, sub, ray_base, phi2, rays)
        dsec = em["d"]
        shp = dsec.shape[:-1]
        Nin = shp[0]
        nsec = int(np.prod(shp[1:]))
        o = em["o"][:, None, :].expand(Nin, nsec, 3).reshape(-1, 3)
        ray = {"o": o, "d": dsec.reshape(-1, 3), "a": em["a"].reshape(-1),
               "opl": em["opl"][:, None].expand(Nin, nsec).reshape(-1),
               "alive": em["alive"].reshape(-1)}
        ray, n_s = G.trace(ray, params[di + 1:], n_out)
        x, y, opl = S.to_sensor(ray["o"], ray["d"], ray["opl"], sen.z, n_s)
        if sen.coherent:
            field = field + S.coherent_field(x, y, opl, ray["d"], ray["a"], ray["alive"],
                                             nx, ny, sen.pitch, job.sensor_cx,
                                             job.sensor_cy, job.lam, n_s, sen.window)
        else:
            w = ray["a"].real ** 2 + ray["a"].imag ** 2
            img = img + S.splat_incoherent(x, y, w, ray["alive"], nx, ny, sen.pitch,
                                           job.sensor_cx, job.sensor_cy)
    if sen.coherent:
        img = field.real ** 2 + field.imag ** 2
    return img.reshape(ny, nx)


def psf(workload, params=None, phi=None, amp=None, subsets=None, chunk=256, phi2=None,
        ray_bases=None):
    """PSF stack [njob, ny, nx].  subsets[j] optionally lists ray indices of job j.
    Ray i of job j has id ray_bases[j] + i in the sampling stream (default: the
    rays of all jobs numbered consecutively in job order)."""
    system = workload.system
    if params is None:
        params = params_of(system)
    phi, amp = map_tensors(system, phi, amp)
    phi2 = phi2_tensor(system, phi2)
    out = []
    base = 0
    for j, job in enumerate(workload.jobs):
        idx = None if subsets is None else subsets[j]
        pj = G.at_wavelength(params, job.lam)          # Sellmeier media at this job's lambda
        b0 = base if ray_bases is None else int(ray_bases[j])
        out.append(psf_job(system, job, workload.z_start, pj, phi, amp, idx, b0, chunk,
                           phi2))
        base += job.n_rays
    return torch.stack(out, 0)
