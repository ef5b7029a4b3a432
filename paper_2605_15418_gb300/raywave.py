"""Python binding of librw.so with the C-ABI names (argument marshalling only).

Every step of the ray-wave path runs in the library's CUDA kernels; torch
is used for device memory and the current CUDA stream.  Host descriptors
come from `rwinputs` dataclasses (Surface, DOE, Sensor, System, Job).
"""
import ctypes as C
import math

import numpy as np
import torch

from . import _capi as A

_GATHER = {"nearest": A.RW_GATHER_NEAREST, "bilinear": A.RW_GATHER_BILINEAR}
_EMIT = {"exhaustive": A.RW_EMIT_EXHAUSTIVE, "sampled": A.RW_EMIT_SAMPLED,
         "sampled_uniform": A.RW_EMIT_SAMPLED_UNIFORM}
_PHASE = {"height": A.RW_PHASE_HEIGHT, "fixed": A.RW_PHASE_FIXED}
_DFT = {"fft32": A.RW_DFT_FFT32, "tc": A.RW_DFT_TC}
RAY_FIELDS = ("ox", "oy", "oz", "dx", "dy", "dz", "a_re", "a_im")


class RayWaveError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{A.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return C.c_void_p(t.data_ptr())


class Context:
    """One librw context on one CUDA device; calls follow torch's current stream."""

    def __init__(self, device=0):
        self.lib = A.load()
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        idx = self.device.index if self.device.index is not None else 0
        self.h = C.c_void_p()
        st = self.lib.rw_create(C.byref(self.h), idx, None)
        if st != A.RW_OK:
            raise RayWaveError(st, "rw_create failed")

    def _stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        self.lib.rw_set_stream(self.h, C.c_void_p(s))

    def check(self, st, what):
        if st != A.RW_OK:
            raise RayWaveError(st, f"{what}: {self.lib.rw_last_error(self.h).decode()}")

    @property
    def launches(self):
        return int(self.lib.rw_launch_count(self.h))

    def profile(self, enable=True):
        """Start (clearing the totals) or stop per-launch CUDA-event timing."""
        self._stream()
        self.check(self.lib.rw_profile(self.h, 1 if enable else 0), "rw_profile")

    def profile_read(self):
        """{kernel: (total ms, launches)} since profile() was last called."""
        self._stream()
        n = C.c_int32(0)
        self.check(self.lib.rw_profile_read(self.h, C.byref(n)), "rw_profile_read")
        out = {}
        for i in range(n.value):
            name, ms, cnt = C.c_char_p(), C.c_double(), C.c_int64()
            self.check(self.lib.rw_profile_entry(self.h, i, C.byref(name), C.byref(ms),
                                                 C.byref(cnt)), "rw_profile_entry")
            out[name.value.decode()] = (ms.value, cnt.value)
        return out

    def autotune(self, sim, dl_dpsf=None, vis=None):
        """Tune the persistent grid of every kernel on `sim`'s workload (one
        forward with `vis`, plus the adjoint when dl_dpsf is given, per
        candidate grid); returns {kernel: grid} (0 = occupancy default)."""
        self._stream()
        s, keep = sim.sys_struct()
        rs = rays_struct(sim.rays)
        psf = torch.empty(sim.psf_shape, dtype=torch.float32, device=sim.dev)
        dphi = torch.zeros_like(sim.phi)
        dsurf = torch.zeros(len(sim.w.system.surfaces), 8, dtype=torch.float64, device=sim.dev)
        out = (C.c_int64 * len(A.KERNEL_KINDS))()
        self.check(self.lib.rw_autotune(self.h, C.byref(s), sim.jobs, len(sim.jobs), C.byref(rs),
                                        _ptr(psf), _ptr(dl_dpsf), _ptr(vis),
                                        0 if vis is None else vis.numel(), _ptr(dphi),
                                        _ptr(dsurf), out), "rw_autotune")
        return dict(zip(A.KERNEL_KINDS, [int(v) for v in out]))

    def set_grids(self, grids):
        """Per-kernel grids ({kernel: grid}, missing or 0 = occupancy default)."""
        arr = (C.c_int64 * len(A.KERNEL_KINDS))(*[int(grids.get(k, 0)) for k in A.KERNEL_KINDS])
        self.check(self.lib.rw_set_grids(self.h, arr), "rw_set_grids")

    def probe_red(self, map2d, win, nwin):
        """Enqueue win*win*nwin float atomic adds onto map2d (device float
        [H][W]) in the pattern of the adjoint's map scatter (rw_probe_red)."""
        H, W = map2d.shape
        self.check(self.lib.rw_probe_red(self.h, map2d.data_ptr(), H, W, win, nwin),
                   "rw_probe_red")

    def cull_stats(self):
        """(8 x 8 bin blocks, blocks kept) of the last culled forward."""
        self._stream()
        b, k = C.c_int64(), C.c_int64()
        self.check(self.lib.rw_cull_stats(self.h, C.byref(b), C.byref(k)), "rw_cull_stats")
        return int(b.value), int(k.value)

    def device_status(self):
        self._stream()
        v = C.c_uint32(0)
        self.check(self.lib.rw_device_status(self.h, C.byref(v)), "rw_device_status")
        return int(v.value)

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.rw_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ marshalling
def surfaces_struct(surfaces):
    arr = (A.rw_surface * len(surfaces))()
    for i, s in enumerate(surfaces):
        arr[i].kind = int(s.kind)
        arr[i].z = float(s.z)
        arr[i].c = float(s.c)
        arr[i].k = float(s.k)
        arr[i].A4, arr[i].A6, arr[i].A8, arr[i].A10 = (float(a) for a in s.A)
        arr[i].n_after = float(s.n_after)
        arr[i].r_ap = float(s.r_ap)
        sm = getattr(s, "sellmeier", None)
        if sm is not None:
            for k in range(6):
                arr[i].sellmeier[k] = float(sm[k])
    return arr


def system_struct(system, phi, amp=None, dft="fft32", surfaces=None, trace_all=False):
    """rw_system for `system` with device maps phi (and amp).  A DOE with two
    phase profiles takes phi as one contiguous [2, H, W] tensor (phi, phi2).
    Returns (struct, keepalive)."""
    doe = system.doe
    surfs = surfaces_struct(surfaces if surfaces is not None else system.surfaces)
    s = A.rw_system()
    s.surfaces = C.cast(surfs, C.POINTER(A.rw_surface))
    s.nsurf = len(surfs)
    s.doe_index = int(system.doe_index)
    s.n_object = float(system.n_object)
    H, W = phi.shape[-2:]
    s.doe.H, s.doe.W = int(H), int(W)
    s.doe.pitch = float(doe.pitch)
    s.doe.lambda0 = float(doe.lambda0)
    if phi.dim() == 3:
        if phi.shape[0] != 2 or not phi.is_contiguous():
            raise ValueError("two phase profiles: phi must be a contiguous [2, H, W] tensor")
        s.doe.phi = _ptr(phi[0])
        s.doe.phi2 = _ptr(phi[1])
    else:
        s.doe.phi = _ptr(phi)
    s.doe.amp = _ptr(amp)
    s.doe.D = int(doe.D)
    s.doe.gather = _GATHER[doe.gather]
    s.doe.emit = _EMIT[doe.emit]
    s.doe.n_ssr = int(doe.n_ssr)
    s.doe.phase_model = _PHASE[doe.phase_model]
    s.doe.dft = _DFT[dft]
    s.doe.seed = int(doe.seed)
    s.doe.rng_offset = int(doe.rng_offset)
    s.doe.pad = int(getattr(doe, "pad", 1))
    s.doe.flags = ((A.RW_DOE_TRACE_ALL if trace_all else 0)
                   | (A.RW_DOE_REFLECTIVE if getattr(doe, "reflective", False) else 0))
    sen = system.sensor
    s.sensor.z = float(sen.z)
    s.sensor.nx, s.sensor.ny = int(sen.nx), int(sen.ny)
    s.sensor.pitch = float(sen.pitch)
    s.sensor.coherent = 1 if sen.coherent else 0
    s.sensor.window = int(sen.window)
    return s, (surfs, phi, amp)


def jobs_struct(jobs, offsets=None, counts=None):
    """rw_job array; rays of job i are [offsets[i], offsets[i] + counts[i])."""
    arr = (A.rw_job * len(jobs))()
    off = 0
    for i, j in enumerate(jobs):
        cnt = j.n_rays if counts is None else int(counts[i])
        o = off if offsets is None else int(offsets[i])
        arr[i].lambda_ = float(j.lam)
        arr[i].theta_x = float(j.theta_x)
        arr[i].theta_y = float(j.theta_y)
        arr[i].ray_offset = o
        arr[i].ray_count = cnt
        arr[i].sensor_cx = float(j.sensor_cx)
        arr[i].sensor_cy = float(j.sensor_cy)
        arr[i].grid_n = int(j.grid_n)
        arr[i].spacing = float(j.spacing)
        arr[i].x0 = float(j.x0)
        arr[i].y0 = float(j.y0)
        off = o + cnt
    return arr


def alloc_rays(n, device):
    r = {k: torch.empty(n, dtype=torch.float32, device=device) for k in RAY_FIELDS}
    r["opl"] = torch.empty(n, dtype=torch.float64, device=device)
    return r


def rays_struct(rays):
    s = A.rw_rays()
    s.n = int(rays["ox"].numel())
    for k in RAY_FIELDS + ("opl",):
        setattr(s, k, _ptr(rays[k]))
    return s


def alloc_emitted(n_in, slots, device, with_bin=True):
    cap = n_in * slots
    e = {k: torch.empty(cap, dtype=torch.float32, device=device)
         for k in ("dx", "dy", "dz", "a_re", "a_im")}
    e["bin"] = torch.empty(cap, dtype=torch.int32, device=device) if with_bin else None
    for k in ("hx", "hy", "hz"):
        e[k] = torch.empty(n_in, dtype=torch.float32, device=device)
    e["opl"] = torch.empty(n_in, dtype=torch.float64, device=device)
    e["capacity"] = cap
    return e


def emitted_struct(e):
    s = A.rw_emitted()
    s.capacity = int(e["capacity"])
    for k in ("dx", "dy", "dz", "a_re", "a_im", "bin", "hx", "hy", "hz", "opl"):
        setattr(s, k, _ptr(e[k]))
    return s


def device_map(arr, device):
    return torch.as_tensor(np.ascontiguousarray(arr, dtype=np.float32), device=device)


# ------------------------------------------------------------------ C-ABI calls
def rw_generate_rays(ctx, z_start, n_object, jobs_arr, rays):
    ctx._stream()
    rs = rays_struct(rays)
    ctx.check(ctx.lib.rw_generate_rays(ctx.h, float(z_start), float(n_object), jobs_arr,
                                       len(jobs_arr), C.byref(rs)), "rw_generate_rays")


def rw_doe_emit(ctx, sys_struct, jobs_arr, rays, out):
    ctx._stream()
    rs = rays_struct(rays)
    es = emitted_struct(out)
    ctx.check(ctx.lib.rw_doe_emit(ctx.h, C.byref(sys_struct), jobs_arr, len(jobs_arr),
                                  C.byref(rs), C.byref(es)), "rw_doe_emit")


def rw_forward(ctx, sys_struct, jobs_arr, rays, psf):
    ctx._stream()
    rs = rays_struct(rays)
    ctx.check(ctx.lib.rw_forward(ctx.h, C.byref(sys_struct), jobs_arr, len(jobs_arr),
                                 C.byref(rs), _ptr(psf)), "rw_forward")


def rw_forward_vis(ctx, sys_struct, jobs_arr, rays, psf, vis):
    ctx._stream()
    rs = rays_struct(rays)
    ctx.check(ctx.lib.rw_forward_vis(ctx.h, C.byref(sys_struct), jobs_arr, len(jobs_arr),
                                     C.byref(rs), _ptr(psf), _ptr(vis), int(vis.numel())),
              "rw_forward_vis")


def rw_backward_vis(ctx, sys_struct, jobs_arr, rays, dl_dpsf, vis, dphi=None, damp=None,
                    dsurf=None):
    ctx._stream()
    rs = rays_struct(rays)
    ctx.check(ctx.lib.rw_backward_vis(ctx.h, C.byref(sys_struct), jobs_arr, len(jobs_arr),
                                      C.byref(rs), _ptr(dl_dpsf), _ptr(vis), int(vis.numel()),
                                      _ptr(dphi), _ptr(damp), _ptr(dsurf)), "rw_backward_vis")


def alloc_vis(n_rays, M, device):
    """One visibility bit per secondary ray, M x M bins per incident ray
    (M = pad * D; int32 words, bit-exact uint32)."""
    return torch.empty(n_rays * M * M // 32, dtype=torch.int32, device=device)


def rw_patch_spectra(ctx, sys_struct, jobs_arr, rays, spectra):
    ctx._stream()
    rs = rays_struct(rays)
    ctx.check(ctx.lib.rw_patch_spectra(ctx.h, C.byref(sys_struct), jobs_arr, len(jobs_arr),
                                       C.byref(rs), _ptr(spectra), int(spectra.numel() // 2)),
              "rw_patch_spectra")


def rw_loss_eq3(ctx, psf, target, loss_out, dl_dpsf=None):
    ctx._stream()
    ctx.check(ctx.lib.rw_loss_eq3(ctx.h, _ptr(psf), _ptr(target), int(psf.numel()),
                                  _ptr(loss_out), _ptr(dl_dpsf)), "rw_loss_eq3")


def rw_backward(ctx, sys_struct, jobs_arr, rays, dl_dpsf, dphi=None, damp=None, dsurf=None):
    ctx._stream()
    rs = rays_struct(rays)
    ctx.check(ctx.lib.rw_backward(ctx.h, C.byref(sys_struct), jobs_arr, len(jobs_arr),
                                  C.byref(rs), _ptr(dl_dpsf), _ptr(dphi), _ptr(damp),
                                  _ptr(dsurf)), "rw_backward")


# ------------------------------------------------------------------ convenience
class Simulator:
    """A workload bound to a context: device maps, jobs and generated rays."""

    def __init__(self, workload, ctx=None, device=0, dft="fft32", rays=None, trace_all=False):
        self.ctx = ctx or Context(device)
        self.trace_all = trace_all
        self.w = workload
        self.dev = self.ctx.device
        sysm = workload.system
        self.phi = device_map(sysm.doe.phi, self.dev)
        if getattr(sysm.doe, "phi2", None) is not None:
            # two phase profiles: one [2, H, W] map (dL/dphi comes back the same shape)
            self.phi = torch.stack([self.phi, device_map(sysm.doe.phi2, self.dev)]).contiguous()
        self.amp = None if sysm.doe.amp is None else device_map(sysm.doe.amp, self.dev)
        self.dft = dft
        self.jobs = jobs_struct(workload.jobs)
        self.n_rays = workload.n_rays
        if rays is None:
            rays = alloc_rays(self.n_rays, self.dev)
            rw_generate_rays(self.ctx, workload.z_start, sysm.n_object, self.jobs, rays)
        self.rays = rays
        sen = sysm.sensor
        self.psf_shape = (len(workload.jobs), sen.ny, sen.nx)

    def sys_struct(self, phi=None, amp=None, surfaces=None):
        return system_struct(self.w.system, self.phi if phi is None else phi,
                             self.amp if amp is None else amp, self.dft, surfaces,
                             self.trace_all)

    def forward(self, phi=None, surfaces=None, psf=None, vis=None):
        """PSF [njob, ny, nx]; with `vis` (alloc_vis) also the visibility mask."""
        s, keep = self.sys_struct(phi, surfaces=surfaces)
        if psf is None:
            psf = torch.empty(self.psf_shape, dtype=torch.float32, device=self.dev)
        if vis is None:
            rw_forward(self.ctx, s, self.jobs, self.rays, psf)
        else:
            rw_forward_vis(self.ctx, s, self.jobs, self.rays, psf, vis)
        return psf

    def emit(self, out=None):
        sysm = self.w.system
        slots = sysm.doe.M ** 2 if sysm.doe.emit == "exhaustive" else sysm.doe.n_ssr
        if out is None:
            out = alloc_emitted(self.n_rays, slots, self.dev)
        s, keep = self.sys_struct()
        rw_doe_emit(self.ctx, s, self.jobs, self.rays, out)
        return out

    def spectra(self, dft=None, out=None):
        """Patch spectra U~ [n_rays, M, M] (complex64) with the FFT or tensor cores."""
        M = self.w.system.doe.M
        if out is None:
            out = torch.empty(self.n_rays, M, M, 2, dtype=torch.float32, device=self.dev)
        s, keep = system_struct(self.w.system, self.phi, self.amp, dft or self.dft)
        rw_patch_spectra(self.ctx, s, self.jobs, self.rays, out)
        return torch.view_as_complex(out)

    def backward(self, dl_dpsf, phi=None, surfaces=None, want_amp=False, vis=None):
        """(dphi, damp, dsurf); `vis` from forward(vis=...) on the same inputs
        restricts the adjoint to secondary rays that reached the sensor."""
        s, keep = self.sys_struct(phi, surfaces=surfaces)
        dphi = torch.zeros_like(self.phi)
        damp = torch.zeros_like(self.amp) if (want_amp and self.amp is not None) else None
        dsurf = torch.zeros(len(self.w.system.surfaces), 8, dtype=torch.float64, device=self.dev)
        if vis is None:
            rw_backward(self.ctx, s, self.jobs, self.rays, dl_dpsf.contiguous(), dphi, damp,
                        dsurf)
        else:
            rw_backward_vis(self.ctx, s, self.jobs, self.rays, dl_dpsf.contiguous(), vis, dphi,
                            damp, dsurf)
        return dphi, damp, dsurf

    def loss(self, psf, target, dl_dpsf=None):
        out = torch.empty(3, dtype=torch.float64, device=self.dev)
        rw_loss_eq3(self.ctx, psf, target, out, dl_dpsf)
        return out
