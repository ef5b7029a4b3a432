"""Sellmeier dispersion on the GPU against the FP64 oracle: the BK7 singlets
of the C2 system follow N-BK7's Sellmeier formula, so every wavelength has
its own indices (the library runs one launch per wavelength).  Forward
(exhaustive and sampled, incoherent and coherent), adjoint (dL/dphi and
surface gradients, the index slot being the derivative for a shift common to
all wavelengths), invariance to the order of the job table, the chromatic
spread at the sensor, and the calls that refuse dispersive media."""
import numpy as np
import pytest
import torch

import coherent_cases as CC
import rwinputs as R
from oracle import loss as OL
from oracle import pipeline as OP

from gpu_helpers import oracle_psf, rel_l2

pytestmark = pytest.mark.gpu

LAMS = (486.1327e-6, 587.5618e-6, 656.2725e-6)


@pytest.fixture(scope="module")
def RW():
    from paper_2605_15418_gb300 import raywave
    return raywave


@pytest.fixture(scope="module")
def ctx(RW):
    c = RW.Context(0)
    yield c
    c.close()


def _c2_dispersive(n_side=11, D=16, fields=(0.0, 1.0)):
    w = R.configs.c2(n_side=n_side, D=D, lams=LAMS, fields_deg=fields, sensor_n=96,
                     map_side=128)
    w.system.sensor.pitch = 8e-3
    w.system.surfaces = R.configs.dispersive(w.system.surfaces)
    assert sum(s.sellmeier is not None for s in w.system.surfaces) == 2
    w.target = R.gaussian_spots_target(len(w.jobs), 96, 96, seed=3)
    return w


def test_dispersive_forward_matches_oracle(RW, ctx):
    w = _c2_dispersive()
    ctx.device_status()
    psf = RW.Simulator(w, ctx=ctx).forward().cpu().numpy()
    assert ctx.device_status() == 0
    ref = oracle_psf(w)
    assert rel_l2(psf, ref) <= 1e-4, rel_l2(psf, ref)
    # the blue and red images differ from the constant-index system's
    w0 = _c2_dispersive()
    w0.system.surfaces = [R.Surface(s.kind, s.z, c=s.c, k=s.k, A=s.A, n_after=s.n_after,
                                    r_ap=s.r_ap) for s in w0.system.surfaces]
    const = RW.Simulator(w0, ctx=ctx).forward().cpu().numpy()
    assert rel_l2(psf[0], const[0]) > 1e-2      # F line (n = 1.5224, not 1.5168)


def test_dispersive_result_does_not_depend_on_job_order(RW, ctx):
    """Jobs of different wavelengths interleaved (each wavelength's launch then
    writes scattered images): every job's image is the same as in the sorted
    table.  Sampled emission draws from a stream set by the ray's index in the
    ray arrays, so the interleaved sampled run equals the oracle on the
    interleaved table with each job's rays numbered from its ray offset."""
    w = _c2_dispersive()
    sim = RW.Simulator(w, ctx=ctx)
    base = sim.forward().cpu().numpy()
    order = [5, 0, 3, 1, 4, 2]
    off = R.systems.jobs_offsets(w.jobs)
    jobs = [w.jobs[i] for i in order]
    js = RW.jobs_struct(jobs, offsets=[int(off[i]) for i in order],
                        counts=[w.jobs[i].n_rays for i in order])
    s, keep = sim.sys_struct()
    out = torch.zeros(base.shape, dtype=torch.float32, device=sim.dev)
    RW.rw_forward(ctx, s, js, sim.rays, out)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), base[order]) < 1e-6
    # sampled, interleaved, against the oracle on the interleaved table
    w.system.doe.emit, w.system.doe.n_ssr, w.system.doe.seed = "sampled", 32, 77
    s, keep = sim.sys_struct()
    RW.rw_forward(ctx, s, js, sim.rays, out)
    torch.cuda.synchronize()
    w.jobs = jobs
    ref = oracle_psf(w, ray_bases=[int(off[i]) for i in order])
    assert rel_l2(out.cpu().numpy(), ref) <= 1e-3, rel_l2(out.cpu().numpy(), ref)


def test_dispersive_sampled_matches_oracle(RW, ctx):
    w = _c2_dispersive()
    w.system.doe.emit, w.system.doe.n_ssr, w.system.doe.seed = "sampled", 32, (9 << 32) | 4
    psf = RW.Simulator(w, ctx=ctx).forward().cpu().numpy()
    ref = oracle_psf(w)
    assert rel_l2(psf, ref) <= 1e-3, rel_l2(psf, ref)


def test_dispersive_adjoint_matches_oracle(RW, ctx):
    w = R.configs.c3(n_side=12, D=16)
    sysm = w.system
    sysm.surfaces = R.configs.dispersive(sysm.surfaces)
    w.jobs = [R.Job(lam=lam, grid_n=12, spacing=w.jobs[0].spacing) for lam in LAMS]
    sysm.sensor.nx = sysm.sensor.ny = 64
    sysm.sensor.pitch = 30e-3
    w.target = R.gaussian_spots_target(3, 64, 64, seed=5, n_spots=3)
    ctx.device_status()
    sim = RW.Simulator(w, ctx=ctx)
    psf = sim.forward()
    gI = torch.empty_like(psf)
    sim.loss(psf, torch.as_tensor(w.target, device=sim.dev), gI)
    dphi, _, dsurf = sim.backward(gI)
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    prm = OP.params_of(sysm, requires_grad=True)
    phi = torch.from_numpy(sysm.doe.phi.astype(np.float64)).requires_grad_(True)
    img = OP.psf(w, params=prm, phi=phi)
    assert rel_l2(psf.cpu().numpy(), img.detach().numpy()) <= 1e-4
    Lv, _ = OL.eq3_loss(img, torch.from_numpy(w.target.astype(np.float64)))
    Lv.backward()
    assert rel_l2(dphi.cpu().numpy(), phi.grad.numpy()) <= 1e-3
    ds = dsurf.cpu().numpy()
    big = max(abs(float(p[k].grad)) for p in prm for k in ("z", "c", "n_after")
              if p[k].grad is not None)
    for si in range(1, len(prm)):
        for k, name in ((0, "z"), (1, "c"), (7, "n_after")):
            ref = prm[si][name].grad
            ref = 0.0 if ref is None else float(ref)
            assert abs(ds[si, k] - ref) <= 1e-3 * abs(ref) + 1e-4 * big, (si, name, ds[si, k], ref)


def test_dispersive_coherent_forward_and_adjoint(RW, ctx):
    w = CC.lens_after(n_side=7, window=5)
    w.system.surfaces = R.configs.dispersive(w.system.surfaces)
    w.jobs = [R.Job(lam=lam, theta_y=w.jobs[0].theta_y, grid_n=7, spacing=w.jobs[0].spacing)
              for lam in (520e-6, 600e-6)]
    w.target = R.gaussian_spots_target(2, 32, 32, seed=92, n_spots=3, sigma_px=(2.0, 5.0))
    sim = RW.Simulator(w, ctx=ctx)
    psf = sim.forward()
    gI = torch.empty_like(psf)
    sim.loss(psf, torch.as_tensor(w.target, device=sim.dev), gI)
    dphi, _, _ = sim.backward(gI)
    torch.cuda.synchronize()
    phi = torch.from_numpy(w.system.doe.phi.astype(np.float64)).requires_grad_(True)
    img = OP.psf(w, phi=phi)
    assert rel_l2(psf.cpu().numpy(), img.detach().numpy()) <= 1e-4
    Lv, _ = OL.eq3_loss(img, torch.from_numpy(w.target.astype(np.float64)))
    Lv.backward()
    assert rel_l2(dphi.cpu().numpy(), phi.grad.numpy()) <= 5e-4


def test_dispersion_spreads_the_colours(RW, ctx):
    """Sensor at the d-line focus of a BK7 singlet: the F and C images are
    broader than the d image (longitudinal chromatic aberration)."""
    s = R.configs.dispersive(R.configs._singlet(5.0))
    surfaces = [R.Surface(R.PLANE, 0.0)] + s
    zs = R.configs.back_focal_z(surfaces[1:])
    phi = np.zeros((256, 256), np.float32)
    doe = R.DOE(phi=phi, pitch=8e-3, D=16)                    # T = 1 over 2 mm
    sysm = R.System(surfaces, 0, doe, R.Sensor(z=zs, nx=128, ny=128, pitch=2e-3))
    jobs = [R.Job(lam=lam, grid_n=15, spacing=0.1) for lam in LAMS]   # 1.4 mm pupil
    w = R.systems.Workload("singlet colours", sysm, jobs, z_start=-1.0)
    img = RW.Simulator(w, ctx=ctx).forward().cpu().numpy()
    x = (np.arange(128) - 63.5) * 2e-3
    X, Y = np.meshgrid(x, x)
    rms = [np.sqrt((im * (X ** 2 + Y ** 2)).sum() / im.sum()) for im in img]
    assert rms[1] < rms[0] and rms[1] < rms[2], rms


def test_dispersive_media_refused_where_unsupported(RW, ctx):
    w = _c2_dispersive(n_side=3)
    sim = RW.Simulator(w, ctx=ctx)
    with pytest.raises(RW.RayWaveError) as e:
        sim.emit()
    assert e.value.status == 1
    vis = RW.alloc_vis(sim.n_rays, w.system.doe.M, sim.dev)
    with pytest.raises(RW.RayWaveError) as e:
        sim.forward(vis=vis)
    assert e.value.status == 1
