"""Zero-padded patches (M = P D) on the GPU against the FP64 oracle.

The patch keeps its D x D samples and is transformed on M = P D points:
finer bins (k_j = 2 pi j / (M p)), M^2 secondary rays per incident ray in
exhaustive mode, spectrum scale 1/(D M) (incoherent sensor) or 1/M^2
(coherent).  Same tolerances as the unpadded parity tests.
"""
import numpy as np
import pytest
import torch

import rwinputs as R
from oracle import loss as OL
from oracle import pipeline as OP

from gpu_helpers import angle, oracle_psf, rel_l2

pytestmark = pytest.mark.gpu

PSF_TOL = 1e-4
DIR_TOL = 1e-6
A_TOL = 1e-5


@pytest.fixture(scope="module")
def RW():
    from paper_2605_15418_gb300 import raywave
    return raywave


@pytest.fixture(scope="module")
def ctx(RW):
    c = RW.Context(0)
    yield c
    c.close()


def _c2_padded(n_side, D, P, map_side=256, lams=(486e-6, 656e-6), fields=(0.0, 2.0),
               sensor_n=96):
    w = R.configs.c2(n_side=n_side, D=D, lams=lams, fields_deg=fields, sensor_n=sensor_n,
                     map_side=map_side)
    w.system.sensor.pitch = 8e-3
    w.system.doe.pad = P
    return w


def _c3_padded(n_side, D=16, P=2):
    w = R.configs.c3(n_side=n_side, D=D)
    sysm = w.system
    sysm.doe.phi = (R.maps.random_phase(512, 512, 11) * 0.3 + sysm.doe.phi).astype(np.float32)
    sysm.doe.pad = P
    sysm.sensor.nx = sysm.sensor.ny = 64
    sysm.sensor.pitch = 30e-3
    w.target = R.gaussian_spots_target(1, 64, 64, seed=5, n_spots=3)
    return w


def _oracle_grads(w):
    prm = OP.params_of(w.system, requires_grad=True)
    phi = torch.from_numpy(w.system.doe.phi.astype(np.float64)).requires_grad_(True)
    img = OP.psf(w, params=prm, phi=phi)
    Lv, _ = OL.eq3_loss(img, torch.from_numpy(w.target.astype(np.float64)))
    Lv.backward()
    return img.detach().numpy(), phi.grad.numpy(), prm


# ------------------------------------------------------------------ forward
@pytest.mark.parametrize("D,P,n_side", [(16, 2, 29), (32, 2, 17), (32, 3, 9), (64, 2, 7)])
def test_forward_psf_padded_planar(RW, ctx, D, P, n_side):
    """Transform sizes 32, 64, 96 and 128; every case spans several 32-ray
    tiles with a ragged last tile."""
    w = _c2_padded(n_side, D, P)
    sim = RW.Simulator(w, ctx=ctx)
    psf = sim.forward().cpu().numpy()
    ref = oracle_psf(w)
    assert ref.sum() > 0
    assert rel_l2(psf, ref) <= PSF_TOL, rel_l2(psf, ref)


def test_padding_changes_the_psf(RW, ctx):
    """P = 2 samples the spectrum on twice as many bins: the image differs
    from the unpadded one, and both keep the same total power (the
    incoherent scale 1/(D M) preserves sum |U~|^2)."""
    w1 = _c2_padded(17, 32, 1)
    w2 = _c2_padded(17, 32, 2)
    p1 = RW.Simulator(w1, ctx=ctx).forward().cpu().numpy()
    p2 = RW.Simulator(w2, ctx=ctx).forward().cpu().numpy()
    assert rel_l2(p2, p1) > 1e-3
    r1, r2 = oracle_psf(w1), oracle_psf(w2)
    assert abs(p2.sum() / p1.sum() - r2.sum() / r1.sum()) < 1e-5


def test_forward_coherent_padded(RW, ctx):
    for window in (0, 6):
        w = _c2_padded(9, 16, 2, map_side=64, lams=(550e-6,), fields=(0.5,), sensor_n=48)
        w.system.surfaces = w.system.surfaces[:1]
        w.system.sensor.z = 0.2
        w.system.sensor.pitch = 2e-3
        w.system.sensor.coherent = True
        w.system.sensor.window = window
        sim = RW.Simulator(w, ctx=ctx)
        psf = sim.forward().cpu().numpy()
        ref = oracle_psf(w)
        assert rel_l2(psf, ref) <= PSF_TOL, (window, rel_l2(psf, ref))


# ------------------------------------------------------------------ emission
def test_emit_padded_exhaustive_directions_and_weights(RW, ctx):
    w = _c2_padded(12, 16, 2, map_side=128, lams=(550e-6,), fields=(1.0,))
    sim = RW.Simulator(w, ctx=ctx)
    out = sim.emit()
    torch.cuda.synchronize()
    M = w.system.doe.M
    d = torch.stack([out["dx"], out["dy"], out["dz"]], -1).cpu().numpy().reshape(-1, M, M, 3)
    a = (out["a_re"].double() + 1j * out["a_im"].double()).cpu().numpy().reshape(-1, M, M)
    with torch.no_grad():
        em, _ = OP.emit_job(w.system, w.jobs[0], w.z_start, OP.params_of(w.system),
                            *OP.map_tensors(w.system))
    alive = em["alive"].numpy()
    ang = angle(d[alive], em["d"].numpy()[alive])
    assert ang.max() <= DIR_TOL, ang.max()
    ar = em["a"].numpy()
    assert np.abs(a - np.where(alive, ar, 0)).max() <= A_TOL * np.abs(ar).max()


@pytest.mark.parametrize("coherent", [False, True])
def test_sampled_emission_padded(RW, ctx, coherent):
    w = _c2_padded(8, 16, 2, map_side=128, lams=(550e-6,), fields=(0.0, 1.0))
    w.system.doe.emit = "sampled"
    w.system.doe.n_ssr = 48
    w.system.doe.seed = (4242 << 32) | 17
    w.system.sensor.coherent = coherent
    sim = RW.Simulator(w, ctx=ctx)
    out = sim.emit()
    torch.cuda.synchronize()
    N = w.system.doe.n_ssr
    bins = out["bin"].cpu().numpy().reshape(-1, N)
    d = torch.stack([out["dx"], out["dy"], out["dz"]], -1).cpu().numpy().reshape(-1, N, 3)
    a = (out["a_re"].double() + 1j * out["a_im"].double()).cpu().numpy().reshape(-1, N)
    base = agree = total = 0
    for job in w.jobs:
        with torch.no_grad():
            em, _ = OP.emit_job(w.system, job, w.z_start, OP.params_of(w.system),
                                *OP.map_tensors(w.system), ray_base=base)
        g = base + np.arange(job.n_rays)
        same = bins[g] == em["idx"].numpy()
        agree += same.sum()
        total += same.size
        assert angle(d[g][same], em["d"].numpy()[same]).max() <= DIR_TOL
        ar = em["a"].numpy()
        assert np.abs(a[g][same] - ar[same]).max() <= A_TOL * np.abs(ar).max()
        base += job.n_rays
    assert agree >= total * (1 - 1e-3), (agree, total)


# ------------------------------------------------------------------ spectra
def test_patch_spectra_padded_match_fp64_dft(RW, ctx):
    w = _c2_padded(11, 32, 2, lams=(486e-6,), fields=(0.0, 2.0), sensor_n=32)
    sim = RW.Simulator(w, ctx=ctx)
    got = sim.spectra("fft32").cpu().numpy()
    ref = []
    base = 0
    with torch.no_grad():
        for job in w.jobs:
            em, _ = OP.emit_job(w.system, job, w.z_start, OP.params_of(w.system),
                                *OP.map_tensors(w.system), ray_base=base)
            ref.append(em["U"].numpy())
            base += job.n_rays
    ref = np.concatenate(ref, 0)
    assert got.shape == ref.shape == (w.n_rays, 64, 64)
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)
    with pytest.raises(RW.RayWaveError) as e:
        sim.spectra("tc")                  # tensor-core transform: D = 64, no padding
    assert e.value.status == 1


# ------------------------------------------------------------------ adjoint
def test_backward_padded_matches_oracle_gradient(RW, ctx):
    """Fused adjoint at M = 32 (D = 16, P = 2)."""
    w = _c3_padded(20)
    sim = RW.Simulator(w, ctx=ctx)
    psf = sim.forward()
    gI = torch.empty_like(psf)
    sim.loss(psf, torch.as_tensor(w.target, device=sim.dev), gI)
    dphi, _, dsurf = sim.backward(gI)
    torch.cuda.synchronize()
    img, gphi, prm = _oracle_grads(w)
    assert rel_l2(psf.cpu().numpy(), img) <= PSF_TOL
    assert rel_l2(dphi.cpu().numpy(), gphi) <= 1e-3, rel_l2(dphi.cpu().numpy(), gphi)
    ds = dsurf.cpu().numpy()
    cmax = max(abs(float(p["c"].grad or 0)) for p in prm[1:])
    for si in range(1, len(prm)):
        for k, name in ((0, "z"), (1, "c"), (7, "n_after")):
            ref = prm[si][name].grad
            ref = 0.0 if ref is None else float(ref)
            assert abs(ds[si, k] - ref) <= 1e-3 * max(abs(ref), 1e-3 * cmax) + 1e-9, \
                (si, name, ds[si, k], ref)


def test_backward_padded_m128_split_adjoint(RW, ctx):
    """M = 128 (D = 64, P = 2) has no fused adjoint (shared memory); the
    masked split adjoint serves it and matches the oracle's autograd."""
    w = _c3_padded(7, D=64, P=2)
    ctx.device_status()
    sim = RW.Simulator(w, ctx=ctx)
    vis = RW.alloc_vis(sim.n_rays, w.system.doe.M, sim.dev)
    psf = sim.forward(vis=vis)
    gI = torch.empty_like(psf)
    sim.loss(psf, torch.as_tensor(w.target, device=sim.dev), gI)
    with pytest.raises(RW.RayWaveError) as e:
        sim.backward(gI)                   # fused path: refused with RW_EINVAL
    assert e.value.status == 1
    dphi, _, dsurf = sim.backward(gI, vis=vis)
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    img, gphi, prm = _oracle_grads(w)
    assert rel_l2(psf.cpu().numpy(), img) <= PSF_TOL
    assert rel_l2(dphi.cpu().numpy(), gphi) <= 1e-3, rel_l2(dphi.cpu().numpy(), gphi)
    ds = dsurf.cpu().numpy()
    for si in range(1, len(prm)):
        ref = float(prm[si]["c"].grad)
        assert abs(ds[si, 1] - ref) <= 1e-3 * abs(ref) + 1e-6, (si, ds[si, 1], ref)


def test_visibility_mask_backward_padded_equals_full(RW, ctx):
    """M = 64 (D = 32, P = 2): the split adjoint over the mask equals the
    fused adjoint over every bin."""
    w = _c2_padded(13, 32, 2)
    ctx.device_status()
    sim = RW.Simulator(w, ctx=ctx)
    vis = RW.alloc_vis(sim.n_rays, w.system.doe.M, sim.dev)
    psf = sim.forward(vis=vis)
    tgt = torch.as_tensor(R.gaussian_spots_target(len(w.jobs), 96, 96, seed=3), device=sim.dev)
    gI = torch.empty_like(psf)
    sim.loss(psf, tgt, gI)
    full = sim.backward(gI)
    culled = sim.backward(gI, vis=vis)
    torch.cuda.synchronize()
    assert rel_l2(culled[0].cpu().numpy(), full[0].cpu().numpy()) < 1e-5
    assert rel_l2(culled[2].cpu().numpy(), full[2].cpu().numpy()) < 1e-5
    assert ctx.device_status() == 0
