"""Reflective DOEs on the GPU against the FP64 oracle: a planar mirror DOE
and a conformal one on a Gaussian bump (apex radius 506 lambda), incoherent
and coherent sensor in front of the DOE, one or two superposed phase
profiles (U = A (exp(i phi) + exp(i phi2))), forward and adjoint (dL/dphi,
dL/dphi2, dL/dA), and the argument checks of the reflective geometry."""
import numpy as np
import pytest
import torch

import reflective_cases as RC
import rwinputs as R
from oracle import loss as OL
from oracle import pipeline as OP

from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

PSF_TOL = 1e-4
MAP_TOL = 5e-4


@pytest.fixture(scope="module")
def RW():
    from paper_2605_15418_gb300 import raywave
    return raywave


@pytest.fixture(scope="module")
def ctx(RW):
    c = RW.Context(0)
    yield c
    c.close()


def _oracle_grads(w):
    prm = OP.params_of(w.system, requires_grad=True)
    doe = w.system.doe
    phi = torch.from_numpy(doe.phi.astype(np.float64)).requires_grad_(True)
    phi2 = None if doe.phi2 is None else torch.from_numpy(
        doe.phi2.astype(np.float64)).requires_grad_(True)
    amp = None if doe.amp is None else torch.from_numpy(
        doe.amp.astype(np.float64)).requires_grad_(True)
    img = OP.psf(w, params=prm, phi=phi, amp=amp, phi2=phi2)
    Lv, _ = OL.eq3_loss(img, torch.from_numpy(w.target.astype(np.float64)))
    Lv.backward()
    g = phi.grad.numpy() if phi2 is None else np.stack([phi.grad.numpy(), phi2.grad.numpy()])
    return img.detach().numpy(), g, None if amp is None else amp.grad.numpy()


def _gpu(RW, ctx, w, vis=False):
    ctx.device_status()
    sim = RW.Simulator(w, ctx=ctx)
    v = RW.alloc_vis(sim.n_rays, w.system.doe.M, sim.dev) if vis else None
    psf = sim.forward(vis=v)
    gI = torch.empty_like(psf)
    sim.loss(psf, torch.as_tensor(w.target, device=sim.dev), gI)
    dphi, damp, _ = sim.backward(gI, want_amp=True, vis=v)
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    return (psf.cpu().numpy(), dphi.cpu().numpy(),
            None if damp is None else damp.cpu().numpy())


def _compare(RW, ctx, w, vis=False, map_tol=MAP_TOL):
    psf, dphi, damp = _gpu(RW, ctx, w, vis)
    img, gphi, gamp = _oracle_grads(w)
    assert img.sum() > 0
    assert rel_l2(psf, img) <= PSF_TOL, rel_l2(psf, img)
    assert dphi.shape == gphi.shape
    assert rel_l2(dphi, gphi) <= map_tol, rel_l2(dphi, gphi)
    if gamp is not None:
        assert rel_l2(damp, gamp) <= map_tol, rel_l2(damp, gamp)


# ------------------------------------------------------------------ planar mirror DOE
def test_reflective_planar_incoherent(RW, ctx):
    _compare(RW, ctx, RC.planar(n_side=9, amp=True))


def test_reflective_planar_incoherent_masked_adjoint(RW, ctx):
    """Exhaustive incoherent forward with the visibility mask (block culling
    applies) and the split adjoint over it."""
    _compare(RW, ctx, RC.planar(n_side=9), vis=True)


def test_reflective_planar_coherent_windowed(RW, ctx):
    _compare(RW, ctx, RC.planar(n_side=9, coherent=True, window=5))


def test_reflective_planar_two_phases_coherent(RW, ctx):
    _compare(RW, ctx, RC.planar(n_side=9, coherent=True, two_phase=True, amp=True))


def test_reflective_planar_sampled_coherent(RW, ctx):
    _compare(RW, ctx, RC.planar(n_side=9, coherent=True, emit="sampled"), map_tol=2e-3)


# ------------------------------------------------------------------ conformal DOE on a Gaussian bump
def test_reflective_gaussian_bump_coherent(RW, ctx):
    _compare(RW, ctx, RC.gauss(n_side=7))


def test_reflective_gaussian_bump_two_phases_with_amplitude(RW, ctx):
    _compare(RW, ctx, RC.gauss(n_side=7, two_phase=True, amp=True))


def test_reflective_gaussian_bump_incoherent_padded(RW, ctx):
    w = RC.gauss(n_side=7, coherent=False)
    w.system.doe.pad = 2
    _compare(RW, ctx, w)


def test_gaussian_bump_emission_directions_match_oracle(RW, ctx):
    """Secondary directions and weights of the reflective conformal DOE (FP64
    Newton hit, normal of the bump, outgoing normal reversed).  At a pitch of
    lambda/2 the spectrum reaches grazing directions (sin theta -> 1), where an
    error e of the tangential components would turn the direction by ~e / a_n;
    near grazing the normal component is formed in double from double-float
    tangential components, so 1e-6 rad holds over every propagating bin."""
    from gpu_helpers import angle
    w = RC.gauss(n_side=5, coherent=False, field_deg=3.0)
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
    dref = em["d"].numpy()
    ang = angle(d[alive], dref[alive])
    assert ang.max() <= 1e-6, ang.max()
    # every secondary ray leaves on the incident side of the local surface
    # (grazing ones may still have d_z > 0 where the bump is tilted)
    n_out = em["frame"][2].numpy()                      # outgoing normal per ray
    cosn = (d * n_out[:, None, None, :]).sum(-1)
    assert (cosn[alive] > 0).all()
    ar = em["a"].numpy()
    assert np.abs(a - np.where(alive, ar, 0)).max() <= 1e-5 * np.abs(ar).max()


# ------------------------------------------------------------------ argument checks
def test_reflective_geometry_is_checked(RW, ctx):
    w = RC.planar(n_side=2)
    w.system.sensor.z = 0.1                            # behind the mirror
    with pytest.raises(RW.RayWaveError) as e:
        RW.Simulator(w, ctx=ctx).forward()
    assert e.value.status == 1
    w = RC.planar(n_side=2)
    w.system.surfaces = [w.system.surfaces[0], R.Surface(R.PLANE, 1.0)]   # not the last surface
    with pytest.raises(RW.RayWaveError) as e:
        RW.Simulator(w, ctx=ctx).forward()
    assert e.value.status == 1
    w = RC.gauss(n_side=2)                                       # a Gaussian bump as a lens
    w.system.surfaces = [R.Surface(R.GAUSS, -1.0, c=0.01, k=0.1), w.system.surfaces[0]]
    w.system.doe_index = 1
    with pytest.raises(RW.RayWaveError) as e:
        RW.Simulator(w, ctx=ctx).forward()
    assert e.value.status == 1
