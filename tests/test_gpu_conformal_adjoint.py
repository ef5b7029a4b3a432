"""Adjoint through a conformal DOE against the FP64 oracle's autograd.

The curved substrate makes the DOE hit, its tangent frame (u, v, n) and the
tangent-plane patch samples (read bilinearly at their orthographic (x, y))
functions of the incident ray and of the substrate's parameters; the emitted
directions depend on the frame and the incident wavevector.  The adjoint
reverses all of it, so the surfaces before the DOE and the substrate itself
receive gradients.

Cases: the C4 geometry scaled down (even asphere -> plane -> DOE on a sphere,
incoherent sensor), through the fused adjoint and the split adjoint over the
visibility mask, checking every slot of the asphere (z, c, k, A4..A10, n),
the plane and the sphere (z, c); and the reflective DOE on a Gaussian bump
with a coherent sensor (height and width of the bump, mirror z).
"""
import numpy as np
import pytest
import torch

import reflective_cases as RC
import rwinputs as R
from oracle import loss as OL
from oracle import pipeline as OP

from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

NAMES = ["z", "c", "k", "A4", "A6", "A8", "A10", "n_after"]


@pytest.fixture(scope="module")
def RW():
    from paper_2605_15418_gb300 import raywave
    return raywave


def _oracle(w):
    prm = OP.params_of(w.system, requires_grad=True)
    phi = torch.from_numpy(w.system.doe.phi.astype(np.float64)).requires_grad_(True)
    amp = None
    if w.system.doe.amp is not None:
        amp = torch.from_numpy(w.system.doe.amp.astype(np.float64)).requires_grad_(True)
    img = OP.psf(w, params=prm, phi=phi, amp=amp)
    Lv, _ = OL.eq3_loss(img, torch.from_numpy(w.target.astype(np.float64)))
    Lv.backward()
    gs = np.zeros((len(prm), 8))
    for si, p in enumerate(prm):
        for k, name in enumerate(NAMES):
            g = p[name].grad
            gs[si, k] = 0.0 if g is None else float(g)
    return (img.detach().numpy(), phi.grad.numpy(),
            None if amp is None else amp.grad.numpy(), gs)


def _gpu(RW, w, masked):
    sim = RW.Simulator(w)
    vis = RW.alloc_vis(sim.n_rays, w.system.doe.M, sim.dev) if masked else None
    psf = sim.forward(vis=vis)
    gI = torch.empty_like(psf)
    sim.loss(psf, torch.as_tensor(w.target, device=sim.dev), gI)
    dphi, damp, dsurf = sim.backward(gI, want_amp=True, vis=vis)
    torch.cuda.synchronize()
    assert sim.ctx.device_status() == 0
    return (psf.cpu().numpy(), dphi.cpu().numpy(),
            None if damp is None else damp.cpu().numpy(), dsurf.cpu().numpy())


def _c4_small(aperture=0.2, map_side=512):
    """C4's surfaces, 10 x 10 rays per field over the central `aperture` mm
    of the map (map_side pixels at 0.5 um)."""
    w = R.configs.c4(n_side=10, D=16, n_fields=3, max_field_deg=5.0, map_side=map_side,
                     lams=(550e-6,))
    for j in w.jobs:
        j.spacing = aperture / 10
    sysm = w.system
    # a weakly scattering map (phase up to 0.3 rad, amplitude 0.8..1), so that
    # most of the light reaches the focus on the sensor
    rng = np.random.default_rng(43)
    sysm.doe.phi = (0.3 * rng.uniform(size=(map_side, map_side))).astype(np.float32)
    sysm.doe.amp = (0.8 + 0.2 * rng.uniform(size=(map_side, map_side))).astype(np.float32)
    sysm.sensor.nx = sysm.sensor.ny = 64
    sysm.sensor.pitch = 6e-3 * max(1.0, aperture / 0.2)
    w.target = R.gaussian_spots_target(len(w.jobs), 64, 64, seed=41, n_spots=3)
    return w


_C4_CASES = {"0.2mm": (0.2, 512), "2mm": (2.0, 4096)}


@pytest.fixture(scope="module")
def c4_oracles():
    cache = {}

    def get(name):
        if name not in cache:
            w = _c4_small(*_C4_CASES[name])
            cache[name] = (w,) + _oracle(w)
        return cache[name]
    return get


@pytest.mark.parametrize("masked", [False, True])
@pytest.mark.parametrize("case", list(_C4_CASES))
def test_conformal_sphere_behind_asphere_all_slots(RW, c4_oracles, case, masked):
    w, img, gphi, gamp, gs = c4_oracles(case)
    psf, dphi, damp, dsurf = _gpu(RW, w, masked)
    assert rel_l2(psf, img) <= 1e-4, rel_l2(psf, img)
    assert rel_l2(dphi, gphi) <= 1e-3, rel_l2(dphi, gphi)
    assert rel_l2(damp, gamp) <= 1e-3, rel_l2(damp, gamp)
    # the asphere before the DOE: every slot, each against its own magnitude
    bad = []
    for k in range(8):
        if abs(dsurf[0, k] - gs[0, k]) > 1e-3 * abs(gs[0, k]):
            bad.append((0, NAMES[k], dsurf[0, k], gs[0, k]))
    # the plane behind it (z, n) and the DOE sphere (z, c).  Near the apex
    # (0.2 mm aperture) the sphere's curvature gradient is only 1.6e-4 and
    # carries an absolute float error of ~6e-5; over 2 mm it is 4.5e-2 and
    # within 1e-3 -- hence an absolute floor of 1e-4 on that slot.
    for si, k in ((1, 0), (1, 7), (2, 0), (2, 1)):
        floor = 1e-4 if (si, k) == (2, 1) else 0.0
        if abs(dsurf[si, k] - gs[si, k]) > 1e-3 * abs(gs[si, k]) + floor:
            bad.append((si, NAMES[k], dsurf[si, k], gs[si, k]))
    assert not bad, bad
    assert all(gs[0, k] != 0.0 for k in range(8))


def test_conformal_gaussian_bump_mirror_coherent(RW):
    w = RC.gauss(n_side=6, D=16, coherent=True, window=0, amp=True, field_deg=0.3)
    psf, dphi, damp, dsurf = _gpu(RW, w, False)
    img, gphi, gamp, gs = _oracle(w)
    assert rel_l2(psf, img) <= 1e-4, rel_l2(psf, img)
    assert rel_l2(dphi, gphi) <= 5e-4, rel_l2(dphi, gphi)
    assert rel_l2(damp, gamp) <= 5e-4, rel_l2(damp, gamp)
    # mirror z, bump height (c slot) and width (k slot)
    bad = [(NAMES[k], dsurf[0, k], gs[0, k]) for k in (0, 1, 2)
           if abs(dsurf[0, k] - gs[0, k]) > 2e-3 * abs(gs[0, k])]
    assert not bad, bad
