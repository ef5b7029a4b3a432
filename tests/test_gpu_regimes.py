"""Regime studies of the paper's convergence section as automated GPU tests.

Patch size vs incident-ray count (Fig. 2a-c, scaled down): a planar
hologram of 128 lambda x 128 lambda (lambda = 1 um, pitch lambda/2, a lens of
NA 0.7 plus a smooth random phase) imaged coherently at its focal plane.  The
reference is the angular-spectrum propagation of the whole hologram (NumPy
FFT, obliquity k_z/k as in Eq. 2).  Every patch size D is transformed on
M = 128 points (P = 128/D), so the periodic copies of a patch's field land
outside the sensor for every D and only the patch size and the ray density
differ.  Rays hit at seeded uniform random points (the patches' coverage
of the hologram is then random, as with any unstructured ray set).

What the paper reports and this test checks:
* one incident ray: a larger patch gives a higher NCC;
* an ensemble: NCC rises with the number of rays for every D, towards 1;
* the rays needed for a given NCC (here 0.85) fall as D grows (Fig. 2c).
Measured (NCC for N = 64, 256, 1024, 4096): D = 16: 0.21, 0.51, 0.79, 0.94;
D = 32: 0.41, 0.76, 0.90, 0.97; D = 64: 0.64, 0.91, 0.95, 0.98.
"""
import math

import numpy as np
import pytest
import torch

import rwinputs as R

from physics_refs import asm_propagate

pytestmark = pytest.mark.gpu

LAM, PITCH, NMAP, NSEN, NA = 1e-3, 0.5e-3, 256, 64, 0.7


def _hologram():
    x = (np.arange(NMAP) - NMAP / 2 + 0.5) * PITCH
    X, Y = np.meshgrid(x, x)
    f = NMAP * PITCH / 2 / math.tan(math.asin(NA))
    rng = np.random.Generator(np.random.PCG64(2024))
    phi = -2 * math.pi / LAM * (np.sqrt(X ** 2 + Y ** 2 + f ** 2) - f)
    for _ in range(12):
        kx, ky = rng.normal(0, 0.06, 2) * 2 * math.pi / LAM
        phi += 1.2 * np.cos(kx * X + ky * Y + rng.uniform(0, 2 * math.pi))
    return np.mod(phi, 2 * math.pi).astype(np.float32), f


def _reference(phi, f):
    pad = 1024
    T = np.zeros((pad, pad), np.complex128)
    o = (pad - NMAP) // 2
    T[o:o + NMAP, o:o + NMAP] = np.exp(1j * phi.astype(np.float64))
    U = asm_propagate(T, PITCH, LAM, f)
    c = o + NMAP // 2 - NSEN // 2            # sensor pixels sit on map pixel centres
    return np.abs(U[c:c + NSEN, c:c + NSEN]) ** 2


def _ncc(a, b):
    a = a - a.mean()
    b = b - b.mean()
    return float((a * b).sum() / math.sqrt((a * a).sum() * (b * b).sum()))


def _image(RW, ctx, phi, f, D, pos):
    n = pos.shape[0]
    g = int(round(math.sqrt(n)))
    assert g * g == n
    doe = R.DOE(phi=phi, pitch=PITCH, D=D, lambda0=LAM, pad=128 // D)
    sen = R.Sensor(z=f, nx=NSEN, ny=NSEN, pitch=PITCH, coherent=True)
    sysm = R.System([R.Surface(R.PLANE, 0.0)], 0, doe, sen)
    w = R.systems.Workload("hologram", sysm, [R.Job(lam=LAM, grid_n=g)], z_start=-0.01)
    rays = RW.alloc_rays(n, ctx.device)
    rays["ox"].copy_(torch.as_tensor(pos[:, 0], dtype=torch.float32))
    rays["oy"].copy_(torch.as_tensor(pos[:, 1], dtype=torch.float32))
    rays["oz"].fill_(-0.01)
    rays["dx"].zero_()
    rays["dy"].zero_()
    rays["dz"].fill_(1.0)
    rays["a_re"].fill_(1.0)
    rays["a_im"].zero_()
    rays["opl"].fill_(-0.01)                 # n_object (d . o) of the axial plane wave
    return RW.Simulator(w, ctx=ctx, rays=rays).forward().cpu().numpy()[0]


def test_patch_size_and_ray_count_regimes():
    from paper_2605_15418_gb300 import raywave as RW
    ctx = RW.Context(0)
    phi, f = _hologram()
    ref = _reference(phi, f)
    Ds, Ns = (16, 32, 64), (64, 256, 1024, 4096)
    single, ens = {}, {}
    for D in Ds:
        single[D] = _ncc(_image(RW, ctx, phi, f, D, np.array([[0.1 * PITCH, 0.2 * PITCH]])),
                         ref)
        half = NMAP * PITCH / 2 + D * PITCH / 2
        for n in Ns:
            pos = np.random.Generator(np.random.PCG64(7 + n)).uniform(-half, half, (n, 2))
            ens[D, n] = _ncc(_image(RW, ctx, phi, f, D, pos), ref)
    assert ctx.device_status() == 0
    ctx.close()
    # one ray: the larger patch samples more of the hologram
    assert single[64] > single[16] + 0.03, single
    # an ensemble: NCC rises with the ray count and, at a given count, with D
    for D in Ds:
        for a, b in zip(Ns, Ns[1:]):
            assert ens[D, b] > ens[D, a], (D, a, b, ens)
    for n in Ns:
        assert ens[64, n] > ens[32, n] > ens[16, n], (n, ens)
    assert ens[64, 4096] >= 0.97 and ens[16, 4096] >= 0.9, ens
    # rays needed for NCC >= 0.85 fall as the patch grows (Fig. 2c): 4096, 1024, 256
    need = [min([n for n in Ns if ens[D, n] >= 0.85], default=10 ** 9) for D in Ds]
    assert need[0] > need[1] > need[2], (need, ens)
