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


# ------------------------------------------------------------------ SSR sampling (Fig. 3)
def _patch_image(RW, ctx, phi, z, emit, n_ssr=0, rng_offset=0):
    D = 96
    doe = R.DOE(phi=phi, pitch=PITCH, D=D, lambda0=LAM, emit=emit, n_ssr=n_ssr,
                seed=(77 << 32) | 1, rng_offset=rng_offset)
    sen = R.Sensor(z=z, nx=64, ny=64, pitch=1e-3, coherent=True)
    sysm = R.System([R.Surface(R.PLANE, 0.0)], 0, doe, sen)
    job = R.Job(lam=LAM, grid_n=1, x0=0.1 * PITCH, y0=0.2 * PITCH)
    w = R.systems.Workload("one patch", sysm, [job], z_start=-0.01)
    return RW.Simulator(w, ctx=ctx).forward().cpu().numpy()[0].astype(np.float64)


def test_ssr_sampling_density_regimes():
    """Monte-Carlo convergence of sampled secondary rays for one ray at the
    centre of a 48 lambda patch (Fig. 3, scaled down): the error of the
    coherent image against the exhaustive one (every bin: the patch's
    angular spectrum, pinned to angular-spectrum propagation) falls at least
    like 1/N for both densities; for a metalens patch (NA 0.1, one spectral
    lobe) p_mag ~ |U~| converges much faster than p_uni; for a holographic
    patch (random phase, a spectrum spread over every bin -- standing in for
    the paper's Siemens-star hologram) the two are similar.  Measured
    normalised MSE at N = 256, 1024, 4096: metalens p_mag 7.8e-2, 9.1e-3,
    1.8e-3 vs p_uni 1.1e2, 6.5, 0.41; hologram p_mag 5.7e2, 38, 3.7 vs p_uni
    8.8e2, 59, 5.2."""
    from paper_2605_15418_gb300 import raywave as RW
    ctx = RW.Context(0)
    n = 128
    x = (np.arange(n) - n / 2 + 0.5) * PITCH
    X, Y = np.meshgrid(x, x)
    f = 96 * PITCH / 2 / math.tan(math.asin(0.1))
    metalens = np.mod(-2 * math.pi / LAM * (np.sqrt(X ** 2 + Y ** 2 + f ** 2) - f),
                      2 * math.pi).astype(np.float32)
    holo = np.random.Generator(np.random.PCG64(99)).uniform(0, 2 * math.pi,
                                                          (n, n)).astype(np.float32)
    Ns, K = (256, 1024, 4096), 8
    mse = {}
    for name, phi, z in (("metalens", metalens, f), ("holo", holo, 0.05)):
        ref = _patch_image(RW, ctx, phi, z, "exhaustive")
        for dens in ("sampled", "sampled_uniform"):
            for N in Ns:
                e = 0.0
                for k in range(K):
                    img = _patch_image(RW, ctx, phi, z, dens, N, k)
                    e += ((img - ref) ** 2).mean() / (ref ** 2).mean()
                mse[name, dens, N] = e / K
    assert ctx.device_status() == 0
    ctx.close()
    for name in ("metalens", "holo"):
        for dens in ("sampled", "sampled_uniform"):
            for a, b in zip(Ns, Ns[1:]):
                assert mse[name, dens, b] < mse[name, dens, a] / 2.5, (name, dens, mse)
    for N in Ns:
        assert mse["metalens", "sampled", N] < mse["metalens", "sampled_uniform", N] / 20, mse
        r = mse["holo", "sampled", N] / mse["holo", "sampled_uniform", N]
        assert 0.4 < r < 1.5, (N, r, mse)
