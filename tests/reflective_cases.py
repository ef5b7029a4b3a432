"""Small seeded workloads with a reflective DOE (the reflective conformal DOE
of the paper's inverse-design section, scaled down): lambda = 1 um, pixel
pitch lambda/2, collimated illumination along the axis, sensor in front of
the DOE.

planar  reflective planar DOE (64 x 64 px), sensor 0.2 mm in front
gauss   reflective DOE on a Gaussian bump z = h exp(-r^2 / (2 w^2)) with
        w = 0.1 mm and apex radius of curvature 506 lambda (the paper's
        minimum substrate radius), 128 x 128 px, sensor 0.25 mm in front

Options: coherent sensor (+- window pixels), sampled emission, a second phase
profile (U = exp(i phi) + exp(i phi2)), an amplitude map.
"""
import math

import numpy as np

import rwinputs as R

UM = 1e-3
LAM = 1e-3            # 1 um
PITCH = 0.5 * UM      # lambda / 2


def _maps(n, seed, with_amp, two_phase):
    rng = np.random.Generator(np.random.PCG64(seed))
    yy, xx = np.mgrid[0:n, 0:n]
    phi = (0.11 * xx - 0.05 * yy + rng.uniform(0.0, 1.0, (n, n))).astype(np.float32)
    phi2 = None
    if two_phase:
        phi2 = (-0.13 * xx + 0.04 * yy + rng.uniform(0.0, 1.0, (n, n))).astype(np.float32)
    amp = rng.uniform(0.5, 1.0, (n, n)).astype(np.float32) if with_amp else None
    return phi, phi2, amp


def _workload(name, surface, doe, sensor, n_side, spacing, field_deg, seed):
    sysm = R.System([surface], 0, doe, sensor)
    job = R.Job(lam=LAM, theta_x=math.radians(field_deg), theta_y=0.0, grid_n=n_side,
                spacing=spacing, x0=0.0, y0=0.0)
    w = R.systems.Workload(name, sysm, [job], z_start=-0.5)
    w.target = R.gaussian_spots_target(1, sensor.ny, sensor.nx, seed=seed, n_spots=3,
                                       sigma_px=(2.0, 5.0))
    return w


def planar(n_side=8, D=16, coherent=False, window=0, amp=False, two_phase=False,
           emit="exhaustive", n_ssr=64, field_deg=0.4):
    phi, phi2, a = _maps(64, 121, amp, two_phase)
    doe = R.DOE(phi=phi, amp=a, pitch=PITCH, D=D, lambda0=LAM, reflective=True, phi2=phi2)
    if emit == "sampled":
        doe.emit, doe.n_ssr, doe.seed = "sampled", n_ssr, (31 << 32) | 9
    sen = R.Sensor(z=-0.2, nx=32, ny=32, pitch=2 * UM, coherent=coherent, window=window)
    return _workload("reflective planar DOE", R.Surface(R.PLANE, 0.0), doe, sen, n_side,
                     20 * UM / n_side, field_deg, 131)


def gauss(n_side=6, D=16, coherent=True, window=0, amp=False, two_phase=False,
          emit="exhaustive", n_ssr=64, field_deg=0.0):
    wd = 0.1
    h = wd * wd / (506 * LAM)
    phi, phi2, a = _maps(128, 122, amp, two_phase)
    doe = R.DOE(phi=phi, amp=a, pitch=PITCH, D=D, lambda0=LAM, kind=R.CONFORMAL,
                gather="bilinear", reflective=True, phi2=phi2)
    if emit == "sampled":
        doe.emit, doe.n_ssr, doe.seed = "sampled", n_ssr, (33 << 32) | 7
    sen = R.Sensor(z=-0.25, nx=32, ny=32, pitch=3 * UM, coherent=coherent, window=window)
    surf = R.Surface(R.GAUSS, 0.0, c=h, k=wd)
    return _workload("reflective DOE on a Gaussian bump", surf, doe, sen, n_side,
                     40 * UM / n_side, field_deg, 132)
