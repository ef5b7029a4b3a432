"""Small seeded coherent-sensor workloads (Eq. 2) for the oracle's gradient
pin and the GPU adjoint parity tests.

free_space   planar complex DOE (64 x 64 px at 1 um) alone, sensor 0.2 mm behind
lens_after   the same DOE followed by a BK7 singlet (R = +-20 mm, 3 mm thick),
             sensor 1 mm behind the lens
lens_before  the singlet first, the DOE 2 mm behind it, sensor 0.2 mm behind the DOE
conformal    a complex map on a sphere (R = 25 mm) behind the singlet, bilinear gather

Every sensor is 32 x 32 pixels; the Eq. 3 target is a seeded sum of Gaussian
spots.  `window` > 0 limits each wavelet to +-window pixels (default: the
whole sensor).
"""
import math

import numpy as np

import rwinputs as R

UM = 1e-3
N_BK7 = 1.5168


def _maps(H, W, seed, with_amp):
    rng = np.random.Generator(np.random.PCG64(seed))
    # a smooth tilt plus a random term, so patches are neither flat nor white
    yy, xx = np.mgrid[0:H, 0:W]
    phi = (0.15 * xx + 0.07 * yy + rng.uniform(0.0, 1.2, (H, W))).astype(np.float32)
    amp = rng.uniform(0.4, 1.0, (H, W)).astype(np.float32) if with_amp else None
    return phi, amp


def _singlet(z0, R_=20.0, ct=3.0):
    return [R.Surface(R.SPHERE, z0, c=1.0 / R_, n_after=N_BK7, r_ap=6.0),
            R.Surface(R.SPHERE, z0 + ct, c=-1.0 / R_, n_after=1.0, r_ap=6.0)]


def _workload(name, surfaces, doe_index, doe, sensor, n_side, spacing, field_deg, seed):
    sysm = R.System(surfaces, doe_index, doe, sensor)
    job = R.Job(lam=550e-6, theta_x=0.0, theta_y=math.radians(field_deg), grid_n=n_side,
                spacing=spacing, x0=0.0, y0=0.0)
    w = R.systems.Workload(name, sysm, [job], z_start=-1.0)
    w.target = R.gaussian_spots_target(1, sensor.ny, sensor.nx, seed=seed, n_spots=3,
                                       sigma_px=(2.0, 5.0))
    return w


def _doe(D, pad, amp, emit, n_ssr, seed=81, kind=R.PLANAR, gather="nearest"):
    phi, a = _maps(64, 64, seed, amp)
    doe = R.DOE(phi=phi, amp=a, pitch=1 * UM, D=D, lambda0=550e-6, pad=pad, kind=kind,
                gather=gather)
    if emit != "exhaustive":
        doe.emit = emit
        doe.n_ssr = n_ssr
        doe.seed = (97 << 32) | 5
    return doe


def free_space(n_side=8, D=16, pad=1, window=0, amp=True, emit="exhaustive", n_ssr=64):
    doe = _doe(D, pad, amp, emit, n_ssr)
    sen = R.Sensor(z=0.2, nx=32, ny=32, pitch=2 * UM, coherent=True, window=window)
    return _workload("coherent free space", [R.Surface(R.PLANE, 0.0)], 0, doe, sen, n_side,
                     40 * UM / n_side, 0.5, 91)


def lens_after(n_side=8, D=16, pad=1, amp=False, emit="exhaustive", n_ssr=64, window=0):
    doe = _doe(D, pad, amp, emit, n_ssr)
    surfaces = [R.Surface(R.PLANE, 0.0)] + _singlet(0.5)
    sen = R.Sensor(z=4.5, nx=32, ny=32, pitch=4 * UM, coherent=True, window=window)
    return _workload("coherent DOE + singlet", surfaces, 0, doe, sen, n_side, 40 * UM / n_side,
                     0.3, 92)


def lens_before(n_side=8, D=16, amp=False, window=0):
    doe = _doe(D, 1, amp, "exhaustive", 0)
    surfaces = _singlet(0.0) + [R.Surface(R.PLANE, 5.0)]
    sen = R.Sensor(z=5.2, nx=32, ny=32, pitch=2 * UM, coherent=True, window=window)
    return _workload("coherent singlet + DOE", surfaces, 2, doe, sen, n_side, 40 * UM / n_side,
                     0.4, 93)


def conformal(n_side=8, D=16, window=0):
    doe = _doe(D, 1, True, "exhaustive", 0, kind=R.CONFORMAL, gather="bilinear")
    surfaces = _singlet(0.0) + [R.Surface(R.SPHERE, 5.0, c=1.0 / 25.0)]
    sen = R.Sensor(z=5.2, nx=32, ny=32, pitch=2 * UM, coherent=True, window=window)
    return _workload("coherent singlet + conformal DOE", surfaces, 2, doe, sen, n_side,
                     40 * UM / n_side, 0.4, 94)
