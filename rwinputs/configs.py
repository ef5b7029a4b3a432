"""The five synthetic workloads (C1..C5) and their scaled-down test variants.

C1  planar binary grating, emit only (grating-equation check).
C2  two singlets behind a planar Zernike+holographic DOE, incoherent PSF.
C3  C1's grating DOE followed by C2's singlets; forward + backward.
C4  conformal DOE (sphere R = 25 mm) behind an even asphere, 9 fields x 3 wavelengths.
C5  31 wavelengths x 16 fields, uneven ray counts, 96 x 96 patches, sampled emission.

Sensor placement uses first-order (paraxial y-u) optics on the lens
prescription; that is system set-up, not part of the ray-wave method.
"""
import math
from functools import lru_cache

import numpy as np

from .systems import (Surface, DOE, Sensor, System, Job, Workload,
                      PLANE, SPHERE, ASPHERE, CONFORMAL, PLANAR)
from . import maps

N_BK7 = 1.5168
# Sellmeier coefficients of N-BK7 (B1, B2, B3, C1, C2, C3; C in um^2), from
# the glass maker's published data sheet
N_BK7_SELLMEIER = (1.03961212, 0.231792344, 1.01046945, 0.00600069867, 0.0200179144,
                   103.560653)


def dispersive(surfaces):
    """Copies of `surfaces` whose N-BK7 media (n_after = 1.5168) follow the
    N-BK7 Sellmeier formula."""
    import dataclasses
    return [dataclasses.replace(s, sellmeier=N_BK7_SELLMEIER) if s.n_after == N_BK7 else
            dataclasses.replace(s) for s in surfaces]
UM = 1e-3  # one micrometre in mm


# --------------------------------------------------------------------------
# first-order optics used only to place sensors and aim ray bundles
# --------------------------------------------------------------------------
def _paraxial_matrix(surfaces, z_from, z_to, n_start):
    """2x2 y-u transfer matrix (reduced angle n*u) from plane z_from to z_to
    through the surfaces lying between them."""
    M = np.eye(2)
    z, n = z_from, n_start
    for s in surfaces:
        if s.z < z_from or s.z > z_to:
            continue
        T = np.array([[1.0, (s.z - z) / n], [0.0, 1.0]])
        R = np.array([[1.0, 0.0], [-(s.n_after - n) * s.c, 1.0]])
        M = R @ T @ M
        z, n = s.z, s.n_after
    T = np.array([[1.0, (z_to - z) / n], [0.0, 1.0]])
    return T @ M, n


def back_focal_z(surfaces, n_start=1.0):
    """z of the paraxial focus of a collimated axial beam behind `surfaces`."""
    zl = surfaces[-1].z
    M, n = _paraxial_matrix(surfaces, surfaces[0].z - 1e-9, zl, n_start)
    y, nu = M @ np.array([1.0, 0.0])
    return zl - y * n / nu


def chief_aim(surfaces, z_start, z_stop, tan_theta, n_start=1.0):
    """Launch height at z_start so the paraxial ray of slope tan_theta crosses
    the axis at z_stop, and that ray's height at any later plane."""
    M, n = _paraxial_matrix(surfaces, z_start, z_stop, n_start)
    # y_stop = M00 y0 + M01 (n u0) = 0
    y0 = -M[0, 1] * n_start * tan_theta / M[0, 0]
    return y0


def chief_height(surfaces, z_start, z_at, y0, tan_theta, n_start=1.0):
    M, n = _paraxial_matrix(surfaces, z_start, z_at, n_start)
    return (M @ np.array([y0, n_start * tan_theta]))[0]


def _singlet(z0, R=20.0, ct=3.0, n=N_BK7, r_ap=6.0):
    return [Surface(SPHERE, z0, c=1.0 / R, n_after=n, r_ap=r_ap),
            Surface(SPHERE, z0 + ct, c=-1.0 / R, n_after=1.0, r_ap=r_ap)]


@lru_cache(maxsize=4)
def _c2_phase(H=2048, W=2048, pitch=1 * UM, seed=1506):
    return maps.zernike_holographic_phase(H, W, pitch, seed)


def _grid_jobs(lams, fields, n_side, spacing, surfaces, z_start, z_stop,
               sensor_z=None, center_sensor=False):
    jobs = []
    for lam in lams:
        for (tx, ty) in fields:
            x0 = chief_aim(surfaces, z_start, z_stop, math.tan(tx))
            y0 = chief_aim(surfaces, z_start, z_stop, math.tan(ty))
            cx = cy = 0.0
            if center_sensor:
                cx = chief_height(surfaces, z_start, sensor_z, x0, math.tan(tx))
                cy = chief_height(surfaces, z_start, sensor_z, y0, math.tan(ty))
            jobs.append(Job(lam=lam, theta_x=tx, theta_y=ty, grid_n=n_side,
                            spacing=spacing, x0=x0, y0=y0,
                            sensor_cx=cx, sensor_cy=cy))
    return jobs


# --------------------------------------------------------------------------
# C1: planar binary grating, emit only
# --------------------------------------------------------------------------
def c1(n_side=64, D=32, angles_deg=(0.0, 10.0)):
    H = W = 512
    pitch = 0.5 * UM
    phi = maps.binary_grating(H, W, period_px=16)
    doe = DOE(phi=phi, pitch=pitch, D=D, lambda0=550e-6)
    surfaces = [Surface(PLANE, 0.0)]
    sensor = Sensor(z=1.0, nx=64, ny=64, pitch=2 * UM)
    system = System(surfaces=surfaces, doe_index=0, doe=doe, sensor=sensor)
    spacing = 3 * UM * 64 / n_side
    jobs = _grid_jobs([550e-6], [(math.radians(a), 0.0) for a in angles_deg],
                      n_side, spacing, surfaces, -0.5, 0.0)
    return Workload("C1 planar binary grating emit", system, jobs, z_start=-0.5)


# --------------------------------------------------------------------------
# C2: two singlets behind a planar holographic DOE
# --------------------------------------------------------------------------
def c2(n_side=1024, D=64, lams=(486e-6, 550e-6, 656e-6), fields_deg=(0.0, 1.0, 2.0),
       sensor_n=512, map_side=2048):
    pitch = 1 * UM
    phi = _c2_phase(map_side, map_side, pitch)
    doe = DOE(phi=phi, pitch=pitch, D=D, lambda0=550e-6)
    surfaces = [Surface(PLANE, 0.0)] + _singlet(5.0) + _singlet(10.0)
    zs = back_focal_z(surfaces[1:])
    sensor = Sensor(z=zs, nx=sensor_n, ny=sensor_n, pitch=2 * UM)
    system = System(surfaces=surfaces, doe_index=0, doe=doe, sensor=sensor)
    spacing = map_side * pitch / n_side
    jobs = _grid_jobs(list(lams), [(0.0, math.radians(f)) for f in fields_deg],
                      n_side, spacing, surfaces, -1.0, 0.0)
    w = Workload("C2 two singlets + planar holographic DOE, incoherent PSF",
                 system, jobs, z_start=-1.0)
    w.target = maps.gaussian_spots_target(len(jobs), sensor_n, sensor_n, seed=2002)
    return w


# --------------------------------------------------------------------------
# C3: C1's grating DOE + C2's singlets, forward + backward
# --------------------------------------------------------------------------
def c3(n_side=128, D=32):
    H = W = 512
    pitch = 0.5 * UM
    phi = maps.binary_grating(H, W, period_px=16)
    doe = DOE(phi=phi, pitch=pitch, D=D, lambda0=550e-6)
    surfaces = [Surface(PLANE, 0.0)] + _singlet(5.0) + _singlet(10.0)
    zs = back_focal_z(surfaces[1:])
    # 8 um pixels: the +-1 orders of the 8 um grating land ~0.69 mm off axis
    sensor = Sensor(z=zs, nx=256, ny=256, pitch=8 * UM)
    system = System(surfaces=surfaces, doe_index=0, doe=doe, sensor=sensor)
    spacing = 1.5 * UM * 128 / n_side
    jobs = _grid_jobs([550e-6], [(0.0, 0.0)], n_side, spacing, surfaces, -1.0, 0.0)
    w = Workload("C3 grating DOE + two singlets, fwd+bwd", system, jobs, z_start=-1.0)
    w.target = maps.gaussian_spots_target(1, 256, 256, seed=2003, n_spots=4)
    return w


# --------------------------------------------------------------------------
# C4: conformal DOE behind an even asphere
# --------------------------------------------------------------------------
def c4(n_side=2048, D=64, lams=(486e-6, 550e-6, 656e-6), n_fields=9,
       max_field_deg=30.0, map_side=4096, seed=1508):
    pitch = 0.5 * UM
    amp, phi = maps.random_amp_phase(map_side, map_side, seed)
    doe = DOE(phi=phi, amp=amp, pitch=pitch, D=D, lambda0=550e-6, kind=CONFORMAL,
              gather="bilinear")
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    A = tuple(float(a) for a in rng.normal(0.0, 1e-6, 4))
    asph = Surface(ASPHERE, 0.0, c=1.0 / 20.0, k=-1.0, A=A, n_after=N_BK7, r_ap=12.0)
    back = Surface(PLANE, 3.0, n_after=1.0, r_ap=12.0)
    doe_s = Surface(SPHERE, 8.0, c=1.0 / 25.0, n_after=1.0)
    surfaces = [asph, back, doe_s]
    zs = back_focal_z([asph, back])
    sensor = Sensor(z=zs, nx=512, ny=512, pitch=2 * UM)
    system = System(surfaces=surfaces, doe_index=2, doe=doe, sensor=sensor)
    spacing = 0.75 * UM * 2048 / n_side
    fl = np.linspace(-max_field_deg, max_field_deg, n_fields)
    jobs = _grid_jobs(list(lams), [(0.0, math.radians(f)) for f in fl], n_side, spacing,
                      surfaces, -1.0, 8.0, sensor_z=zs, center_sensor=True)
    return Workload("C4 conformal DOE (R=25 mm) behind an even asphere", system, jobs,
                    z_start=-1.0)


# --------------------------------------------------------------------------
# C5: batched optimisation workload
# --------------------------------------------------------------------------
def c5(n_lams=31, n_fields=16, count_lo=65536, count_hi=2 * 1024 * 1024, D=96,
       n_ssr=1024, seed=1509, map_side=2048, sensor_n=512):
    pitch = 1 * UM
    phi = _c2_phase(map_side, map_side, pitch)
    doe = DOE(phi=phi, pitch=pitch, D=D, lambda0=550e-6, emit="sampled", n_ssr=n_ssr,
              seed=seed)
    surfaces = [Surface(PLANE, 0.0)] + _singlet(5.0) + _singlet(10.0) + _singlet(15.0)
    zs = back_focal_z(surfaces[1:])
    sensor = Sensor(z=zs, nx=sensor_n, ny=sensor_n, pitch=2 * UM)
    system = System(surfaces=surfaces, doe_index=0, doe=doe, sensor=sensor)
    rng = np.random.Generator(np.random.PCG64(seed))
    lams = np.linspace(400e-6, 700e-6, n_lams)
    side = int(round(math.sqrt(n_fields)))
    fl = np.linspace(-1.5, 1.5, side)
    fields = [(math.radians(a), math.radians(b)) for b in fl for a in fl]
    jobs = []
    for lam in lams:
        for (tx, ty) in fields:
            cnt = math.exp(rng.uniform(math.log(count_lo), math.log(count_hi)))
            n_side = max(1, int(round(math.sqrt(cnt))))
            spacing = map_side * pitch / n_side
            x0 = chief_aim(surfaces, -1.0, 0.0, math.tan(tx))
            y0 = chief_aim(surfaces, -1.0, 0.0, math.tan(ty))
            jobs.append(Job(lam=float(lam), theta_x=tx, theta_y=ty, grid_n=n_side,
                            spacing=spacing, x0=x0, y0=y0))
    w = Workload("C5 31 lambda x 16 fields, uneven counts, sampled emission", system,
                 jobs, z_start=-1.0)
    w.target = maps.gaussian_spots_target(len(jobs), sensor_n, sensor_n, seed=2005,
                                          n_spots=3)
    return w
