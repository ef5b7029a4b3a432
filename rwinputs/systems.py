"""Plain data descriptions of a hybrid refractive-diffractive system.

Units are millimetres throughout; wavelengths are vacuum wavelengths in mm
(550 nm = 550e-6).  The optical axis is +z and light travels towards +z.

Surfaces are sequential.  One of them carries the DOE (`System.doe_index`);
its geometry (plane for a planar DOE, sphere for a conformal DOE) is the
surface entry, its transmission map lives in `System.doe`.
"""
from dataclasses import dataclass
from typing import List, Optional, Tuple

import numpy as np

PLANE, SPHERE, ASPHERE, GAUSS = 0, 1, 2, 3
PLANAR, CONFORMAL = 0, 1


@dataclass
class Surface:
    """One refracting surface (vertex form, rotationally symmetric).

    kind: PLANE, SPHERE (curvature c) or ASPHERE (even asphere: conic k and
    A4..A10 polynomial terms on r^2); GAUSS only as the substrate of a
    conformal DOE: a Gaussian bump z - z = c exp(-r^2 / (2 k^2)) of height c
    and width k.  n_after is the refractive index of the
    medium behind the surface.  r_ap > 0 clips rays whose hit radius exceeds
    it; r_ap <= 0 means no clip.  sellmeier = (B1, B2, B3, C1, C2, C3), C in
    um^2, makes that medium dispersive: at vacuum wavelength lambda its index
    is sqrt(1 + sum_i B_i lambda^2 / (lambda^2 - C_i)) (lambda in um) and
    n_after is not used.
    """
    kind: int
    z: float
    c: float = 0.0
    k: float = 0.0
    A: Tuple[float, float, float, float] = (0.0, 0.0, 0.0, 0.0)
    n_after: float = 1.0
    r_ap: float = 0.0
    sellmeier: Optional[Tuple[float, float, float, float, float, float]] = None


@dataclass
class DOE:
    """Transmission map of the diffractive element, U = A exp(i phi).

    phi: float32 [H, W] phase in radians at the design wavelength lambda0.
    amp: float32 [H, W] or None (amplitude 1).
    Pixel (r, c) has its centre at x = (c - W/2 + 1/2) p, y = (r - H/2 + 1/2) p,
    i.e. the map is centred on the optical axis and rows run along y.
    phase_model 'height': phi_lambda = phi * lambda0 / lambda; 'fixed': phi.
    gather 'nearest' (planar default) or 'bilinear' (conformal default).
    emit 'exhaustive' (one secondary ray per propagating bin), 'sampled'
    (n_ssr Gumbel-max draws from p ~ |U~|, |U~|^2 for an incoherent sensor) or
    'sampled_uniform' (n_ssr draws from the uniform density over the
    propagating bins).
    pad P >= 1: the D x D patch is zero-padded to M = P D samples before its
    transform, so the spectrum is sampled on the finer k-grid 2 pi j / (M p).
    reflective: the DOE reflects; secondary rays leave on the incident side
    (outgoing normal component reversed, index n_in); it must be the last
    surface and the sensor lies in front of it.
    phi2: optional second phase map [H, W]: U = A (exp(i phi) + exp(i phi2)),
    the complex-amplitude field of two superposed phase profiles.
    """
    phi: np.ndarray
    pitch: float
    D: int
    lambda0: float = 550e-6
    amp: Optional[np.ndarray] = None
    kind: int = PLANAR
    phase_model: str = "height"
    gather: str = "nearest"
    emit: str = "exhaustive"
    n_ssr: int = 0
    seed: int = 0
    rng_offset: int = 0
    pad: int = 1
    reflective: bool = False
    phi2: Optional[np.ndarray] = None

    @property
    def M(self):
        return int(self.pad) * int(self.D)

    @property
    def H(self):
        return int(self.phi.shape[0])

    @property
    def W(self):
        return int(self.phi.shape[1])


@dataclass
class Sensor:
    """Sensor plane z = const, nx x ny pixels at `pitch`.

    Pixel (i, j) of job J has its centre at
    x = cx_J + (i - nx/2 + 1/2) pitch, y = cy_J + (j - ny/2 + 1/2) pitch,
    where (cx_J, cy_J) is the job's window centre.  coherent=False deposits
    |a|^2 bilinearly; coherent=True evaluates the plane-wavelet sum of Eq. 2
    over a window of +-`window` pixels (0 = whole sensor).
    """
    z: float
    nx: int
    ny: int
    pitch: float
    coherent: bool = False
    window: int = 0


@dataclass
class System:
    surfaces: List[Surface]
    doe_index: int
    doe: DOE
    sensor: Sensor
    n_object: float = 1.0


@dataclass
class Job:
    """One (wavelength, field) pair and its collimated ray bundle.

    Field angles in radians; every ray of the job has direction
    normalise(tan(theta_x), tan(theta_y), 1).  The bundle is a grid_n x grid_n
    square grid at `spacing` in the launch plane z = z_start of the workload,
    centred at (x0, y0); ray (ix, iy) has index iy * grid_n + ix and starts at
    x = x0 + (ix - (grid_n - 1)/2) spacing, y = y0 + (iy - (grid_n - 1)/2) spacing.
    Amplitude 1; the starting optical path is n_object * (d . o), the phase of
    the incident plane wave at the start point.
    """
    lam: float
    theta_x: float = 0.0
    theta_y: float = 0.0
    grid_n: int = 1
    spacing: float = 0.0
    x0: float = 0.0
    y0: float = 0.0
    sensor_cx: float = 0.0
    sensor_cy: float = 0.0

    @property
    def n_rays(self):
        return int(self.grid_n) * int(self.grid_n)


def jobs_offsets(jobs: List[Job]) -> np.ndarray:
    """Exclusive prefix sum of ray counts (int64 [njob + 1])."""
    off = np.zeros(len(jobs) + 1, dtype=np.int64)
    for i, j in enumerate(jobs):
        off[i + 1] = off[i] + int(j.n_rays)
    return off


@dataclass
class Workload:
    """A system plus its jobs and ray grid: everything one step consumes."""
    name: str
    system: System
    jobs: List[Job]
    z_start: float = -1.0
    target: Optional[np.ndarray] = None   # float32 [njob, ny, nx] for Eq. 3

    @property
    def n_rays(self):
        return int(sum(j.n_rays for j in self.jobs))


def ray_blocks(jobs: List[Job], per_job: int, seed: int):
    """Seeded sample of incident rays for spot checks at full workload size:
    per job one contiguous run of `per_job` ray indices (along grid rows)
    starting at a random index.  Returns (starts [njob] int64, subsets
    list of index arrays).  A contiguous run keeps every sampled ray at its
    own index, so a launch over [offset + start, offset + start + per_job)
    draws the same sampling stream as the whole workload."""
    rng = np.random.default_rng(seed)
    starts, subsets = [], []
    for j in jobs:
        n = int(j.n_rays)
        m = min(per_job, n)
        s0 = int(rng.integers(0, n - m + 1))
        starts.append(s0)
        subsets.append(np.arange(s0, s0 + m, dtype=np.int64))
    return np.asarray(starts, dtype=np.int64), subsets
