"""Seeded synthetic inputs shared by the CUDA path, the FP64 oracle and the tests.

This package only describes optical systems and draws the seeded arrays
(DOE maps, job tables, targets).  It holds none of the ray-wave method's
arithmetic: no tracing, no patch transform, no emission and no splatting.
Both sides read exactly the same float32 arrays produced here.
"""
from .systems import (  # noqa: F401
    Surface, DOE, Sensor, System, Job, Workload, jobs_offsets, ray_blocks,
    PLANE, SPHERE, ASPHERE, GAUSS, PLANAR, CONFORMAL,
)
from .maps import (  # noqa: F401
    binary_grating, staircase_grating, zernike_holographic_phase,
    random_amp_phase, gaussian_spots_target,
)
from . import configs  # noqa: F401
