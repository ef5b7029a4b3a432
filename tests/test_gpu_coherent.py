"""Coherent sensor (Eq. 2) at scale on the GPU.

1. One patch covering a whole 64 x 64 map, zero-padded to M = 128 (16,384
   secondary rays summed over 4,096 sensor pixels): the wavelet sum equals
   the angular-spectrum propagation of the zero-padded field (NumPy FFT), the
   same identity the oracle is pinned to.
2. Many overlapping patches (64 rays, D = 32, P = 2: 4,096 secondary rays
   each) summed over the whole sensor, against the FP64 oracle.  (A windowed
   sum decides each ray's window from its rounded hit pixel; near a pixel
   boundary FP32 and FP64 can round differently and move a whole
   contribution, so parity at scale is checked on the full sum.)
"""
import math

import numpy as np
import pytest
import torch

import rwinputs as R

from gpu_helpers import oracle_psf, rel_l2
from physics_refs import asm_propagate

pytestmark = pytest.mark.gpu


def test_padded_full_patch_wavelet_sum_equals_angular_spectrum_m128():
    from paper_2605_15418_gb300 import raywave as RW
    D, P, p, lam, zs = 64, 2, 1e-3, 0.8e-3, 0.03
    M = P * D
    rng = np.random.Generator(np.random.PCG64(8))
    phi = rng.uniform(0, 2 * math.pi, (D, D)).astype(np.float32)
    amp = rng.uniform(0.3, 1.0, (D, D)).astype(np.float32)
    doe = R.DOE(phi=phi, amp=amp, pitch=p, D=D, lambda0=lam, pad=P)
    sen = R.Sensor(z=zs, nx=D, ny=D, pitch=p, coherent=True)
    sysm = R.System([R.Surface(R.PLANE, 0.0)], 0, doe, sen)
    job = R.Job(lam=lam, grid_n=1, spacing=0.0, x0=0.31 * p, y0=0.77 * p)
    w = R.systems.Workload("full patch M=128", sysm, [job], z_start=-0.01)
    sim = RW.Simulator(w)
    img = sim.forward().cpu().numpy()[0]
    Tpad = np.zeros((M, M), np.complex128)
    Tpad[:D, :D] = amp.astype(np.float64) * np.exp(1j * phi.astype(np.float64))
    ref = np.abs(asm_propagate(Tpad, p, lam, zs)[:D, :D]) ** 2
    assert rel_l2(img, ref) <= 1e-4, rel_l2(img, ref)


def test_coherent_overlapping_patches_padded_against_oracle():
    from paper_2605_15418_gb300 import raywave as RW
    w = R.configs.c2(n_side=8, D=32, lams=(550e-6,), fields_deg=(0.3,), sensor_n=32,
                     map_side=128)
    w.system.surfaces = w.system.surfaces[:1]          # DOE alone, sensor 0.2 mm behind
    w.system.doe.pad = 2
    w.system.sensor.z = 0.2
    w.system.sensor.pitch = 2e-3
    w.system.sensor.coherent = True
    w.system.sensor.window = 0
    sim = RW.Simulator(w)
    psf = sim.forward().cpu().numpy()
    ref = oracle_psf(w)
    assert ref.sum() > 0
    assert rel_l2(psf, ref) <= 1e-3, rel_l2(psf, ref)
