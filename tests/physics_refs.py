"""Independent physics references used to pin the oracle (NumPy, float64).

None of this calls the oracle: the angular-spectrum propagator is written
from Fourier optics (Goodman, "Introduction to Fourier Optics", ch. 3) on
NumPy's FFT, the thick-lens focus from the lensmaker's equation, and the
grating efficiencies from the Fourier series of a staircase.
"""
import math

import numpy as np


def asm_propagate(T, pitch, lam, z, obliquity=True):
    """Angular-spectrum propagation of the field T (sampled at pixel centres)
    over distance z in vacuum; evanescent components removed.  With
    obliquity=True each plane wave is also weighted by k_z / k, the
    projection factor <n, d> of the wavelet sum."""
    Hh, Ww = T.shape
    k0 = 2 * math.pi / lam
    fx = np.fft.fftfreq(Ww, d=pitch) * 2 * math.pi
    fy = np.fft.fftfreq(Hh, d=pitch) * 2 * math.pi
    # fftfreq gives +N/2-1 .. -N/2 ; the Nyquist bin sits at -N/2 as in the oracle
    KX, KY = np.meshgrid(fx, fy)
    kz2 = k0 * k0 - KX ** 2 - KY ** 2
    prop = kz2 > 0
    kz = np.sqrt(np.where(prop, kz2, 0.0))
    H = np.where(prop, np.exp(1j * kz * z), 0.0)
    if obliquity:
        H = H * kz / k0
    return np.fft.ifft2(np.fft.fft2(T) * H)


def thick_lens_bfl(n, R1, R2, ct):
    """Back focal distance of a thick singlet in air (lensmaker's equation)."""
    inv_f = (n - 1) * (1 / R1 - 1 / R2 + (n - 1) * ct / (n * R1 * R2))
    f = 1 / inv_f
    return f * (1 - (n - 1) * ct / (n * R1)), f


def binary_grating_efficiency(m, period_px):
    """Pixelated 0/pi 50% grating: |c_m|^2 of its Fourier series."""
    if m % 2 == 0:
        return 0.0
    return (2.0 / (period_px * math.sin(math.pi * m / period_px))) ** 2


def staircase_efficiency(m, n_levels, q):
    """N-level staircase with q pixels per level: nonzero for m = 1 mod N."""
    if (m - 1) % n_levels != 0:
        return 0.0
    return (math.sin(math.pi * m / n_levels) ** 2
            / (q * q * math.sin(math.pi * m / (n_levels * q)) ** 2))
