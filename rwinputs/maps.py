"""Seeded DOE maps and target images (float32, row index = y, column = x).

All generators are deterministic functions of their arguments and a seed
(NumPy PCG64).  They only synthesise input data.
"""
import math

import numpy as np


def binary_grating(H, W, period_px, duty=0.5, axis="x", levels=(0.0, math.pi)):
    """1D binary phase grating: phase levels[0] on the first `duty` fraction of
    each period, levels[1] on the rest; lines run perpendicular to `axis`."""
    idx = np.arange(W if axis == "x" else H)
    first = (idx % period_px) < int(round(duty * period_px))
    line = np.where(first, levels[0], levels[1]).astype(np.float32)
    if axis == "x":
        return np.broadcast_to(line[None, :], (H, W)).copy()
    return np.broadcast_to(line[:, None], (H, W)).copy()


def staircase_grating(H, W, n_levels, px_per_level, axis="x"):
    """Blazed N-level staircase: level l = floor(i / q) mod N has phase 2 pi l / N."""
    idx = np.arange(W if axis == "x" else H)
    lvl = (idx // px_per_level) % n_levels
    line = (2.0 * math.pi * lvl / n_levels).astype(np.float32)
    if axis == "x":
        return np.broadcast_to(line[None, :], (H, W)).copy()
    return np.broadcast_to(line[:, None], (H, W)).copy()


def _noll_to_nm(j):
    """Noll index (j >= 1) to radial order n and signed azimuthal order m."""
    n, j1 = 0, j - 1
    while j1 > n:
        n += 1
        j1 -= n
    m = (n % 2) + 2 * ((j1 + ((n + 1) % 2)) // 2)
    if j % 2 == 1:
        m = -m
    return n, m


def _zernike_radial(n, m, rho):
    m = abs(m)
    out = np.zeros_like(rho)
    for s in range((n - m) // 2 + 1):
        coef = ((-1) ** s * math.factorial(n - s)
                / (math.factorial(s) * math.factorial((n + m) // 2 - s)
                   * math.factorial((n - m) // 2 - s)))
        out += coef * rho ** (n - 2 * s)
    return out


def zernike_holographic_phase(H, W, pitch, seed, n_modes=64, n_holo=256,
                              f_max_per_mm=400.0, holo_amp=math.pi / 16):
    """Phase map (radians, wrapped to [0, 2 pi)) = sum of `n_modes` Zernike
    modes (Noll 2 .. n_modes+1, coefficients ~ N(0, 1) rad) on the disk whose
    radius is the map half-diagonal, plus a holographic term
    sum_q holo_amp * cos(2 pi f_q . r + psi_q) with |f_q| ~ U[0, f_max],
    orientation and psi_q ~ U[0, 2 pi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = (np.arange(W) - W / 2 + 0.5) * pitch
    y = (np.arange(H) - H / 2 + 0.5) * pitch
    rad = math.hypot(W * pitch / 2, H * pitch / 2)
    X, Y = np.meshgrid(x / rad, y / rad)
    rho = np.hypot(X, Y)
    th = np.arctan2(Y, X)
    coef = rng.standard_normal(n_modes)
    phase = np.zeros((H, W))
    for i in range(n_modes):
        n, m = _noll_to_nm(i + 2)
        R = _zernike_radial(n, m, rho)
        if m > 0:
            phase += coef[i] * R * np.cos(m * th)
        elif m < 0:
            phase += coef[i] * R * np.sin(-m * th)
        else:
            phase += coef[i] * R
    fmag = rng.uniform(0.0, f_max_per_mm, n_holo)
    fang = rng.uniform(0.0, 2 * math.pi, n_holo)
    psi = rng.uniform(0.0, 2 * math.pi, n_holo)
    fx = fmag * np.cos(fang)
    fy = fmag * np.sin(fang)
    # cos(ax + by + psi) = cos(ax) cos(by + psi) - sin(ax) sin(by + psi): the sum
    # over q is then two (H x n_holo) @ (n_holo x W) products.
    ax = 2 * math.pi * np.outer(x, fx)              # [W, q]
    by = 2 * math.pi * np.outer(y, fy) + psi[None]  # [H, q]
    phase += holo_amp * (np.cos(by) @ np.cos(ax).T - np.sin(by) @ np.sin(ax).T)
    return np.mod(phase, 2 * math.pi).astype(np.float32)


def random_amp_phase(H, W, seed, amp_lo=0.2, amp_hi=1.0):
    """IID per-pixel amplitude ~ U[amp_lo, amp_hi] and phase ~ U[0, 2 pi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    amp = rng.uniform(amp_lo, amp_hi, (H, W)).astype(np.float32)
    phi = rng.uniform(0.0, 2 * math.pi, (H, W)).astype(np.float32)
    return amp, phi


def random_phase(H, W, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.0, 2 * math.pi, (H, W)).astype(np.float32)


def gaussian_spots_target(njob, ny, nx, seed, n_spots=6, sigma_px=(3.0, 12.0)):
    """Seeded target intensity per job: a sum of isotropic Gaussian spots."""
    rng = np.random.Generator(np.random.PCG64(seed))
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    out = np.zeros((njob, ny, nx), dtype=np.float64)
    for jb in range(njob):
        for _ in range(n_spots):
            cx = rng.uniform(0.25, 0.75) * nx
            cy = rng.uniform(0.25, 0.75) * ny
            s = rng.uniform(*sigma_px)
            w = rng.uniform(0.5, 1.0)
            out[jb] += w * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * s * s))
    return out.astype(np.float32)
