"""Sensor reconstruction, float64 (oracle).

Incoherent: each ray deposits |a|^2 on the four pixels around its hit point
with bilinear weights (pixel centres at cx + (i - nx/2 + 1/2) pitch); a tap
that falls off the sensor loses only its own share.

Coherent (Eq. 2, section "Ray-Wave Simulator Formalism"):
    U(x, y) = sum_i a_i exp(i k (OPL_i + dr_i(x, y))) <n, d_i>
with k = 2 pi / lambda, OPL_i the optical path up to the sensor hit r_i,
dr_i(x, y) = n_s d_t,i . ((x, y) - r_i) the extra path of the tilted wavelet
across the sensor (d_t the transverse part of the direction, n_s the index
at the sensor) and <n, d_i> = d_z,i for the sensor normal +z.  A window of
+-W pixels around each ray's hit pixel limits the sum when W > 0.
"""
import math

import torch


def to_sensor(o, d, opl, z_s, n_s):
    t = (z_s - o[..., 2]) / d[..., 2]
    x = o[..., 0] + t * d[..., 0]
    y = o[..., 1] + t * d[..., 1]
    return x, y, opl + n_s * t


def splat_incoherent(x, y, w, alive, nx, ny, pitch, cx, cy):
    """Bilinear deposit of weights w at (x, y); returns a flat [ny*nx] image."""
    u = (x - cx) / pitch + nx / 2 - 0.5
    v = (y - cy) / pitch + ny / 2 - 0.5
    i0 = torch.floor(u.detach()).long()
    j0 = torch.floor(v.detach()).long()
    fu = u - i0
    fv = v - j0
    img = torch.zeros(nx * ny, dtype=torch.float64)
    for di, dj, wt in ((0, 0, (1 - fu) * (1 - fv)), (1, 0, fu * (1 - fv)),
                       (0, 1, (1 - fu) * fv), (1, 1, fu * fv)):
        i = i0 + di
        j = j0 + dj
        ok = alive & (i >= 0) & (i < nx) & (j >= 0) & (j < ny)
        idx = (j * nx + i)[ok]
        img = img.index_add(0, idx, (w * wt)[ok])
    return img


def coherent_field(x, y, opl, d, a, alive, nx, ny, pitch, cx, cy, lam, n_s, window=0,
                   chunk=4096):
    """Eq. 2 summed over rays; returns the complex field flat [ny*nx]."""
    k0 = 2.0 * math.pi / lam
    px = cx + (torch.arange(nx, dtype=torch.float64) - nx / 2 + 0.5) * pitch
    py = cy + (torch.arange(ny, dtype=torch.float64) - ny / 2 + 0.5) * pitch
    PX = px[None, :].expand(ny, nx).reshape(-1)
    PY = py[:, None].expand(ny, nx).reshape(-1)
    sel = alive.nonzero()[:, 0]
    field = torch.zeros(nx * ny, dtype=torch.complex128)
    for s0 in range(0, sel.numel(), chunk):
        ii = sel[s0:s0 + chunk]
        xr, yr, lr = x[ii], y[ii], opl[ii]
        dr = d[ii]
        ar = a[ii]
        ph = k0 * (lr[:, None] + n_s * (dr[:, 0:1] * (PX[None, :] - xr[:, None])
                                        + dr[:, 1:2] * (PY[None, :] - yr[:, None])))
        contrib = ar[:, None] * torch.polar(torch.ones_like(ph), ph) * dr[:, 2:3]
        if window > 0:
            iu = torch.round((xr - cx) / pitch + nx / 2 - 0.5)
            jv = torch.round((yr - cy) / pitch + ny / 2 - 0.5)
            ipx = torch.arange(nx, dtype=torch.float64)[None, :].expand(ny, nx).reshape(-1)
            jpx = torch.arange(ny, dtype=torch.float64)[:, None].expand(ny, nx).reshape(-1)
            m = ((ipx[None, :] - iu[:, None]).abs() <= window) & \
                ((jpx[None, :] - jv[:, None]).abs() <= window)
            contrib = torch.where(m, contrib, torch.zeros_like(contrib))
        field = field + contrib.sum(0)
    return field
