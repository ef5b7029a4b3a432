"""The ray -> wave -> ray step at a DOE, float64 (oracle).

Follows section "Ray-Wave Simulator Formalism", second paragraph and Eq. 1:
a tangent frame (u, v, n) at the ray-DOE intersection; a square D x D patch
of U = A exp(i phi) centred on the hit point; its Fourier transform U~(k_u, k_v);
evanescent components (k_u^2 + k_v^2 >= k^2) discarded; each secondary ray
carries a = U~ / p (Eq. 1) and points along its wavevector; sampling draws
wavevectors by Gumbel-max with a softmax relaxation for gradients (third
paragraph of the same section).

Readings (the paper does not fix these):
* spectrum: U~_j = c sum_{a,b} T_ab exp(-i (k_ju s_a + k_jv t_b)), with
  (s_a, t_b) the tangent-plane offsets of sample (a, b) from the hit point;
  without padding c = 1/D^2: the Fourier-series coefficient of the patch
  referenced to the hit point, and sum_j |U~_j|^2 = mean |T|^2 (Parseval);
* zero padding (section "Benchmark and Inverse Design Demonstrations": patches
  padded to a larger area for a finer angular spectrum): the D x D samples
  are transformed on the grid of M = P D; a coherent sensor takes
  c = 1/M^2 (the Fourier-series coefficient of the padded, M-periodic
  patch, so the wavelet sum reproduces the padded field), an incoherent one
  c = 1/(D M) (so that sum_j |U~_j|^2 = mean |T|^2 stays the ray's power);
* k-grid: k_j = 2 pi j / (M p), j in [-M/2, M/2);
* planar patch (gather 'nearest'): columns floor(x/p + W/2) - D/2 .. + D/2 - 1,
  rows likewise, offsets = pixel centres minus the hit point, so a binary map
  stays binary; conformal patch (gather 'bilinear'): samples at
  P + s_a u + t_b v with s_a = (a - D/2) p, t_b = (b - D/2) p, looked up
  bilinearly on the complex transmission at their orthographic (x, y)
  (the map is "projected to a flat xy-plane"); outside the map T = 0;
* the incident ray enters through its tangential wavevector: the outgoing
  tangential wavevector is kappa = k0 n_in (d.u, d.v) + k_j, which is the
  spectrum of the patch multiplied by the incident plane wave, exactly;
* kept bins: |kappa|^2 < (k0 n_out)^2; direction
  d' = (kappa_u u + kappa_v v + sqrt((k0 n_out)^2 - |kappa|^2) n) / (k0 n_out)
  with n oriented along the incident ray; origin = hit point; OPL unchanged;
* exhaustive mode is Eq. 1 with the uniform density over all M^2 bins and
  one stratum per bin: a = a_in U~_j;
* sampled mode draws N bins from p over the propagating bins by Gumbel-max
  (Philox4x32-10 noise); coherent sensor: p ~ |U~|, a = a_in U~ / (N p);
  incoherent sensor: p ~ |U~|^2 and |a|^2 = |a_in|^2 |U~|^2 / (N p) with the
  phase of U~ (the unbiased power weight); 'sampled_uniform' draws from the
  uniform density over the propagating bins instead (the paper's p_uni,
  convergence section), with the same weights;
* phase at wavelength lambda: 'height' model phi * lambda0 / lambda, or 'fixed';
* reflective DOE (section "Benchmark and Inverse Design Demonstrations",
  reflective conformal DOE): the same frame and spectrum, the outgoing
  normal component reversed, d' = (kappa_u u + kappa_v v - kn n) / (k0 n_in),
  so secondary rays return into the incident medium (T = 1: the law of
  reflection);
* two superposed phase profiles (the same section's complex-amplitude
  field): U = A (exp(i phi) + exp(i phi2)).
"""
import math

import numpy as np
import torch

from .geometry import normal
from .philox import sample_uniforms

TWO_PI = 2.0 * math.pi


def frame(hit, doe_surface, d_in):
    """Tangent frame at the hit: planar -> (x, y, z); curved ->
    n = surface normal, u = normalise(x - (x.n) n), v = n x u; n is oriented
    along the incident direction (transmission)."""
    N = hit.shape[0]
    n, _ = normal(hit[:, 0], hit[:, 1], doe_surface)
    flip = (n * d_in).sum(-1) < 0
    n = torch.where(flip[:, None], -n, n)
    ex = torch.zeros(N, 3, dtype=hit.dtype)
    ex[:, 0] = 1.0
    u = ex - (ex * n).sum(-1, keepdim=True) * n
    u = u / torch.linalg.norm(u, dim=-1, keepdim=True)
    v = torch.cross(n, u, dim=-1)
    return u, v, n


def transmission(phi, amp, rows, cols, lam, doe, phi2=None):
    """T = A exp(i phi_lambda) (+ A exp(i phi2_lambda)) at integer pixel
    indices, 0 outside the map."""
    H, W = phi.shape
    inside = (rows >= 0) & (rows < H) & (cols >= 0) & (cols < W)
    r = rows.clamp(0, H - 1)
    c = cols.clamp(0, W - 1)
    scale = doe.lambda0 / lam if doe.phase_model == "height" else 1.0
    ph = phi[r, c] * scale
    T = torch.polar(torch.ones_like(ph), ph)
    if phi2 is not None:
        ph2 = phi2[r, c] * scale
        T = T + torch.polar(torch.ones_like(ph2), ph2)
    if amp is not None:
        T = T * amp[r, c]
    return torch.where(inside, T, torch.zeros_like(T))


def gather_nearest(hit, phi, amp, lam, doe, phi2=None):
    """Planar nearest-pixel patch.  Returns T [N, D(rows b), D(cols a)],
    offsets s [N, D] (along u = x) and t [N, D] (along v = y)."""
    D, p = doe.D, doe.pitch
    H, W = phi.shape
    x, y = hit[:, 0], hit[:, 1]
    cstar = torch.floor(x.detach() / p + W / 2).long()
    rstar = torch.floor(y.detach() / p + H / 2).long()
    ar = torch.arange(D)
    cols = cstar[:, None] - D // 2 + ar[None, :]
    rows = rstar[:, None] - D // 2 + ar[None, :]
    T = transmission(phi, amp, rows[:, :, None], cols[:, None, :], lam, doe, phi2)
    s = (cols.to(torch.float64) - W / 2 + 0.5) * p - x[:, None]
    t = (rows.to(torch.float64) - H / 2 + 0.5) * p - y[:, None]
    return T, s, t


def gather_bilinear(hit, u, v, phi, amp, lam, doe, phi2=None):
    """Bilinear complex patch at P + s_a u + t_b v (orthographic map lookup)."""
    D, p = doe.D, doe.pitch
    H, W = phi.shape
    off = (torch.arange(D, dtype=torch.float64) - D // 2) * p          # [D]
    # sample (b, a) -> point P + off[a] u + off[b] v
    q = (hit[:, None, None, :] + off[None, None, :, None] * u[:, None, None, :]
         + off[None, :, None, None] * v[:, None, None, :])            # [N, D, D, 3]
    uc = q[..., 0] / p + W / 2 - 0.5
    vc = q[..., 1] / p + H / 2 - 0.5
    i0 = torch.floor(uc.detach()).long()
    j0 = torch.floor(vc.detach()).long()
    fu = uc - i0
    fv = vc - j0
    T = ((1 - fu) * (1 - fv) * transmission(phi, amp, j0, i0, lam, doe, phi2)
         + fu * (1 - fv) * transmission(phi, amp, j0, i0 + 1, lam, doe, phi2)
         + (1 - fu) * fv * transmission(phi, amp, j0 + 1, i0, lam, doe, phi2)
         + fu * fv * transmission(phi, amp, j0 + 1, i0 + 1, lam, doe, phi2))
    N = hit.shape[0]
    s = off[None, :].expand(N, D)
    return T, s, s.clone()


def kgrid(M, pitch):
    j = torch.arange(-(M // 2), M - M // 2, dtype=torch.float64)
    return TWO_PI * j / (M * pitch)


def spectrum(T, s, t, pitch, M=None, coherent=False):
    """Direct separable DFT on the k-grid of size M (default D, no padding):
    U~[jv, ju] = c sum_b sum_a exp(-i k_jv t_b) T[b, a] exp(-i k_ju s_a),
    c = 1/M^2 (coherent sensor) or 1/(D M) (incoherent); both 1/D^2 at M = D.
    The zero samples of a padded patch add nothing to the sums."""
    D = T.shape[-1]
    M = D if M is None else int(M)
    k = kgrid(M, pitch)
    Eu = torch.polar(torch.ones(1, dtype=torch.float64), -(k[None, :, None] * s[:, None, :]))
    Ev = torch.polar(torch.ones(1, dtype=torch.float64), -(k[None, :, None] * t[:, None, :]))
    c = 1.0 / (M * M) if coherent else 1.0 / (D * M)
    # [N, M, D] @ [N, D, D] @ [N, D, M]
    return (Ev @ T @ Eu.transpose(1, 2)) * c


def outgoing(d_in, u, v, n, k0, n_in, n_out, M, pitch):
    """Directions of all bins: d' [N, M(jv), M(ju), 3] and the propagating mask."""
    k = kgrid(M, pitch)
    ku_in = k0 * n_in * (d_in * u).sum(-1)
    kv_in = k0 * n_in * (d_in * v).sum(-1)
    kap_u = ku_in[:, None, None] + k[None, None, :]
    kap_v = kv_in[:, None, None] + k[None, :, None]
    K = k0 * n_out
    kt2 = kap_u ** 2 + kap_v ** 2
    prop = kt2 < K * K
    kn = torch.sqrt(torch.where(prop, K * K - kt2, torch.ones_like(kt2)))
    dvec = (kap_u[..., None] * u[:, None, None, :] + kap_v[..., None] * v[:, None, None, :]
            + kn[..., None] * n[:, None, None, :]) / K
    return dvec, prop


def doe_step(ray, doe_surface, doe, phi, amp, lam, n_in, n_out, ray_ids=None,
             coherent=False, phi2=None):
    """Intersect the DOE, build the patch spectrum and emit secondary rays.

    Exhaustive mode: returns a dict with d [N, M, M, 3], a [N, M, M],
    alive [N, M, M], o [N, 3] (hit point), opl [N], U [N, M, M].
    Sampled mode: same with the bin axis replaced by [N, n_ssr] draws.
    """
    from .geometry import intersect
    o, d = ray["o"], ray["d"]
    tt, ok = intersect(o, d, doe_surface)
    hit = o + tt[:, None] * d
    opl = ray["opl"] + n_in * tt
    u, v, nrm = frame(hit, doe_surface, d)
    if getattr(doe, "reflective", False):
        nrm = -nrm                       # outgoing side: back into the incident medium
        n_out = n_in
    if doe.gather == "nearest":
        T, s, t = gather_nearest(hit, phi, amp, lam, doe, phi2)
    else:
        T, s, t = gather_bilinear(hit, u, v, phi, amp, lam, doe, phi2)
    M = doe.pad * doe.D
    U = spectrum(T, s, t, doe.pitch, M=M, coherent=coherent)
    k0 = TWO_PI / lam
    dvec, prop = outgoing(d, u, v, nrm, k0, n_in, n_out, M, doe.pitch)
    alive_in = ray["alive"] & ok
    base = {"o": hit, "opl": opl, "U": U, "frame": (u, v, nrm)}
    if doe.emit == "exhaustive":
        a = ray["a"][:, None, None] * U
        base.update(d=dvec, a=a, alive=alive_in[:, None, None] & prop)
        return base
    # ---- sampled: Gumbel-max over propagating bins, straight-through softmax ----
    N = o.shape[0]
    nb = M * M
    Uf = U.reshape(N, nb)
    propf = prop.reshape(N, nb)
    if doe.emit == "sampled_uniform":
        # the uniform density over the propagating bins (p_uni)
        mag = torch.ones_like(Uf.real)
    else:
        mag = Uf.abs() ** (2 if not coherent else 1)
    mag = torch.where(propf, mag, torch.zeros_like(mag))
    tot = mag.sum(-1, keepdim=True)
    pj = mag / torch.where(tot > 0, tot, torch.ones_like(tot))
    logp = torch.where(pj > 0, torch.log(torch.where(pj > 0, pj, torch.ones_like(pj))),
                       torch.full_like(pj, -math.inf))
    ns = doe.n_ssr
    ids = np.arange(N) if ray_ids is None else np.asarray(ray_ids)
    uni = torch.from_numpy(sample_uniforms(doe.seed, doe.rng_offset, ids, ns, nb))
    g = -torch.log(-torch.log(uni))                                   # [N, ns, nb]
    score = logp[:, None, :] + g
    idx = torch.argmax(score.detach(), dim=-1)                         # [N, ns]
    soft = torch.softmax(torch.where(torch.isfinite(score), score,
                                     torch.full_like(score, -1e300)), dim=-1)
    hard = torch.nn.functional.one_hot(idx, nb).to(soft.dtype)
    y = hard + soft - soft.detach()                                    # straight-through
    if coherent:
        w = Uf / (ns * torch.where(pj > 0, pj, torch.ones_like(pj)))
    else:
        w = Uf / torch.sqrt(ns * torch.where(pj > 0, pj, torch.ones_like(pj)))
    w = torch.where(propf, w, torch.zeros_like(w))
    a = ray["a"][:, None] * (y.to(w.dtype) @ w[:, :, None])[..., 0]
    dflat = dvec.reshape(N, nb, 3)
    dsel = y @ dflat                                                   # [N, ns, 3]
    anyp = propf.any(-1)
    base.update(d=dsel, a=a, alive=(alive_in & anyp)[:, None].expand(N, ns),
                idx=idx, p=pj)
    return base
