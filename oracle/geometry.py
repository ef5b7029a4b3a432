"""Sequential refractive ray tracing in float64 (oracle).

The paper traces rays between surfaces with "conventional ray tracing
principles" (section "Ray-Wave Simulator Formalism", first paragraph) and
gives no formulas; this module writes out the textbook ones:

* even-asphere sag in vertex form,
      z - z_v = c s / (1 + sqrt(1 - (1+k) c^2 s)) + A4 s^2 + A6 s^3 + A8 s^4 + A10 s^5,
  with s = x^2 + y^2 (a sphere is k = 0, A = 0; a plane is c = 0);
* ray-sphere intersection as the root of
      c (x^2 + y^2 + F^2) - 2 F = 0,   F = z - z_v,
  taken in the cancellation-free form t = C / q that tends to the plane
  root as c -> 0 (the vertex-side intersection);
* even-asphere intersection by Newton's method on
      g(t) = F(t) - sag(s(t))
  started from the base-sphere root, |dt| < 1e-13 mm or 50 iterations;
* the surface normal grad(z - z_v - sag) and vector Snell refraction
      d' = eta d + (sqrt(1 - eta^2 (1 - cos_i^2)) - eta cos_i) n,
  eta = n1 / n2, n oriented along d; total internal reflection drops the ray;
* optical path length OPL += n1 * t; a clear-aperture radius drops rays;
* a Gaussian bump z - z_v = c exp(-s / (2 k^2)) (height c, width k), the
  "Gaussian-like sag" substrate of a conformal DOE (section "Benchmark and
  Inverse Design Demonstrations", reflective conformal DOE), intersected by
  Newton's method on g(t) = F(t) - sag(s(t)) from the plane through the
  sag at the ray's current (x, y).

Rays are dicts of tensors: o [N,3], d [N,3], a complex [N], opl [N],
alive bool [N].  Dropped rays keep finite placeholder values.
"""
import torch

PLANE, SPHERE, ASPHERE, GAUSS = 0, 1, 2, 3
NEWTON_TOL = 1e-13
NEWTON_MAXIT = 50


def surface_params(s, requires_grad=False):
    """float64 scalar tensors for one rwinputs.Surface (leaves if requires_grad)."""
    def t(v):
        return torch.tensor(float(v), dtype=torch.float64, requires_grad=requires_grad)
    sm = getattr(s, "sellmeier", None)
    return {"kind": int(s.kind), "z": t(s.z), "c": t(s.c), "k": t(s.k),
            "A4": t(s.A[0]), "A6": t(s.A[1]), "A8": t(s.A[2]), "A10": t(s.A[3]),
            "n_after": t(s.n_after), "r_ap": float(s.r_ap),
            "sellmeier": None if sm is None else tuple(float(v) for v in sm),
            "n_after0": float(s.n_after)}


def sellmeier_index(coeffs, lam_mm):
    """Sellmeier dispersion formula: n^2 = 1 + sum_i B_i L^2 / (L^2 - C_i), with
    L the vacuum wavelength in micrometres and (B1, B2, B3, C1, C2, C3)."""
    L2 = (lam_mm * 1e3) ** 2
    B, C = coeffs[:3], coeffs[3:]
    return (1.0 + sum(b * L2 / (L2 - c) for b, c in zip(B, C))) ** 0.5


def at_wavelength(params, lam_mm):
    """Surface parameters at one wavelength: a dispersive medium gets its
    Sellmeier index, shifted by the n_after leaf's departure from the
    surface's nominal n_after -- an index shift common to every wavelength,
    zero at the nominal value, whose derivative is the sum over wavelengths
    of dL/dn."""
    out = []
    for p in params:
        if p.get("sellmeier") is None:
            out.append(p)
            continue
        q = dict(p)
        shift = p["n_after"] - p["n_after0"]
        q["n_after"] = sellmeier_index(p["sellmeier"], lam_mm) + shift
        out.append(q)
    return out


def sag(s, p):
    """Sag z - z_v at radius^2 s, its derivative d(sag)/ds, and the domain mask."""
    c, k = p["c"], p["k"]
    if p["kind"] == GAUSS:
        e = torch.exp(-s / (2.0 * k * k))
        return c * e, -c * e / (2.0 * k * k), torch.ones_like(s, dtype=torch.bool)
    arg = 1.0 - (1.0 + k) * c * c * s
    ok = arg > 0
    q = torch.sqrt(torch.where(ok, arg, torch.ones_like(arg)))
    z = (c * s / (1.0 + q) + p["A4"] * s ** 2 + p["A6"] * s ** 3
         + p["A8"] * s ** 4 + p["A10"] * s ** 5)
    dz = (c / (2.0 * q) + 2.0 * p["A4"] * s + 3.0 * p["A6"] * s ** 2
          + 4.0 * p["A8"] * s ** 3 + 5.0 * p["A10"] * s ** 4)
    return z, dz, ok


def _sphere_root(o, d, z_v, c):
    F0 = o[:, 2] - z_v
    A = c
    B = c * (o[:, 0] * d[:, 0] + o[:, 1] * d[:, 1] + F0 * d[:, 2]) - d[:, 2]
    C = c * (o[:, 0] ** 2 + o[:, 1] ** 2 + F0 ** 2) - 2.0 * F0
    disc = B * B - A * C
    ok = disc >= 0
    sq = torch.sqrt(torch.where(ok, disc, torch.zeros_like(disc)))
    sgn = torch.where(B >= 0, torch.ones_like(B), -torch.ones_like(B))
    q = -B - sgn * sq
    ok = ok & (q != 0)
    t = C / torch.where(q != 0, q, torch.ones_like(q))
    return t, ok


def _newton_g(t, o, d, p):
    x = o[:, 0] + t * d[:, 0]
    y = o[:, 1] + t * d[:, 1]
    s = x * x + y * y
    z, dz, ok = sag(s, p)
    g = o[:, 2] + t * d[:, 2] - p["z"] - z
    gp = d[:, 2] - dz * 2.0 * (x * d[:, 0] + y * d[:, 1])
    return g, gp, ok


def intersect(o, d, p):
    """Distance t along d to the surface and a validity mask."""
    kind = p["kind"]
    if kind == PLANE:
        ok = d[:, 2] != 0
        t = (p["z"] - o[:, 2]) / torch.where(ok, d[:, 2], torch.ones_like(d[:, 2]))
        return t, ok
    if kind == GAUSS:
        z0, _, _ = sag(o[:, 0] ** 2 + o[:, 1] ** 2, p)
        t = (p["z"] + z0 - o[:, 2]) / d[:, 2]
        ok = torch.ones_like(t, dtype=torch.bool)
    else:
        t, ok = _sphere_root(o, d, p["z"], p["c"])
    if kind == SPHERE:
        return t, ok
    # even asphere (Gaussian bump): Newton from the base-sphere root (from the
    # plane through the sag at the ray's (x, y)); the plane root if that fails;
    # iterate without autograd, then one differentiable step, whose derivative
    # at convergence is the implicit-function derivative -g_theta / g_t.
    with torch.no_grad():
        tp = (p["z"] - o[:, 2]) / d[:, 2]
        tn = torch.where(ok, t, tp).detach().clone()
        conv = torch.zeros_like(ok)
        good = torch.ones_like(ok)
        for _ in range(NEWTON_MAXIT):
            g, gp, okd = _newton_g(tn, o.detach(), d.detach(),
                                   {kk: (v.detach() if torch.is_tensor(v) else v)
                                    for kk, v in p.items()})
            good = good & okd & (gp != 0)
            step = torch.where(good & ~conv, g / torch.where(gp != 0, gp, torch.ones_like(gp)),
                               torch.zeros_like(g))
            tn = tn - step
            conv = conv | (step.abs() < NEWTON_TOL)
            if bool(conv[good].all()):
                break
    g, gp, okd = _newton_g(tn, o, d, p)
    t = tn - g / torch.where(gp != 0, gp, torch.ones_like(gp))
    return t, good & conv & okd


def normal(x, y, p):
    """Unit normal grad(z - z_v - sag) = (-2x sag', -2y sag', 1)/norm."""
    if p["kind"] == PLANE:
        z = torch.zeros_like(x)
        return torch.stack([z, z, torch.ones_like(x)], -1), torch.ones_like(x, dtype=torch.bool)
    s = x * x + y * y
    _, dz, ok = sag(s, p)
    nx = -2.0 * x * dz
    ny = -2.0 * y * dz
    nz = torch.ones_like(x)
    nrm = torch.sqrt(nx * nx + ny * ny + 1.0)
    return torch.stack([nx / nrm, ny / nrm, nz / nrm], -1), ok


def refract(d, n, n1, n2):
    """Vector Snell; returns the refracted direction and a no-TIR mask."""
    cos_i = (n * d).sum(-1)
    flip = cos_i < 0
    n = torch.where(flip[:, None], -n, n)
    cos_i = cos_i.abs()
    eta = n1 / n2
    k = 1.0 - eta * eta * (1.0 - cos_i * cos_i)
    ok = k >= 0
    ct = torch.sqrt(torch.where(ok, k, torch.zeros_like(k)))
    dn = eta * d + (ct - eta * cos_i)[:, None] * n
    return dn, ok


def trace_surface(ray, p, n_before):
    """Intersect, clip, refract and accumulate OPL at one surface."""
    o, d = ray["o"], ray["d"]
    t, ok = intersect(o, d, p)
    hit = o + t[:, None] * d
    s = hit[:, 0] ** 2 + hit[:, 1] ** 2
    if p["r_ap"] > 0:
        ok = ok & (s <= p["r_ap"] ** 2)
    nrm, okn = normal(hit[:, 0], hit[:, 1], p)
    dn, okr = refract(d, nrm, n_before, p["n_after"])
    alive = ray["alive"] & ok & okn & okr
    out = dict(ray)
    out["o"] = hit
    out["d"] = dn
    out["opl"] = ray["opl"] + n_before * t
    out["alive"] = alive
    return out


def trace(ray, params, n_start):
    """Trace through a list of surface-parameter dicts; returns ray, final index."""
    n = n_start
    for p in params:
        ray = trace_surface(ray, p, n)
        n = p["n_after"]
    return ray, n


def to_plane(ray, z_plane):
    """Propagate to the plane z = z_plane (no refraction); adds path t (index 1)."""
    o, d = ray["o"], ray["d"]
    t = (z_plane - o[:, 2]) / d[:, 2]
    out = dict(ray)
    out["o"] = o + t[:, None] * d
    out["t_last"] = t
    return out
