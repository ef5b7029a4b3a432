"""torch.autograd.Function around rw_forward / rw_backward.

PSF = RayWavePSF.apply(sim, phi, surf_params) with surf_params a float64
tensor [nsurf, 8] = (z, c, k, A4, A6, A8, A10, n_after) per surface.  The
backward recomputes patches and spectra in the adjoint kernel; nothing but
the inputs is saved.  Thicknesses are z differences, so a user who
optimises thicknesses writes z = z0 + cumsum(t) and autograd does the rest.
"""
import torch

from rwinputs import Surface
from . import raywave as RW

PARAM_NAMES = ("z", "c", "k", "A4", "A6", "A8", "A10", "n_after")


def surface_params(surfaces, device):
    return torch.tensor([[s.z, s.c, s.k, *s.A, s.n_after] for s in surfaces],
                        dtype=torch.float64, device=device)


def surfaces_from_params(template, params):
    p = params.detach().cpu().tolist()
    out = []
    for s, v in zip(template, p):
        out.append(Surface(s.kind, v[0], c=v[1], k=v[2], A=tuple(v[3:7]), n_after=v[7],
                           r_ap=s.r_ap, sellmeier=getattr(s, "sellmeier", None)))
    return out


def _vis_ok(sim):
    sysm = sim.w.system
    return (sysm.doe.emit == "exhaustive" and not sysm.sensor.coherent
            and all(getattr(s, "sellmeier", None) is None for s in sysm.surfaces))


class RayWavePSF(torch.autograd.Function):
    """Forward keeps the one-bit-per-secondary-ray visibility mask (exhaustive
    emission) so the adjoint reverses only rays that reached the sensor."""

    @staticmethod
    def forward(ctx, sim, phi, params):
        surfs = surfaces_from_params(sim.w.system.surfaces, params)
        vis = None
        if _vis_ok(sim):
            vis = RW.alloc_vis(sim.n_rays, sim.w.system.doe.M, sim.dev)
        psf = sim.forward(phi=phi.detach().contiguous(), surfaces=surfs, vis=vis)
        ctx.sim = sim
        ctx.surfs = surfs
        ctx.vis = vis
        ctx.save_for_backward(phi)
        return psf

    @staticmethod
    def backward(ctx, g):
        (phi,) = ctx.saved_tensors
        dphi, _, dsurf = ctx.sim.backward(g.contiguous(), phi=phi.detach().contiguous(),
                                          surfaces=ctx.surfs, vis=ctx.vis)
        return None, dphi, dsurf


def psf(sim, phi, params):
    return RayWavePSF.apply(sim, phi, params)
