"""Launch tuning (A10): rw_autotune times every kernel of a forward + adjoint
step at several persistent grid sizes and keeps the fastest per kernel; the
tuned launches compute the same image and gradients."""
import numpy as np
import pytest
import torch

import rwinputs as R

from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu


def test_autotuned_grids_keep_results():
    from paper_2605_15418_gb300 import raywave as RW
    w = R.configs.c2(n_side=64, D=64, lams=(486e-6, 656e-6), fields_deg=(0.0, 2.0),
                     sensor_n=96, map_side=256)
    w.system.sensor.pitch = 8e-3
    sim = RW.Simulator(w)
    M = w.system.doe.M
    vis = RW.alloc_vis(sim.n_rays, M, sim.dev)
    tgt = torch.as_tensor(R.gaussian_spots_target(len(w.jobs), 96, 96, seed=3), device=sim.dev)

    def step():
        psf = sim.forward(vis=vis)
        gI = torch.empty_like(psf)
        sim.loss(psf, tgt, gI)
        dphi, _, dsurf = sim.backward(gI, vis=vis)
        torch.cuda.synchronize()
        return psf.clone(), gI, dphi, dsurf

    psf0, gI, dphi0, dsurf0 = step()
    grids = sim.ctx.autotune(sim, gI, vis)
    assert set(grids) >= {"k_forward", "k_cull", "k_bs_trace", "k_bs_scatter"}
    assert all(isinstance(v, int) and v >= 0 for v in grids.values())
    psf1, _, dphi1, dsurf1 = step()
    assert rel_l2(psf1.cpu().numpy(), psf0.cpu().numpy()) < 1e-6
    assert rel_l2(dphi1.cpu().numpy(), dphi0.cpu().numpy()) < 1e-5
    assert rel_l2(dsurf1.cpu().numpy(), dsurf0.cpu().numpy()) < 1e-5
    # explicit grids (one CTA per SM) and back to the occupancy default
    sim.ctx.set_grids({k: 152 for k in grids})
    psf2 = step()[0]
    sim.ctx.set_grids({})
    assert rel_l2(psf2.cpu().numpy(), psf0.cpu().numpy()) < 1e-6
    assert sim.ctx.device_status() == 0
