"""Block culling of the exhaustive incoherent forward: tracing only the
blocks of bins whose affine enclosure can reach the sensor gives the same
image, and bit for bit the same visibility mask, as tracing every bin
(RW_DOE_TRACE_ALL); both agree with the oracle."""
import numpy as np
import pytest
import torch

import rwinputs as R

from gpu_helpers import oracle_psf, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def RW():
    from paper_2605_15418_gb300 import raywave
    return raywave


@pytest.fixture(scope="module")
def ctx(RW):
    c = RW.Context(0)
    yield c
    c.close()


def _c2(n_side, D, P=1):
    w = R.configs.c2(n_side=n_side, D=D, lams=(486e-6, 656e-6), fields_deg=(0.0, 2.0),
                     sensor_n=96, map_side=256)
    w.system.sensor.pitch = 8e-3
    w.system.doe.pad = P
    return w


def _c5():
    w = R.configs.c5(n_lams=3, n_fields=4, count_lo=60, count_hi=500, D=32, map_side=256,
                     sensor_n=64)
    w.system.doe.emit = "exhaustive"
    w.system.sensor.pitch = 10e-3
    return w


def _c4():
    w = R.configs.c4(n_side=15, D=32, n_fields=3, max_field_deg=20.0, map_side=512,
                     lams=(550e-6,))
    w.system.sensor.pitch = 20e-3
    return w


def _reflective():
    import reflective_cases as RC
    return RC.planar(n_side=13)


CASES = {
    "c2_d64": lambda: _c2(23, 64),
    "reflective_planar": _reflective,
    "c2_d32_pad2": lambda: _c2(19, 32, 2),
    "c2_d16": lambda: _c2(41, 16),
    "c5_six_spheres": _c5,
    "c4_conformal_no_lens": _c4,
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_culled_forward_equals_tracing_every_bin(RW, ctx, case):
    w = CASES[case]()
    M = w.system.doe.M
    culled = RW.Simulator(w, ctx=ctx)
    full = RW.Simulator(w, ctx=ctx, rays=culled.rays, trace_all=True)
    vis_c = RW.alloc_vis(culled.n_rays, M, culled.dev)
    vis_f = RW.alloc_vis(culled.n_rays, M, culled.dev)
    ctx.device_status()
    psf_c = culled.forward(vis=vis_c)
    psf_f = full.forward(vis=vis_f)
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    assert torch.equal(vis_c, vis_f)
    bits = np.unpackbits(vis_f.cpu().numpy().view(np.uint8)).mean()
    assert 0.0 < bits < 1.0
    # same deposits, summed in a different order (float64 accumulation)
    assert rel_l2(psf_c.cpu().numpy(), psf_f.cpu().numpy()) < 1e-6
    ref = oracle_psf(w)
    assert rel_l2(psf_c.cpu().numpy(), ref) <= 1e-4, rel_l2(psf_c.cpu().numpy(), ref)


def test_culling_at_full_c2_size_keeps_every_visible_ray(RW, ctx):
    """Full benchmark size (9 jobs x 1M incident rays, D = 64): the masks
    with and without culling are identical."""
    w = R.configs.c2()
    M = w.system.doe.M
    culled = RW.Simulator(w, ctx=ctx)
    full = RW.Simulator(w, ctx=ctx, rays=culled.rays, trace_all=True)
    vis_c = RW.alloc_vis(culled.n_rays, M, culled.dev)
    vis_f = RW.alloc_vis(culled.n_rays, M, culled.dev)
    psf_c = culled.forward(vis=vis_c)
    psf_f = full.forward(vis=vis_f)
    torch.cuda.synchronize()
    assert torch.equal(vis_c, vis_f)
    assert rel_l2(psf_c.cpu().numpy(), psf_f.cpu().numpy()) < 1e-6


def test_taped_adjoint_equals_recomputed_adjoint(RW, ctx):
    """The forward with a mask tapes its visible secondary rays; the adjoint
    over that tape equals the adjoint that recomputes patches and spectra
    (forced here by a newer forward on another mask, which retires the tape
    of the first)."""
    w = _c2(23, 64)
    M = w.system.doe.M
    sim = RW.Simulator(w, ctx=ctx)
    vis1 = RW.alloc_vis(sim.n_rays, M, sim.dev)
    vis2 = RW.alloc_vis(sim.n_rays, M, sim.dev)
    ctx.device_status()
    psf = sim.forward(vis=vis1)
    tgt = torch.as_tensor(R.gaussian_spots_target(len(w.jobs), 96, 96, seed=3), device=sim.dev)
    gI = torch.empty_like(psf)
    sim.loss(psf, tgt, gI)
    n0 = ctx.launches
    taped = sim.backward(gI, vis=vis1)                 # tape: no spectra kernel
    n_taped = ctx.launches - n0
    sim.forward(vis=vis2)                              # same inputs, new tape for vis2
    n0 = ctx.launches
    recomputed = sim.backward(gI, vis=vis1)            # vis1 has no tape now
    n_recomputed = ctx.launches - n0
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    # maps + trace + scatter; maps + count + spectra + trace + scatter
    assert n_taped == 3 and n_recomputed == 5, (n_taped, n_recomputed)
    assert rel_l2(taped[0].cpu().numpy(), recomputed[0].cpu().numpy()) < 1e-6
    assert rel_l2(taped[2].cpu().numpy(), recomputed[2].cpu().numpy()) < 1e-6
    # and the taped adjoint matches the fused adjoint over every bin
    full = sim.backward(gI)
    torch.cuda.synchronize()
    assert rel_l2(taped[0].cpu().numpy(), full[0].cpu().numpy()) < 1e-5
