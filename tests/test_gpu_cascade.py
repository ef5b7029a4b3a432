"""Two DOEs in cascade through the C ABI: rw_doe_emit writes the secondary
rays of the first DOE (hit point, direction, complex amplitude, optical path),
and those rays are the incident rays of rw_forward on a system that holds the
second DOE.  Compared with the FP64 oracle running the same cascade.  (The
adjoint of a cascade is not formed: rw_backward returns no gradient with
respect to its incident rays.)"""
import numpy as np
import pytest
import torch

import rwinputs as R
from oracle import pipeline as OP

from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu


def _systems():
    # stage 1: a 16 px-period binary grating (D = 16) lit by an 8 x 8 bundle
    w1 = R.configs.c1(n_side=8, D=16, angles_deg=(2.0,))
    # stage 2: a random-phase DOE 20 um behind it, then a sensor 0.1 mm further
    phi2 = R.maps.random_phase(256, 256, 23) * 0.4
    doe2 = R.DOE(phi=phi2.astype(np.float32), pitch=0.5e-3, D=16, lambda0=550e-6)
    sen = R.Sensor(z=0.12, nx=64, ny=64, pitch=2e-3)
    sys2 = R.System([R.Surface(R.PLANE, 0.02)], 0, doe2, sen)
    return w1, sys2


def test_two_doe_cascade_matches_oracle():
    from paper_2605_15418_gb300 import raywave as RW
    w1, sys2 = _systems()
    job = w1.jobs[0]
    sim1 = RW.Simulator(w1)
    out = sim1.emit()
    torch.cuda.synchronize()
    S = w1.system.doe.M ** 2
    n2 = sim1.n_rays * S
    g = int(round(n2 ** 0.5))
    assert g * g == n2
    rays2 = RW.alloc_rays(n2, sim1.dev)
    rays2["ox"].copy_(out["hx"].repeat_interleave(S))
    rays2["oy"].copy_(out["hy"].repeat_interleave(S))
    rays2["oz"].copy_(out["hz"].repeat_interleave(S))
    for k in ("dx", "dy", "dz", "a_re", "a_im"):
        rays2[k].copy_(out[k])                         # evanescent bins: d = 0, dropped
    rays2["opl"].copy_(out["opl"].repeat_interleave(S))
    job2 = R.Job(lam=job.lam, grid_n=g)
    w2 = R.systems.Workload("second DOE", sys2, [job2], z_start=0.0)
    psf = RW.Simulator(w2, ctx=sim1.ctx, rays=rays2).forward().cpu().numpy()
    assert sim1.ctx.device_status() == 0
    # the oracle: the same two steps in float64
    with torch.no_grad():
        em1, _ = OP.emit_job(w1.system, job, w1.z_start, OP.params_of(w1.system),
                             *OP.map_tensors(w1.system))
        N = em1["U"].shape[0]
        rays = {"o": em1["o"][:, None, :].expand(N, S, 3).reshape(-1, 3),
                "d": em1["d"].reshape(-1, 3), "a": em1["a"].reshape(-1),
                "opl": em1["opl"][:, None].expand(N, S).reshape(-1),
                "alive": em1["alive"].reshape(-1)}
        ref = OP.psf_job(sys2, job2, 0.0, OP.params_of(sys2), *OP.map_tensors(sys2),
                         rays=rays).numpy()
    assert ref.sum() > 0
    assert rel_l2(psf[0], ref) <= 1e-4, rel_l2(psf[0], ref)
    # a phase-only cascade: at most the incident power arrives (1 per ray;
    # the high orders miss the 0.128 mm sensor: measured 39 %)
    assert 0.3 * sim1.n_rays < psf.sum() <= sim1.n_rays * (1 + 1e-5)
