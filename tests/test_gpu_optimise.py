"""Optimisation progress through the autograd wrapper (end-to-end design in
the paper's Benchmark section): a few Adam steps on the DOE phase and the
lens curvatures, driven by the CUDA forward and adjoint, lower the Eq. 3
loss against the PSF of a perturbed design, in exhaustive mode and in
sampled mode (straight-through Gumbel-softmax gradient, fixed noise)."""
import numpy as np
import pytest
import torch

import rwinputs as R

pytestmark = pytest.mark.gpu


def eq3(I, T):
    """||alpha I - T||^2 with alpha = <I,T>/<I,I> (Eq. 3), in torch."""
    alpha = (I * T).sum() / (I * I).sum()
    return ((alpha * I - T) ** 2).sum()


def _workload(emit):
    w = R.configs.c3(n_side=40, D=16)
    sysm = w.system
    base = sysm.doe.phi.astype(np.float64)
    sysm.doe.phi = base.astype(np.float32)
    sysm.sensor.nx = sysm.sensor.ny = 64
    sysm.sensor.pitch = 30e-3
    sysm.doe.emit = emit
    if emit == "sampled":
        sysm.doe.n_ssr = 96
        sysm.doe.seed = 31
    # target: the PSF of the same system with a perturbed DOE phase
    pert = (base + 0.6 * R.maps.random_phase(512, 512, 17)).astype(np.float32)
    return w, pert


@pytest.mark.parametrize("emit", ["exhaustive", "sampled"])
def test_adam_steps_lower_the_eq3_loss(emit):
    from paper_2605_15418_gb300 import autograd as AG
    from paper_2605_15418_gb300 import raywave as RW
    w, pert = _workload(emit)
    sim = RW.Simulator(w)
    with torch.no_grad():
        target = sim.forward(phi=torch.as_tensor(pert, device=sim.dev)).clone()
    phi = sim.phi.clone().requires_grad_(True)
    params = AG.surface_params(w.system.surfaces, sim.dev).requires_grad_(True)
    mask = torch.zeros_like(params)
    mask[1:, 1] = 1.0                                  # curvatures of the lens surfaces
    opt = torch.optim.Adam([{"params": [phi], "lr": 0.05},
                            {"params": [params], "lr": 1e-4}])
    losses = []
    for _ in range(12):
        opt.zero_grad()
        L = eq3(AG.psf(sim, phi, params), target)
        L.backward()
        params.grad.mul_(mask)
        assert torch.isfinite(phi.grad).all() and torch.isfinite(params.grad).all()
        opt.step()
        losses.append(float(L))
    assert losses[-1] < 0.8 * losses[0], losses
    assert sim.ctx.device_status() == 0
