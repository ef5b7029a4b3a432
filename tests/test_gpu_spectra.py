"""Patch spectra (A3 + A4): the FP32 FFT kernel and the tensor-core
(tcgen05, BF16x3) contraction against the oracle's direct FP64 DFT."""
import numpy as np
import pytest
import torch

import rwinputs as R
from oracle import pipeline as OP

from gpu_helpers import oracle_psf, rel_l2

pytestmark = pytest.mark.gpu


def _oracle_spectra(w):
    out = []
    base = 0
    with torch.no_grad():
        for job in w.jobs:
            em, _ = OP.emit_job(w.system, job, w.z_start, OP.params_of(w.system),
                                *OP.map_tensors(w.system), ray_base=base)
            out.append(em["U"].numpy())
            base += job.n_rays
    return np.concatenate(out, 0)


@pytest.mark.parametrize("which", ["planar", "conformal"])
def test_fft_and_tensor_core_spectra_match_fp64_dft(which):
    from paper_2605_15418_gb300 import raywave as RW
    if which == "planar":
        w = R.configs.c2(n_side=13, D=64, lams=(486e-6, 656e-6), fields_deg=(0.0, 2.0),
                         sensor_n=64, map_side=256)
    else:
        w = R.configs.c4(n_side=9, D=64, n_fields=3, max_field_deg=20.0, map_side=512,
                         lams=(550e-6,))
    sim = RW.Simulator(w)
    ref = _oracle_spectra(w)
    fft = sim.spectra("fft32").cpu().numpy()
    tc = sim.spectra("tc").cpu().numpy()
    # the conformal case inherits ~1e-4 from the FP32 incident trace to the
    # curved DOE (one ray dominates); both transforms see the same patches
    tol = 1e-5 if which == "planar" else 2e-4
    assert rel_l2(fft, ref) <= tol, rel_l2(fft, ref)
    # BF16x3 (hi*hi + hi*lo + lo*hi): ~2^-16 per product, FP32 accumulation
    assert rel_l2(tc, ref) <= tol, rel_l2(tc, ref)
    # equal accuracy: the two transforms of the same patches agree closely
    assert rel_l2(tc, fft) <= 1e-5, rel_l2(tc, fft)
    assert sim.ctx.device_status() == 0


def test_tensor_core_spectra_reject_unsupported_patch_size():
    from paper_2605_15418_gb300 import raywave as RW
    w = R.configs.c2(n_side=4, D=32, lams=(550e-6,), fields_deg=(0.0,), sensor_n=16,
                     map_side=128)
    sim = RW.Simulator(w)
    with pytest.raises(RW.RayWaveError) as e:
        sim.spectra("tc")
    assert e.value.status == 1


@pytest.mark.parametrize("which", ["planar", "conformal"])
def test_fused_forward_with_tensor_core_transform(which):
    """rw_forward / rw_forward_vis with doe.dft = RW_DFT_TC: the patch spectra
    of the fused forward come from the tcgen05 contraction instead of the FP32
    FFT; culling, emission, splat, mask and tape are the same code.  The PSF
    against the FP64 oracle and against the FFT path, the mask bit for bit
    where the two spectra agree, and the taped adjoint of the TC forward."""
    from paper_2605_15418_gb300 import raywave as RW
    if which == "planar":
        w = R.configs.c2(n_side=24, D=64, lams=(486e-6, 656e-6), fields_deg=(0.0, 2.0),
                         sensor_n=96, map_side=256)
        w.system.sensor.pitch = 8e-3
    else:
        w = R.configs.c4(n_side=12, D=64, n_fields=3, max_field_deg=5.0, map_side=512,
                         lams=(550e-6,))
        for j in w.jobs:
            j.spacing = 0.02
        w.system.sensor.nx = w.system.sensor.ny = 64
        w.system.sensor.pitch = 12e-3
    ref = oracle_psf(w)
    fft = RW.Simulator(w, dft="fft32")
    tc = RW.Simulator(w, dft="tc")
    p_fft = fft.forward().cpu().numpy()
    p_tc = tc.forward().cpu().numpy()
    torch.cuda.synchronize()
    assert tc.ctx.device_status() == 0
    assert ref.sum() > 0
    assert rel_l2(p_tc, ref) <= 1e-4, rel_l2(p_tc, ref)
    assert rel_l2(p_tc, p_fft) <= 1e-5, rel_l2(p_tc, p_fft)
    # with the visibility mask and the forward's tape, then the taped adjoint
    M = w.system.doe.M
    v_fft = RW.alloc_vis(fft.n_rays, M, fft.dev)
    v_tc = RW.alloc_vis(tc.n_rays, M, tc.dev)
    q_fft = fft.forward(vis=v_fft)
    q_tc = tc.forward(vis=v_tc)
    tgt = torch.rand(q_tc.shape, generator=torch.Generator().manual_seed(3)).cuda()
    g_fft, g_tc = torch.empty_like(q_fft), torch.empty_like(q_tc)
    fft.loss(q_fft, tgt, g_fft)
    tc.loss(q_tc, tgt, g_tc)
    d_fft, _, s_fft = fft.backward(g_fft, vis=v_fft)
    d_tc, _, s_tc = tc.backward(g_tc, vis=v_tc)
    torch.cuda.synchronize()
    # a bin can change its visibility only where its secondary ray grazes a
    # pixel edge of the window: compare the masks' popcounts
    lut = torch.tensor([bin(i).count("1") for i in range(256)], device=v_tc.device)
    n_fft = int(lut[v_fft.view(torch.uint8).long()].sum())
    n_tc = int(lut[v_tc.view(torch.uint8).long()].sum())
    assert abs(n_fft - n_tc) <= 1e-4 * n_fft, (n_fft, n_tc)
    assert rel_l2(d_tc.cpu().numpy(), d_fft.cpu().numpy()) <= 1e-4
    assert rel_l2(s_tc.cpu().numpy(), s_fft.cpu().numpy()) <= 1e-4
