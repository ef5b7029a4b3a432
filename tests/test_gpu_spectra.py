"""Patch spectra (A3 + A4): the FP32 FFT kernel and the tensor-core
(tcgen05, BF16x3) contraction against the oracle's direct FP64 DFT."""
import numpy as np
import pytest
import torch

import rwinputs as R
from oracle import pipeline as OP

from gpu_helpers import rel_l2

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
