"""Shared helpers for GPU parity tests: run the CUDA path and the oracle on
the same seeded workload."""
import numpy as np
import torch

from oracle import pipeline as OP


def _as_array(x):
    if isinstance(x, torch.Tensor):
        x = x.detach().cpu().numpy()
    return np.asarray(x)


def rel_l2(a, b):
    """||a - b|| / ||b|| over all entries; complex inputs keep both parts
    (|a - b| and |b| of complex entries), nothing is cast away."""
    a = _as_array(a)
    b = _as_array(b)
    if np.iscomplexobj(a) or np.iscomplexobj(b):
        a = a.astype(np.complex128)
        b = b.astype(np.complex128)
    else:
        a = a.astype(np.float64)
        b = b.astype(np.float64)
    assert a.shape == b.shape, (a.shape, b.shape)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_psf(w, **kw):
    with torch.no_grad():
        return OP.psf(w, **kw).numpy()


def angle(d1, d2):
    """2 asin(|d1 - d2| / 2): the angle between unit vectors, rows."""
    diff = np.linalg.norm(np.asarray(d1, np.float64) - np.asarray(d2, np.float64), axis=-1)
    return 2 * np.arcsin(np.clip(diff / 2, 0, 1))
