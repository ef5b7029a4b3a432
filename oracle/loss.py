"""Image metrics, float64 (oracle).

Eq. 3 (section "Benchmark and Inverse Design Demonstrations"): the
normalised least-squares objective || alpha |S|^2 - I_tgt ||^2 with a scalar
alpha compensating global intensity scale.  Reading: alpha is the optimal
scale alpha* = <I, T> / <I, I> over the whole stack of images; since
dL/dalpha = 0 there, the gradient does not depend on whether alpha is held
fixed.  NCC is the normalised cross-correlation of the patch-size study
(same section as the formalism); MSE is the mean squared error.
"""
import torch


def eq3_loss(I, T):
    a = (I * T).sum() / (I * I).sum()
    return ((a * I - T) ** 2).sum(), a


def ncc(I, ref):
    return (ref * I).sum() / torch.sqrt((ref * ref).sum() * (I * I).sum())


def mse(I, ref):
    return ((I - ref) ** 2).mean()
