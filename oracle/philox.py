"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), NumPy uint arithmetic.

Written from the published definition: ten rounds of
    (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
with M0 = 0xD2511F53, M1 = 0xCD9E8D57, the key bumped by the Weyl constants
(0x9E3779B9, 0xBB67AE85) between rounds.

Uniforms: u = ((x >> 9) + 1/2) * 2^-23, exact in float32 and float64, in (0, 1).
Stream layout for secondary-ray sampling (draw i of incident ray r, bin j):
counter = (j >> 2, i, r, rng_offset), key = (seed & 0xffffffff, seed >> 32),
word j & 3 of the output.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10; all arguments uint32-valued arrays/scalars."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK
    k1 = np.asarray(k1, dtype=np.uint64) & MASK
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return (c0.astype(np.uint32), c1.astype(np.uint32), c2.astype(np.uint32),
            c3.astype(np.uint32))


def uniform_from_u32(x):
    """(0, 1) uniform from a 32-bit word, exactly representable in float32."""
    x = np.asarray(x, dtype=np.uint64)
    return ((x >> np.uint64(9)).astype(np.float64) + 0.5) * (2.0 ** -23)


def sample_uniforms(seed, rng_offset, ray_ids, n_draws, n_bins):
    """u[r, i, j] for the secondary-ray sampling stream (float64 array)."""
    ray_ids = np.asarray(ray_ids, dtype=np.uint64)
    R = ray_ids.shape[0]
    j = np.arange(n_bins, dtype=np.uint64)
    i = np.arange(n_draws, dtype=np.uint64)
    c0 = np.broadcast_to((j >> np.uint64(2))[None, None, :], (R, n_draws, n_bins))
    c1 = np.broadcast_to(i[None, :, None], (R, n_draws, n_bins))
    c2 = np.broadcast_to(ray_ids[:, None, None], (R, n_draws, n_bins))
    c3 = np.full((R, n_draws, n_bins), rng_offset, dtype=np.uint64)
    seed = int(seed)
    out = philox4x32_10(c0, c1, c2, c3, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    words = np.stack(out, -1)                      # [R, n, bins, 4]
    sel = (j & np.uint64(3)).astype(np.int64)
    w = np.take_along_axis(words, np.broadcast_to(sel[None, None, :, None],
                                                  (R, n_draws, n_bins, 1)), -1)[..., 0]
    return uniform_from_u32(w)
