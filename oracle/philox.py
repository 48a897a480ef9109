"""Philox-4x32-10 and Box-Muller normals (oracle side).

Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11): a 4 x 32-bit counter is run through 10 rounds of

    (c0, c1, c2, c3) -> (hi(B*c2) ^ c1 ^ k0, lo(B*c2), hi(A*c0) ^ c3 ^ k1, lo(A*c0))

with A = 0xD2511F53, B = 0xCD9E8D57, and the 2 x 32-bit key advanced by the
Weyl increments (0x9E3779B9, 0xBB67AE85) between rounds.

Auxiliary fields (Eq. 4 draws x_g ~ N(0,1); Sec. II.B shares them between the
paired walkers).  One generator call per pair of field indices:

    key     = (seed mod 2^32, seed div 2^32)
    counter = (j, k, t, 0)    j = g div 2, k = global walker (pair) index,
                              t = propagation step index
    a = (w1 << 32) | w0,  b = (w3 << 32) | w2
    u1 = ((a >> 11) + 1) * 2^-53  in (0, 1],   u2 = (b >> 11) * 2^-53  in [0, 1)
    x_{2j}   = sqrt(-2 ln u1) cos(2 pi u2)
    x_{2j+1} = sqrt(-2 ln u1) sin(2 pi u2)

The stream depends on (seed, t, k, g) only, never on the system, so the two
systems of a pair draw identical x_g for every g they both have.
"""
import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_A = np.uint64(0xD2511F53)
_B = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(counter, key):
    """counter: uint32 [..., 4]; key: uint32 [..., 2] (broadcastable). Returns uint32 [..., 4]."""
    counter = np.asarray(counter, dtype=np.uint32)
    key = np.asarray(key, dtype=np.uint32)
    c0, c1, c2, c3 = (counter[..., i].astype(np.uint64) for i in range(4))
    k0 = key[..., 0].astype(np.uint64)
    k1 = key[..., 1].astype(np.uint64)
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _A * c0
        p1 = _B * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ k0, p1 & _MASK,
                          (p0 >> np.uint64(32)) ^ c3 ^ k1, p0 & _MASK)
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def uniforms53(words):
    """words: uint32 [..., 4] -> (u1 in (0,1], u2 in [0,1)) float64."""
    w = words.astype(np.uint64)
    a = (w[..., 1] << np.uint64(32)) | w[..., 0]
    b = (w[..., 3] << np.uint64(32)) | w[..., 2]
    u1 = ((a >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = (b >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return u1, u2


def box_muller(u1, u2):
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


def gaussian_fields(seed: int, t: int, walkers, X: int):
    """Standard-normal fields x[k, g] for step t and global walker indices ``walkers``."""
    walkers = np.asarray(walkers, dtype=np.int64)
    nj = (X + 1) // 2
    ctr = np.zeros((walkers.size, nj, 4), dtype=np.uint32)
    ctr[..., 0] = np.arange(nj, dtype=np.uint32)[None, :]
    ctr[..., 1] = walkers.astype(np.uint32)[:, None]
    ctr[..., 2] = np.uint32(t)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    u1, u2 = uniforms53(philox4x32_10(ctr, key))
    z0, z1 = box_muller(u1, u2)
    x = np.empty((walkers.size, 2 * nj))
    x[:, 0::2] = z0
    x[:, 1::2] = z1
    return x[:, :X]
