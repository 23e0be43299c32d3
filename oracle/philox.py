"""Philox4x32-10 counter-based generator and Box-Muller normals.

Test infrastructure only (see ``oracle/__init__``).

Philox4x32 is the counter-based generator of Salmon, Moraes, Dror and Shaw
("Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of
    (hi0, lo0) = mulhilo32(0xD2511F53, c0)
    (hi1, lo1) = mulhilo32(0xCD9E8D57, c2)
    c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
with the key bumped by (0x9E3779B9, 0xBB67AE85) between rounds.  The method
draws all its Gaussian numbers (the dry noise W of Eq. step2, the RFD vector
of the thermal forcing, the stochastic stress of Eq. stokes_temporal) from
counters (index, step, replica, tag) under a 64-bit seed, so the oracle and
the GPU path draw identical uint32 words.

Uniforms are (u + 1/2) * 2^-32 in (0, 1); normals come from Box-Muller
pairs: sqrt(-2 ln u0) * (cos 2 pi u1, sin 2 pi u1).
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)

TAG_DRY, TAG_RFD, TAG_STRESS_A, TAG_STRESS_B = 1, 2, 3, 4


def philox4x32(c0, c1, c2, c3, seed):
    """Vectorised Philox4x32-10; counters are arrays of uint32-valued ints."""
    c0 = np.asarray(c0, dtype=np.uint64) & MASK
    c1 = np.broadcast_to(np.asarray(c1, dtype=np.uint64) & MASK, c0.shape).copy()
    c2 = np.broadcast_to(np.asarray(c2, dtype=np.uint64) & MASK, c0.shape).copy()
    c3 = np.broadcast_to(np.asarray(c3, dtype=np.uint64) & MASK, c0.shape).copy()
    c0 = c0.copy()
    k0 = np.uint64(int(seed) & 0xFFFFFFFF)
    k1 = np.uint64((int(seed) >> 32) & 0xFFFFFFFF)
    for rnd in range(10):
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
        if rnd < 9:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
    return c0, c1, c2, c3


def uniforms(words):
    return (np.asarray(words, dtype=np.float64) + 0.5) * 2.0 ** -32


def normals4(c0, c1, c2, c3, seed):
    """Four standard normals per counter (two Box-Muller pairs)."""
    w = philox4x32(c0, c1, c2, c3, seed)
    u = [uniforms(x) for x in w]
    r0 = np.sqrt(-2.0 * np.log(u[0]))
    r1 = np.sqrt(-2.0 * np.log(u[2]))
    return (r0 * np.cos(2.0 * np.pi * u[1]), r0 * np.sin(2.0 * np.pi * u[1]),
            r1 * np.cos(2.0 * np.pi * u[3]), r1 * np.sin(2.0 * np.pi * u[3]))


def ion_normals(n_ions, step, replica, tag, seed, first_index=0):
    """(3, n) normals for ions first_index .. first_index + n - 1."""
    idx = np.arange(first_index, first_index + n_ions, dtype=np.uint64)
    g = normals4(idx, step, replica, tag, seed)
    return np.stack(g[:3], axis=0)
