"""Philox4x32-10 counter-based generator, uniforms and Box-Muller normals (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper does not say which generator draws the Gaussian weights W_j, W'_j
and the frequencies a_j (Sec. 4.1, Eq. DiscreteFT).  Reading taken: a
counter-based generator so that every mode's draws depend only on
(seed, stream, mode index) and never on N or on the order of evaluation.  The
generator is Philox4x32 with 10 rounds as published by Salmon, Moraes, Dror
and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11), written here
from that definition:

* state: a 4x32-bit counter (c0, c1, c2, c3) and a 2x32-bit key (k0, k1);
* one round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (full 64-bit
  products), new counter = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), with
  M0 = 0xD2511F53 and M1 = 0xCD9E8D57;
* between rounds the key is bumped by the Weyl constants
  (0x9E3779B9, 0xBB67AE85);
* 10 rounds; the 4 words of the final counter are the output block.

Stream layout used throughout this project (one block = 4 words):

* key     = (seed mod 2^32, seed >> 32)
* counter = (j mod 2^32, block index b, stream tag, j >> 32)

Uniforms: words (w0, w1) and (w2, w3) of a block form two 64-bit integers
u64 = w_hi * 2^32 + w_lo; each gives u = (floor(u64 / 2^12) + 1/2) * 2^-52,
which is exact in FP64 and lies strictly inside (0, 1).

Normals: block b gives normals 2b and 2b+1 by the Box-Muller transform of its
two uniforms (u0, u1): r = sqrt(-2 ln u0), n0 = r cos(2 pi u1),
n1 = r sin(2 pi u1).
"""
import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32-10 block function.

    ctr: uint array of shape (..., 4); key: uint array of shape (..., 2)
    (broadcastable).  Returns uint64 array of shape (..., 4) holding the four
    32-bit output words.
    """
    c = np.asarray(ctr, dtype=np.uint64) & _MASK32
    k = np.asarray(key, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = k[..., 0], k[..., 1]
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK32
            k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK32
        p0 = m0 * c0  # < 2^64: exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return np.stack(np.broadcast_arrays(c0, c1, c2, c3), axis=-1)


def _key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64)


def block(seed, stream, j, b):
    """Output words of block b of mode j (arrays broadcast), shape (..., 4)."""
    j = np.asarray(j, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    j, b = np.broadcast_arrays(j, b)
    ctr = np.stack([j & _MASK32, b & _MASK32,
                    np.full_like(j, int(stream) & 0xFFFFFFFF),
                    j >> np.uint64(32)], axis=-1)
    return philox4x32_10(ctr, _key(seed))


def words_to_uniforms(w):
    """Four 32-bit words (..., 4) -> two FP64 uniforms (..., 2) in (0, 1)."""
    w = np.asarray(w, dtype=np.uint64)
    u64a = (w[..., 1] << np.uint64(32)) | w[..., 0]
    u64b = (w[..., 3] << np.uint64(32)) | w[..., 2]
    out = np.empty(w.shape[:-1] + (2,), dtype=np.float64)
    scale = 2.0 ** -52
    out[..., 0] = ((u64a >> np.uint64(12)).astype(np.float64) + 0.5) * scale
    out[..., 1] = ((u64b >> np.uint64(12)).astype(np.float64) + 0.5) * scale
    return out


def uniforms(seed, stream, j, b):
    """The two uniforms of block b of mode j, shape (..., 2)."""
    return words_to_uniforms(block(seed, stream, j, b))


def box_muller(u0, u1):
    """Box-Muller: two uniforms in (0, 1) -> two independent N(0, 1)."""
    r = np.sqrt(-2.0 * np.log(u0))
    return r * np.cos(2.0 * np.pi * u1), r * np.sin(2.0 * np.pi * u1)


def normal(seed, stream, j, k):
    """Normal number k of mode j (k = 2b or 2b+1 comes from block b)."""
    k = np.asarray(k, dtype=np.int64)
    u = uniforms(seed, stream, j, k // 2)
    n0, n1 = box_muller(u[..., 0], u[..., 1])
    return np.where(k % 2 == 0, n0, n1)
