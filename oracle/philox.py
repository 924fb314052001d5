"""Philox4x32-10 and a Box-Muller Gaussian stream (oracle side).

Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two
32x32->64-bit multiplications (multipliers 0xD2511F53, 0xCD9E8D57) with the
key bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85) between rounds.
Pinned by that paper's known-answer vectors (tests/golden/philox4x32_10_kat.txt).

Stream convention shared with the CUDA side (each side implements it from
this definition; no code is shared):
  element n of a row-major matrix drawn from (seed, stream) uses
  counter = (b mod 2^32, b >> 32, stream, 0) with b = n // 4 and
  key = (seed mod 2^32, seed >> 32); word w = n % 4 of the output.
  Uniform u_w = (x_w + 0.5) / 2^32.  Gaussian by Box-Muller on the pairs
  (u0,u1) and (u2,u3): z_{2p} = sqrt(-2 ln u_{2p}) cos(2 pi u_{2p+1}),
  z_{2p+1} = sqrt(-2 ln u_{2p}) sin(2 pi u_{2p+1}).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr: (..., 4) uint32-valued array; key: (..., 2).  Returns (..., 4) uint32."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64)
    k1 = np.asarray(key[..., 1], dtype=np.uint64)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c[0]  # < 2^64, exact in uint64
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack([x.astype(np.uint32) for x in c], axis=-1)


def philox_words(seed: int, stream: int, n: int) -> np.ndarray:
    """The first n 32-bit words of the (seed, stream) stream."""
    nb = (n + 3) // 4
    b = np.arange(nb, dtype=np.uint64)
    ctr = np.stack([b & MASK, b >> np.uint64(32), np.full(nb, stream, np.uint64), np.zeros(nb, np.uint64)], -1)
    key = np.broadcast_to(np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], np.uint64), (nb, 2))
    return philox4x32_10(ctr, key).reshape(-1)[:n]


def gaussian(seed: int, stream: int, rows: int, cols: int) -> np.ndarray:
    """rows x cols standard Gaussian matrix (float64) from the stream."""
    n = rows * cols
    nb = (n + 3) // 4
    x = philox_words(seed, stream, 4 * nb).astype(np.float64).reshape(nb, 4)
    u = (x + 0.5) / 4294967296.0
    r0 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r1 = np.sqrt(-2.0 * np.log(u[:, 2]))
    t0 = 2.0 * np.pi * u[:, 1]
    t1 = 2.0 * np.pi * u[:, 3]
    z = np.stack([r0 * np.cos(t0), r0 * np.sin(t0), r1 * np.cos(t1), r1 * np.sin(t1)], -1)
    return z.reshape(-1)[:n].reshape(rows, cols)
