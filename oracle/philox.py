"""Philox4x32-10 counter-based generator and Box-Muller Gaussians (oracle side).

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

Algorithm 1 step 1 draws the Gaussian test matrix Omega (i.i.d. N(0,1), Sec. II).
Both sides implement one counter-based generator from its published definition
so that the same seed gives the same Omega:

  Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
  numbers: as easy as 1, 2, 3", SC'11).  Round function on counter
  (c0, c1, c2, c3) and key (k0, k1):
      (hi0, lo0) = 0xD2511F53 * c0      (64-bit product split in halves)
      (hi1, lo1) = 0xCD9E8D57 * c2
      c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
  and between rounds the key is bumped by the Weyl constants
      k0 += 0x9E3779B9, k1 += 0xBB67AE85   (mod 2^32).

Omega element mapping (column-major N x ell, flat index e = j*N + i):
  Philox block b = e // 4 with counter (b mod 2^32, b >> 32, 0, 0) and key
  (seed mod 2^32, seed >> 32) gives words (x0, x1, x2, x3);
  uniforms u_r = ((x_r >> 9) + 0.5) * 2^-23, exactly representable in fp32;
  Box-Muller (Box & Muller 1958): rho = sqrt(-2 ln u0),
      z[4b+0] = rho cos(2 pi u1), z[4b+1] = rho sin(2 pi u1),
  and likewise (u2, u3) -> z[4b+2], z[4b+3].
The oracle evaluates Box-Muller in float64.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Vectorised Philox4x32-10.

    ctr: uint64 array (..., 4) holding 32-bit words; key: uint64 array (..., 2).
    Returns uint64 array (..., 4) of 32-bit output words.
    """
    c = [ctr[..., r].astype(np.uint64) & MASK for r in range(4)]
    k0 = key[..., 0].astype(np.uint64) & MASK
    k1 = key[..., 1].astype(np.uint64) & MASK
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [(hi1 ^ c[1] ^ k0) & MASK, lo1, (hi0 ^ c[3] ^ k1) & MASK, lo0]
    return np.stack(c, axis=-1)


def gaussian_matrix(N: int, ell: int, seed: int) -> np.ndarray:
    """Omega as an (ell, N) float64 array: row j is probe column j (an image)."""
    total = N * ell
    nblk = (total + 3) // 4
    b = np.arange(nblk, dtype=np.uint64)
    ctr = np.zeros((nblk, 4), dtype=np.uint64)
    ctr[:, 0] = b & MASK
    ctr[:, 1] = b >> np.uint64(32)
    key = np.zeros((nblk, 2), dtype=np.uint64)
    key[:, 0] = np.uint64(seed) & MASK
    key[:, 1] = np.uint64(seed) >> np.uint64(32)
    x = philox4x32_10(ctr, key)
    u = ((x >> np.uint64(9)).astype(np.float64) + 0.5) * (2.0 ** -23)
    rho01 = np.sqrt(-2.0 * np.log(u[:, 0]))
    rho23 = np.sqrt(-2.0 * np.log(u[:, 2]))
    z = np.empty((nblk, 4), dtype=np.float64)
    z[:, 0] = rho01 * np.cos(2.0 * np.pi * u[:, 1])
    z[:, 1] = rho01 * np.sin(2.0 * np.pi * u[:, 1])
    z[:, 2] = rho23 * np.cos(2.0 * np.pi * u[:, 3])
    z[:, 3] = rho23 * np.sin(2.0 * np.pi * u[:, 3])
    return z.reshape(-1)[:total].reshape(ell, N)
