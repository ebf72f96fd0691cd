"""Philox-4x32-10 counter-based generator, written from its published definition
(J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC'11, Sec. 4.2: Philox-4x32 with multipliers 0xD2511F53,
0xCD9E8D57 and Weyl key increments 0x9E3779B9, 0xBB67AE85, 10 rounds).

TEST INFRASTRUCTURE ONLY (part of the CPU oracle): imported by tests/, by the
bench's CPU-baseline leg and by the smoke check, never by the product path.

Stream layout used by the solver (the paper only asks for D ~ U[0,1] i.i.d. and
a Gaussian start block, Alg. 1 (its operator and start block)):
  key     = (seed mod 2^32, seed div 2^32)
  counter = (i mod 2^32, i div 2^32, stream, 0) for element / pair index i
  stream 0: diagonal D, D_i = (w >> 11) * 2^-53 with w = x0 | x1 << 32
  stream 1: start block Omega (row-major n x d), Box-Muller on pairs:
            u1 = ((w0 >> 11) + 1) * 2^-53, u2 = (w1 >> 11) * 2^-53,
            z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2);
            element e takes z0 of pair e//2 if e is even, else z1
  stream 2+k: the k-th replacement block after a Lanczos breakdown (same recipe)
"""

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox-4x32 rounds.  All arguments are arrays (or scalars) of 32-bit values."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _MASK for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for r in range(10):
        p0 = _M0 * c0  # 32 x 32 -> 64-bit products never overflow uint64
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if r < 9:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def _words(seed: int, stream: int, count: int):
    i = np.arange(count, dtype=np.uint64)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return philox4x32_10(i & _MASK, i >> _S32, np.uint64(stream), np.uint64(0),
                         np.uint64(seed & 0xFFFFFFFF), np.uint64(seed >> 32))


def uniform01(seed: int, stream: int, count: int) -> np.ndarray:
    """count uniforms in [0, 1) (53-bit resolution), one per counter."""
    x0, x1, _, _ = _words(seed, stream, count)
    w = x0 | (x1 << _S32)
    return (w >> np.uint64(11)).astype(np.float64) * 2.0**-53


def gaussian(seed: int, stream: int, count: int) -> np.ndarray:
    """count standard normals by Box-Muller on pairs (see module docstring)."""
    npairs = (count + 1) // 2
    x0, x1, x2, x3 = _words(seed, stream, npairs)
    w0 = x0 | (x1 << _S32)
    w1 = x2 | (x3 << _S32)
    u1 = ((w0 >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0**-53
    u2 = (w1 >> np.uint64(11)).astype(np.float64) * 2.0**-53
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * npairs)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def perturbation_diagonal(seed: int, n: int) -> np.ndarray:
    """D of Eq. (defB): n i.i.d. U[0,1) entries (stream 0)."""
    return uniform01(seed, 0, n)


def start_block(seed: int, n: int, d: int, stream: int = 1) -> np.ndarray:
    """Omega of Alg. 1 (its Gaussian start block): n x d i.i.d. N(0,1), row-major element order."""
    return gaussian(seed, stream, n * d).reshape(n, d)
