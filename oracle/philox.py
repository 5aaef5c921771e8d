"""Counter-based Philox4x32-10 generator and the Gaussian test matrix Omega.

TEST INFRASTRUCTURE: this module is part of the CPU oracle.  Only tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline leg may import it; the
product path never does.

The sketch of the randomized range finder draws a Gaussian test matrix
(Halko-Martinsson-Tropp two-stage scheme, paper Sec. 2.2, "Gaussian sampling"
among the sampling strategies).  The paper does not fix a generator; this
build uses Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11), restated here from that paper:

  * state: a 128-bit counter (c0, c1, c2, c3) and a 64-bit key (k0, k1);
  * one round: with the two multipliers M0 = 0xD2511F53, M1 = 0xCD9E8D57,
      (hi0, lo0) = M0 * c0   (64-bit product split in halves)
      (hi1, lo1) = M1 * c2
      counter   <- (hi1 ^ c1 ^ k0,  lo1,  hi0 ^ c3 ^ k1,  lo0)
  * between rounds the key is bumped by the Weyl constants
      W0 = 0x9E3779B9, W1 = 0xBB67AE85 (mod 2^32);
  * ten rounds, the first with the unbumped key.

Counter layout used by both sides of this build (the device generator in the
CUDA library implements the same definition independently):
  key     = (lo32(seed), hi32(seed))
  counter = (lo32(n), hi32(n), stream, 0) for block n = 0, 1, 2, ...
Each block yields four 32-bit words.

Gaussian transform (Box-Muller), defined so that both uniforms are exact
FP32 numbers: from a block's words (x0, x1, x2, x3) two pairs (x0, x1) and
(x2, x3) are formed; for a pair (x, y)
  u1 = ((x >> 8) + 1) * 2^-24        in (0, 1]
  u2 = (2 * (y >> 9) + 1) * 2^-24    in (0, 1)
  z0 = sqrt(-2 ln u1) * cos(2 pi u2)
  z1 = sqrt(-2 ln u1) * sin(2 pi u2)
and the four outputs of block n are (z0(x0,x1), z1(x0,x1), z0(x2,x3),
z1(x2,x3)).  The oracle evaluates the transform in FP64 and rounds to FP32.

Element e of a row-major rows x cols matrix Omega (e = i*cols + j) is output
(e mod 4) of block floor(e/4).
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(counters, key):
    """Apply the ten-round Philox4x32 bijection.

    counters: uint32 array of shape (N, 4); key: pair of python ints (k0, k1).
    Returns a uint32 array of shape (N, 4).
    """
    c = np.asarray(counters, dtype=np.uint32).astype(np.uint64)
    c0, c1, c2, c3 = c[:, 0], c[:, 1], c[:, 2], c[:, 3]
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = M0 * c0          # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def philox_words(seed, stream, n_blocks, first_block=0):
    """Words of blocks first_block .. first_block+n_blocks-1, shape (n_blocks, 4)."""
    n = np.arange(first_block, first_block + n_blocks, dtype=np.uint64)
    ctr = np.zeros((n_blocks, 4), dtype=np.uint32)
    ctr[:, 0] = (n & MASK32).astype(np.uint32)
    ctr[:, 1] = (n >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = np.uint32(stream & 0xFFFFFFFF)
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return philox4x32_10(ctr, key)


def box_muller(x, y):
    """FP64 Box-Muller of one word pair (arrays of uint32) -> (z0, z1) in FP64."""
    x = np.asarray(x, dtype=np.uint64)
    y = np.asarray(y, dtype=np.uint64)
    u1 = ((x >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24
    u2 = (2.0 * (y >> np.uint64(9)).astype(np.float64) + 1.0) * 2.0 ** -24
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return rad * np.cos(ang), rad * np.sin(ang)


def gaussian_matrix(seed, stream, rows, cols):
    """Omega (rows x cols, FP32) by the counter layout in the module docstring."""
    total = rows * cols
    nb = (total + 3) // 4
    w = philox_words(seed, stream, nb)
    za, zb = box_muller(w[:, 0], w[:, 1])
    zc, zd = box_muller(w[:, 2], w[:, 3])
    z = np.stack([za, zb, zc, zd], axis=1).reshape(-1)[:total]
    return z.astype(np.float32).reshape(rows, cols)
