"""Counter-based random numbers for the FP64 oracle (test infrastructure only).

TEST INFRASTRUCTURE: only tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline leg may import this package. The CUDA library never calls it.

Philox4x32-10 is implemented here from its published definition (Salmon,
Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11):
a 4-word counter and 2-word key, ten rounds; each round multiplies words 0 and
2 by the constants 0xD2511F53 / 0xCD9E8D57, recombines the high and low halves
with the other two words and the key, and the key is bumped by the Weyl
constants 0x9E3779B9 / 0xBB67AE85 between rounds.

The paper only asks for "standard Gaussian" matrices (Section 3 and the lemmas
of Section 5) and multinomial draws (the RANDSAMPLE definition in Section 3.2).
Any such numbers satisfy it; this fixed stream exists so that the GPU path and
the oracle consume the same random numbers:

  * key = (seed mod 2^32, seed >> 32);
  * counter = (block mod 2^32, block >> 32, stream, 0);
  * stream = (purpose << 8) | mode, purpose 0 = Gaussian test matrix,
    purpose 1 = fiber-sampling uniforms;
  * Gaussian element e uses block e // 4 and lane e % 4: the words
    (x0, x1) give z0 = r cos(2 pi u1), z1 = r sin(2 pi u1) with
    r = sqrt(-2 ln u0), and (x2, x3) give z2, z3 the same way;
  * a word x maps to the uniform u = ((x >> 9) + 0.5) * 2^-23, which lies
    strictly inside (0, 1) and is exact in FP32 and FP64 (24 significant
    bits; a 24-bit integer plus one half would need 25);
  * sampling draw t uses block t // 2 and the 64-bit word
    r = x_lo | x_hi << 32 from (x0, x1) for even t and (x2, x3) for odd t.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

PURPOSE_GAUSSIAN = 0
PURPOSE_SAMPLING = 1


def stream_id(purpose: int, mode: int) -> int:
    return ((purpose & 0xFFFFFF) << 8) | (mode & 0xFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on uint64 arrays that hold 32-bit words. Returns 4 arrays."""
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = np.uint64(k0 & MASK32)
    k1 = np.uint64(k1 & MASK32)
    m0 = np.uint64(M0)
    m1 = np.uint64(M1)
    s32 = np.uint64(32)
    mk = np.uint64(MASK32)
    for rnd in range(10):
        if rnd > 0:
            k0 = np.uint64((int(k0) + W0) & MASK32)
            k1 = np.uint64((int(k1) + W1) & MASK32)
        p0 = m0 * c0          # < 2^64: exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> s32, p0 & mk
        hi1, lo1 = p1 >> s32, p1 & mk
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & mk, lo1, (hi0 ^ c3 ^ k1) & mk, lo0
    return c0, c1, c2, c3


def blocks(seed: int, stream: int, block_idx):
    """Philox output words for the given block indices of one stream."""
    b = np.asarray(block_idx, dtype=np.uint64)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return philox4x32_10(b & np.uint64(MASK32), b >> np.uint64(32),
                         np.full(b.shape, stream & MASK32, dtype=np.uint64),
                         np.zeros(b.shape, dtype=np.uint64),
                         seed & MASK32, seed >> 32)


def word_to_uniform(x):
    """u = ((x >> 9) + 0.5) * 2^-23 in FP64."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def gaussian_elements(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normal numbers z_e for e = 0..count-1 of one stream (FP64 Box-Muller)."""
    nb = (count + 3) // 4
    x0, x1, x2, x3 = blocks(seed, stream, np.arange(nb, dtype=np.uint64))
    u0, u1, u2, u3 = (word_to_uniform(x) for x in (x0, x1, x2, x3))
    ra = np.sqrt(-2.0 * np.log(u0))
    rb = np.sqrt(-2.0 * np.log(u2))
    z = np.empty((nb, 4))
    z[:, 0] = ra * np.cos(2.0 * np.pi * u1)
    z[:, 1] = ra * np.sin(2.0 * np.pi * u1)
    z[:, 2] = rb * np.cos(2.0 * np.pi * u3)
    z[:, 3] = rb * np.sin(2.0 * np.pi * u3)
    return z.reshape(-1)[:count]


def gaussian_matrix(seed: int, mode: int, rows: int, cols: int) -> np.ndarray:
    """rows x cols standard Gaussian test matrix of a mode: entry (i, l) is element
    e = i * cols + l of the purpose-0 stream of that mode."""
    z = gaussian_elements(seed, stream_id(PURPOSE_GAUSSIAN, mode), rows * cols)
    return z.reshape(rows, cols)


def sampling_words(seed: int, mode: int, count: int) -> list:
    """64-bit words r_t (Python ints) for draws t = 0..count-1 of a mode."""
    nb = (count + 1) // 2
    x0, x1, x2, x3 = blocks(seed, stream_id(PURPOSE_SAMPLING, mode), np.arange(nb, dtype=np.uint64))
    out = []
    for t in range(count):
        b, odd = divmod(t, 2)
        lo, hi = (x2[b], x3[b]) if odd else (x0[b], x1[b])
        out.append(int(lo) | (int(hi) << 32))
    return out
