"""Pins of the oracle's random streams (Philox4x32-10, Gaussians, sampling words)."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        rows.append((int(f[0]), [int(x, 16) for x in f[1:5]], [int(x, 16) for x in f[5:7]],
                     [int(x, 16) for x in f[7:11]]))
    return rows


@pytest.mark.parametrize("row", _kat_rows())
def test_philox_known_answers(row):
    rounds, ctr, key, want = row
    assert rounds == 10
    got = philox.philox4x32_10(*ctr, *key)
    assert [int(g) for g in got] == want


def test_uniform_map_endpoints():
    # u = ((x >> 9) + 0.5) 2^-23: strictly inside (0, 1), symmetric about 1/2,
    # and every value is an FP32 number (24 significant bits)
    assert philox.word_to_uniform(0) == 2.0 ** -24
    assert philox.word_to_uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert philox.word_to_uniform(0x80000000) == 0.5 + 2.0 ** -24
    x = np.array([0, 1 << 9, 0x7FFFFFFF, 0xFFFFFE00, 0xFFFFFFFF], dtype=np.uint64)
    u = philox.word_to_uniform(x)
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)


def test_gaussian_moments_and_ks():
    z = philox.gaussian_elements(seed=12345, stream=philox.stream_id(0, 3), count=1 << 20)
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(stats.skew(z)) < 5 * np.sqrt(6.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # the four lanes of a block are individually standard normal too
    for lane in range(4):
        assert stats.kstest(z[lane::4], "norm").pvalue > 1e-4


def test_gaussian_pairs_are_uncorrelated():
    z = philox.gaussian_elements(seed=7, stream=0, count=1 << 18).reshape(-1, 4)
    c = np.corrcoef(z.T)
    off = c[~np.eye(4, dtype=bool)]
    assert np.max(np.abs(off)) < 5 / np.sqrt(z.shape[0])


def test_streams_and_seeds_differ():
    a = philox.gaussian_matrix(0, 0, 8, 4)
    b = philox.gaussian_matrix(0, 1, 8, 4)
    c = philox.gaussian_matrix(1, 0, 8, 4)
    assert not np.allclose(a, b) and not np.allclose(a, c)
    # element (i, l) is element i*cols + l of the stream: a prefix property
    big = philox.gaussian_matrix(0, 0, 8, 4).reshape(-1)
    assert np.array_equal(philox.gaussian_elements(0, 0, 32), big)


def test_sampling_words_layout():
    # even draws use words (x0, x1), odd draws (x2, x3) of block t // 2
    w = philox.sampling_words(seed=99, mode=2, count=6)
    x = philox.blocks(99, philox.stream_id(1, 2), np.arange(3, dtype=np.uint64))
    for t in range(6):
        b = t // 2
        lo, hi = (x[2][b], x[3][b]) if t % 2 else (x[0][b], x[1][b])
        assert w[t] == int(lo) + (int(hi) << 32)
    # 64-bit words are uniform: top bit balanced over many draws
    ws = philox.sampling_words(seed=1, mode=0, count=20000)
    top = np.array([r >> 63 for r in ws])
    assert abs(top.mean() - 0.5) < 5 * 0.5 / np.sqrt(top.size)
