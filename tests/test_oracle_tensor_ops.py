"""Pins of the oracle's tensor primitives against brute force (Section 2)."""
import itertools

import numpy as np

import synth
from oracle import tucker as ot


def _rand(shape, seed=0):
    return np.asfortranarray(np.random.default_rng(seed).standard_normal(shape))


def test_unfold_index_map_brute_force():
    dims = (3, 4, 5, 2)
    A = _rand(dims)
    for n in range(4):
        M = ot.unfold(A, n)
        assert M.shape == (dims[n], np.prod(dims) // dims[n])
        for idx in itertools.product(*[range(d) for d in dims]):
            # j = i_1 + (i_2 - 1) I_1 + ... skipping mode n (0-based here)
            j, stride = 0, 1
            for m in range(4):
                if m == n:
                    continue
                j += idx[m] * stride
                stride *= dims[m]
            assert M[idx[n], j] == A[idx]


def test_unfold_fold_roundtrip_and_memory_order():
    dims = (3, 4, 5)
    A = _rand(dims, 1)
    for n in range(3):
        assert np.array_equal(ot.fold(ot.unfold(A, n), n, dims), A)
    # mode-1 unfolding is the tensor's memory viewed as I_1 x J (columns = fibers)
    assert np.array_equal(ot.unfold(A, 0), synth.flat(A).reshape(3, 20, order="F"))


def test_ttm_brute_force():
    dims = (3, 4, 5, 2)
    A = _rand(dims, 2)
    for n in range(4):
        M = np.random.default_rng(n).standard_normal((6, dims[n]))
        B = ot.ttm(A, M, n)
        want = np.zeros(B.shape)
        for idx in itertools.product(*[range(d) for d in B.shape]):
            s = 0.0
            for i in range(dims[n]):
                src = list(idx)
                src[n] = i
                s += A[tuple(src)] * M[idx[n], i]
            want[idx] = s
        assert np.allclose(B, want, rtol=1e-13, atol=1e-13)


def test_mode_product_identities():
    # Section 2: (A x_n F) x_m G = (A x_m G) x_n F, (A x_n F) x_n H = A x_n (H F)
    A = _rand((3, 4, 5), 3)
    F = np.random.default_rng(4).standard_normal((6, 4))
    G = np.random.default_rng(5).standard_normal((2, 5))
    H = np.random.default_rng(6).standard_normal((3, 6))
    lhs = ot.ttm(ot.ttm(A, F, 1), G, 2)
    rhs = ot.ttm(ot.ttm(A, G, 2), F, 1)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
    assert np.allclose(ot.ttm(ot.ttm(A, F, 1), H, 1), ot.ttm(A, H @ F, 1), rtol=1e-12, atol=1e-12)


def test_frobenius_matches_inner_product_definition():
    A = _rand((3, 4, 5), 7)
    s = 0.0
    for idx in itertools.product(range(3), range(4), range(5)):
        s += A[idx] * A[idx]
    assert abs(ot.frobenius(A) - np.sqrt(s)) < 1e-12
