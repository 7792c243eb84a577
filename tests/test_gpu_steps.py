"""GPU parity of each step of the path against the FP64 oracle, through the C ABI.

Sizes span several fiber tiles with ragged tails, several column groups, and
each register-tiling variant of the power kernel (I_n up to 256, 512, 1024).
Tolerances (FP32 path): sums of J products carry a relative error of a few
times sqrt(log2 J) * 2^-24 against the FP64 oracle, so 2e-5 relative in the
Frobenius norm; integer work (weights, sampled indices) is bit-exact.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import philox
from oracle import tucker as ot

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    import paper_2303_11612_gb300 as tk
    tk.lib()
    return tk


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def flat_dev(A):
    return dev(synth.flat(A))


def rel(a, b):
    return np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / max(np.linalg.norm(b), 1e-300)


def colmajor(M, dtype=torch.float32):
    M = np.asarray(M)
    return torch.from_numpy(np.ascontiguousarray(M.T)).to(dtype).cuda().t()


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 2e-6), (torch.float64, 1e-13)])
@pytest.mark.parametrize("rows,cols", [(1, 1), (37, 13), (400, 30), (5, 80)])
def test_gaussian(tk, dtype, tol, rows, cols):
    g = tk.gaussian(rows, cols, seed=0xDEADBEEF12345, stream_id=(0 << 8) | 2, dtype=dtype)
    want = philox.gaussian_matrix(0xDEADBEEF12345, 2, rows, cols)
    got = g.double().cpu().numpy()
    assert np.max(np.abs(got - want) / (1 + np.abs(want))) < tol


POWER_CASES = [
    ((9, 13, 7, 11), 5),        # 4th order, tiny rows, tails in every mode
    ((130, 70, 90), 13),        # one column group, ragged tiles
    ((300, 50, 40), 40),        # I > 256 (two rows per thread), two column groups
    ((600, 20, 18), 24),        # I > 512: 16-fiber tiles, 16-column groups
    ((40, 1000, 30), 7),        # L < 8 -> 8-column group
]


@pytest.mark.parametrize("dims,L", POWER_CASES)
def test_power_step_all_modes(tk, dims, L):
    A = synth.lowrank_noise(dims, [min(4, d) for d in dims], rel_noise=0.3, seed=1)
    At = flat_dev(A)
    A64 = A.astype(np.float64)
    for n in range(len(dims)):
        if dims[n] > 1024:
            continue
        X = np.random.default_rng(n).standard_normal((dims[n], L))
        M = ot.unfold(A64, n)
        want = M @ (M.T @ X.astype(np.float32).astype(np.float64))
        got = tk.power_step(At, dims, n, colmajor(X)).double().cpu().numpy()
        assert rel(got, want) < 2e-5, (dims, n)


def test_power_step_fp64(tk):
    dims = (100, 30, 20)
    A = synth.lowrank_noise(dims, (5, 5, 5), rel_noise=0.1, seed=2, dtype=np.float64)
    At = flat_dev(A)
    for n in range(3):
        X = np.random.default_rng(n).standard_normal((dims[n], 15))
        M = ot.unfold(A, n)
        got = tk.power_step(At, dims, n, colmajor(X, torch.float64)).cpu().numpy()
        assert rel(got, M @ (M.T @ X)) < 1e-13


@pytest.mark.parametrize("dims,L", [((50, 40, 33), 9), ((300, 20, 21), 35), ((7, 9, 5, 6), 4)])
def test_range_sketch(tk, dims, L):
    A = synth.lowrank_noise(dims, [3] * len(dims), rel_noise=0.2, seed=3)
    At = flat_dev(A)
    for n in range(len(dims)):
        M = ot.unfold(A.astype(np.float64), n)
        Om = philox.gaussian_matrix(77, n, M.shape[1], L)
        got = tk.range_sketch(At, dims, n, L, seed=77).double().cpu().numpy()
        assert rel(got, M @ Om) < 2e-5


@pytest.mark.parametrize("dims", [(33, 20, 17), (5, 300, 7), (1000, 3, 4), (6, 5, 4, 3), (20, 400, 50), (7, 9, 1100),
                                  (132, 140, 160), (30, 7, 5), (20, 60, 70)])
def test_fiber_norms(tk, dims):
    A = synth.lowrank_noise(dims, [2] * len(dims), rel_noise=0.5, seed=4)
    At = flat_dev(A)
    for n in range(len(dims)):
        want = ot.fiber_weights(ot.unfold(A.astype(np.float64), n), ot.PROB_NEARLY_OPTIMAL)
        got = tk.fiber_norms(At, dims, n).cpu().numpy()
        assert np.max(np.abs(got - want) / want) < 1e-11


def test_quantize_weights_bit_exact(tk):
    rng = np.random.default_rng(5)
    w = rng.pareto(1.2, size=100003) * rng.random(100003)
    w[::17] = 0.0
    got = tk.quantize_weights(dev(w)).cpu().numpy().astype(np.uint64)
    assert np.array_equal(got, ot.quantize_weights(w))
    ones = tk.quantize_weights(dev(w), prob="uniform").cpu().numpy().astype(np.uint64)
    assert np.all(ones == 1)
    zeros = tk.quantize_weights(dev(np.zeros(1000))).cpu().numpy().astype(np.uint64)
    assert np.all(zeros == 1)


@pytest.mark.parametrize("kind", ["mixed", "spiky", "ones"])
@pytest.mark.parametrize("J,T", [(1, 5), (1000, 3), (100000, 4000), (3000, 20000)])
def test_sampler_bit_exact(tk, kind, J, T):
    W = synth.sample_weights(J, seed=6, kind=kind)
    idx, scale = tk.sample_fibers(dev(W.view(np.int64)), T, seed=123456789, mode=2)
    widx, wscale = ot.randsample(W, T, seed=123456789, mode=2)
    assert np.array_equal(idx.cpu().numpy(), widx)
    assert np.array_equal(scale.cpu().numpy(), wscale)


@pytest.mark.parametrize("dims", [(64, 30, 20), (10, 50, 40), (6, 5, 4, 30)])
def test_gather(tk, dims):
    A = synth.lowrank_noise(dims, [2] * len(dims), rel_noise=0.5, seed=7)
    At = flat_dev(A)
    for n in range(len(dims)):
        M = ot.unfold(A.astype(np.float64), n)
        W = ot.quantize_weights(ot.fiber_weights(M, ot.PROB_NEARLY_OPTIMAL))
        idx, scale = ot.randsample(W, 257, seed=9, mode=n)
        got = tk.gather_fibers(At, dims, n, dev(idx), dev(scale)).double().cpu().numpy()
        assert rel(got, ot.amm_matrix(M, idx, scale)) < 1e-7


def _align(U, V):
    s = np.sign(np.sum(U * V, axis=0))
    s[s == 0] = 1
    return U * s


@pytest.mark.parametrize("I,L,R", [(400, 30, 20), (1024, 80, 64), (96, 24, 16), (33, 33, 5), (15, 15, 10)])
def test_leading_factor(tk, I, L, R):
    rng = np.random.default_rng(8)
    Qa, _ = np.linalg.qr(rng.standard_normal((I, L)))
    Qb, _ = np.linalg.qr(rng.standard_normal((L, L)))
    s = 10.0 ** -np.linspace(0, 3, L)                 # distinct singular values
    s[R:] *= 0.5                                      # and a gap after the R-th
    Cm = (Qa * s) @ Qb.T
    Cm = Cm.astype(np.float32).astype(np.float64)
    Uo, _ = ot.leading_left_singular_vectors(Cm, R)
    for dtype, tol in ((torch.float32, 2e-5), (torch.float64, 1e-10)):
        U = tk.leading_factor(colmajor(Cm, dtype), R).double().cpu().numpy()
        # FP32: the Jacobi stops at a pair cosine of 4 eps and the stored factor is
        # rounded once more, so ||U^T U - I||_F stays below 10 R eps_32
        assert np.linalg.norm(U.T @ U - np.eye(R)) < (10 * R * 1.19e-7 if dtype == torch.float32 else 1e-12)
        assert np.linalg.norm(U @ U.T - Uo @ Uo.T, 2) < tol * 10
        assert np.max(np.abs(_align(U, Uo) - Uo)) < tol * 10
        # the sign rule holds on the GPU output itself
        for r in range(R):
            k = np.argmax(np.abs(U[:, r]))
            assert U[k, r] > 0


def test_leading_factor_rank_deficient_sketch(tk):
    """Fewer nonzero singular values than columns: the Gram matrix is singular,
    the shifted pass engages, and the leading subspace is still found."""
    rng = np.random.default_rng(9)
    I, L, R, k = 200, 24, 8, 12
    Cm = rng.standard_normal((I, k)) @ (rng.standard_normal((k, L)) * 10.0 ** -np.linspace(0, 1, L))
    Cm = Cm.astype(np.float32).astype(np.float64)
    Uo, s = ot.leading_left_singular_vectors(Cm, R)
    U = tk.leading_factor(colmajor(Cm), R).double().cpu().numpy()
    assert np.linalg.norm(U.T @ U - np.eye(R)) < 1e-5
    assert np.linalg.norm(U @ U.T - Uo @ Uo.T, 2) < 1e-3


# (64, 48, 40) and (400, 40, 36) take the TMA-fed kernel in every mode (extents
# and slab strides multiples of 4): ragged last index chunks (I = 40, 400),
# slabs narrower than a 128-fiber tile (L_f = 64) and partial tiles (L_f = 400);
# the odd shapes take the register-staged kernel.
@pytest.mark.parametrize("dims", [(30, 20, 17), (7, 6, 5, 4), (100, 3, 2), (64, 48, 40), (400, 40, 36)])
@pytest.mark.parametrize("transpose", [False, True])
def test_ttm(tk, dims, transpose):
    A = synth.lowrank_noise(dims, [2] * len(dims), rel_noise=0.5, seed=10)
    At = flat_dev(A)
    for n in range(len(dims)):
        K = 70 if n == 0 else 3
        M = np.random.default_rng(n).standard_normal((K, dims[n]))
        Mp = M.T if transpose else M
        got = tk.ttm(At, dims, n, colmajor(Mp), transpose=transpose).double().cpu().numpy()
        out_dims = list(dims)
        out_dims[n] = K
        want = synth.flat(ot.ttm(A.astype(np.float64), M.astype(np.float32).astype(np.float64), n))
        assert rel(got, want) < 1e-6


def test_relative_error_explicit(tk):
    dims, ranks = (40, 30, 20), (4, 5, 3)
    A = synth.lowrank_noise(dims, ranks, rel_noise=0.05, seed=11)
    Us, G = ot.rsthosvd(A.astype(np.float64), ranks, P=3, q=1)
    want = ot.relative_error(A.astype(np.float64), Us, G)
    got = tk.relative_error(flat_dev(A), dims, ranks, [colmajor(U) for U in Us],
                            dev(synth.flat(G).astype(np.float32)))
    assert abs(got - want) < 1e-6


def test_bounded_wait_times_out_and_the_context_survives(tk):
    """A device wait that nothing completes ends after its bound with the
    timeout status (as every tensor-core kernel's waits do), frees its tensor
    memory, and the next decomposition on the same context is unaffected."""
    from paper_2303_11612_gb300 import _binding as B
    assert B.check_wait_timeout(1000) == 5                      # TUCKER_ERR_TIMEOUT
    assert B.check_wait_timeout(1) == 5
    assert B.check_wait_timeout(0) == 1                         # TUCKER_ERR_INVALID_ARG
    dims, ranks = (48, 40, 36), (6, 5, 4)
    A = synth.lowrank_noise(dims, ranks, rel_noise=1e-3, seed=1)
    At = torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()
    for prec in ("fp32", "bf16x1"):
        U, G = tk.rsthosvd(At, dims, ranks, P=4, q=1, prec=prec)
        assert tk.last_device_status() == 0
        re = ot.relative_error(A.astype(np.float64), [u.double().cpu().numpy() for u in U],
                               synth.from_flat(G.double().cpu().numpy(), ranks))
        assert re < 2e-3
