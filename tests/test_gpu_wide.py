"""Tensor-core passes for contiguous fibers beyond the fused kernels' tiles
(kernels_wide.cu): extents I_n up to 1024 and sketch widths / output ranks up
to 128, the shapes of the 1024 x 1024 x 512 workload's first mode (I = 1024,
L = 80, R = 64). Against the FP64 oracle's unfoldings and Philox stream.

Split-bf16 operands (prec BF16, and TF32 at these shapes): every FP32 operand is
a_hi + a_lo to 2^-16 and each pass keeps hi.hi + lo.hi + hi.lo, so a power step
(two passes, W = A^T X split again between them) is the exact product to about
6 x 2^-16 ~ 1e-4 relative in the Frobenius norm (bar 2e-4); the mode product
is checked elementwise as in the fused kernel's test. Single-pass bf16 (prec
BF16X1): A, X and W each rounded once, about 3 x 2^-8 against the exact product
(bar 3e-2), and within 5e-4 of the same product evaluated in float64 from the
same bf16 roundings, which a wrong tile, a transposed operand or a dropped
chunk fails by orders of magnitude.
"""
import ctypes as C

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


def bf16(x):
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.float32)))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def split(x):
    x32 = np.asarray(x, dtype=np.float32).astype(np.float64)
    hi = bf16(x32)
    lo = bf16((x32 - hi).astype(np.float32))
    return hi, lo


def colmajor(M):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(M, dtype=np.float32).T)).cuda().t()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def tensor(dims, seed):
    A = synth.lowrank_noise(dims, [min(6, d) for d in dims], rel_noise=0.3, seed=seed)
    return A, torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()


def step(tk, At, dims, X, prec):
    from paper_2303_11612_gb300 import _binding as B
    L = X.shape[1]
    out = tk.factor_tensor(dims[0], L, torch.float32, "cuda")
    o = B.make_opts(prec=prec)
    st = B.lib().tucker_power_step(At.data_ptr(), 0, B._i64(dims), len(dims), 0, colmajor(X).data_ptr(), L,
                                   out.data_ptr(), C.byref(o))
    return st, out.double().cpu().numpy()


POWER = [
    ((1024, 40, 30), 80),     # the 1024^2 x 512 workload's I_1 and L_1 on 1200 fibers (ragged chunk and tile)
    ((1020, 33, 17), 70),     # I_n not a multiple of 64: partial row blocks and zero-filled boxes
    ((600, 100, 50), 48),     # five row blocks: two row groups of 4 and 1
    ((520, 300, 10), 16),     # just past the fused tiles (I_n > 512), 3000 fibers: the rings wrap many times
    ((64, 50, 50), 128),      # the widest sketch
    ((1024, 8, 8), 1),        # one column
    ((1024, 20000, 1), 80),   # the shape of the gathered AMM sample (c = 20000)
]


@pytest.mark.parametrize("dims,L", POWER)
def test_wide_power_step_split(tk, dims, L):
    """Every case lies beyond the fused kernels' tiles (I_n > 512 or L > 64),
    where the two passes run (the fused split kernel rounds X to bf16 once)."""
    A, At = tensor(dims, 3)
    X = np.random.default_rng(L).standard_normal((dims[0], L)).astype(np.float32)
    M = ot.unfold(A.astype(np.float64), 0)
    exact = M @ (M.T @ X.astype(np.float64))
    st, got = step(tk, At, dims, X, "bf16")
    assert st == 0
    assert rel(got, exact) < 2e-4
    st2, got2 = step(tk, At, dims, X, "tf32")              # the TF32 form takes the same passes here
    assert st2 == 0 and np.array_equal(got, got2)


@pytest.mark.parametrize("dims,L", POWER)
def test_wide_power_step_single(tk, dims, L):
    A, At = tensor(dims, 4)
    X = np.random.default_rng(L + 1).standard_normal((dims[0], L)).astype(np.float32)
    M = ot.unfold(A.astype(np.float64), 0)
    st, got = step(tk, At, dims, X, "bf16x1")
    assert st == 0
    assert rel(got, M @ (M.T @ X.astype(np.float64))) < 3e-2
    Mb = bf16(M)
    W = (Mb.T @ bf16(X)).astype(np.float32)
    assert rel(got, Mb @ bf16(W)) < 5e-4


# every case lies beyond the fused mode product (I_n > 512 or K_out > 32)
TTM = [((1024, 40, 30), 64), ((1020, 33, 17), 50), ((600, 100, 50), 128), ((520, 300, 10), 1), ((64, 50, 50), 100)]


@pytest.mark.parametrize("dims,K", TTM)
def test_wide_mode_product(tk, dims, K):
    A, At = tensor(dims, 5)
    U = np.random.default_rng(K).standard_normal((dims[0], K)).astype(np.float32)
    Ut = torch.from_numpy(np.ascontiguousarray(U.T)).cuda().t()
    got = tk.ttm(At, dims, 0, Ut, transpose=True, prec="bf16").double().cpu().numpy()
    M = ot.unfold(A.astype(np.float64), 0)
    J = M.shape[1]
    got = got.reshape(J, K)                                               # out[j * K + o]
    exact = M.T @ U.astype(np.float64)
    absprod = np.abs(M.T) @ np.abs(U.astype(np.float64))
    I = dims[0]
    assert np.all(np.abs(got - exact) <= (4 * 2.0 ** -16 + 4 * I * 2.0 ** -24) * absprod + 1e-30)
    Mh, Ml = split(M)
    Uh, Ul = split(U)
    emul = Mh.T @ Uh + Ml.T @ Uh + Mh.T @ Ul
    assert np.all(np.abs(got - emul) <= 4 * I * 2.0 ** -24 * absprod + 1e-30)


@pytest.mark.parametrize("dims,L", [((1024, 40, 30), 80), ((400, 60, 50), 30), ((1020, 33, 17), 70),
                                    ((64, 50, 50), 128)])
def test_wide_range_sketch(tk, dims, L):
    """Y = A_(1) Omega with Omega generated inside the kernel from the Philox
    stream (element j L + l of the mode's purpose-0 stream): split bf16 within
    2e-4 of the exact product with the oracle's Omega; single-pass bf16 within
    3e-2, and within 5e-4 of the product of the bf16 roundings."""
    A, At = tensor(dims, 6)
    M = ot.unfold(A.astype(np.float64), 0)
    Om = philox.gaussian_matrix(77, 0, M.shape[1], L)
    exact = M @ Om
    got = tk.range_sketch(At, dims, 0, L, seed=77, prec="bf16").double().cpu().numpy()
    assert rel(got, exact) < 2e-4
    got1 = tk.range_sketch(At, dims, 0, L, seed=77, prec="bf16x1").double().cpu().numpy()
    assert rel(got1, exact) < 3e-2
    assert rel(got1, bf16(M) @ bf16(Om)) < 5e-4


def step_mode(tk, At, dims, n, X, prec):
    from paper_2303_11612_gb300 import _binding as B
    L = X.shape[1]
    out = tk.factor_tensor(dims[n], L, torch.float32, "cuda")
    o = B.make_opts(prec=prec)
    st = B.lib().tucker_power_step(At.data_ptr(), 0, B._i64(dims), len(dims), n, colmajor(X).data_ptr(), L,
                                   out.data_ptr(), C.byref(o))
    return st, out.double().cpu().numpy()


# strided fibers (modes 2..N) with a stride that is a multiple of 32
STRIDED = [
    ((64, 1024, 40), 1, 80),      # the 1024^2 x 512 workload's second mode (after truncation) on 40 slabs
    ((96, 600, 20), 1, 48),       # stride 96: groups of 32 fibers, chunks straddling slabs
    ((32, 40, 60, 30), 2, 16),    # 4th order, stride 1280, I_n = 60 (zero-filled boxes)
    ((32, 520, 9), 1, 70),        # 288 fibers: ragged last tile and chunk, beyond the last slab
]


@pytest.mark.parametrize("dims,n,L", STRIDED)
def test_wide_power_step_strided(tk, dims, n, L):
    A, At = tensor(dims, 7)
    X = np.random.default_rng(L).standard_normal((dims[n], L)).astype(np.float32)
    M = ot.unfold(A.astype(np.float64), n)
    exact = M @ (M.T @ X.astype(np.float64))
    prec = "bf16" if dims[n] > 512 or L > 64 else None
    if prec:                                   # beyond the fused split kernel: the two passes run
        st, got = step_mode(tk, At, dims, n, X, "bf16")
        assert st == 0 and rel(got, exact) < 2e-4
    st, got = step_mode(tk, At, dims, n, X, "bf16x1")
    assert st == 0
    assert rel(got, exact) < 3e-2
    Mb = bf16(M)
    assert rel(got, Mb @ bf16((Mb.T @ bf16(X)).astype(np.float32))) < 5e-4


@pytest.mark.parametrize("dims,n,K", [((64, 1024, 40), 1, 64), ((96, 600, 20), 1, 50), ((32, 40, 60, 30), 2, 40),
                                      ((32, 520, 9), 1, 128)])
def test_wide_mode_product_strided(tk, dims, n, K):
    """out(l, o, r) = sum_i A(l, i, r) M(i, o): the output keeps the tensor's layout
    (mode n replaced by K), written by lanes of consecutive l."""
    A, At = tensor(dims, 8)
    U = np.random.default_rng(K).standard_normal((dims[n], K)).astype(np.float32)
    Ut = torch.from_numpy(np.ascontiguousarray(U.T)).cuda().t()
    got = tk.ttm(At, dims, n, Ut, transpose=True, prec="bf16").double().cpu().numpy()
    M = ot.unfold(A.astype(np.float64), n)
    outdims = list(dims)
    outdims[n] = K
    got = ot.unfold(synth.from_flat(got, outdims), n).T                   # J x K
    exact = M.T @ U.astype(np.float64)
    absprod = np.abs(M.T) @ np.abs(U.astype(np.float64))
    I = dims[n]
    assert np.all(np.abs(got - exact) <= (4 * 2.0 ** -16 + 4 * I * 2.0 ** -24) * absprod + 1e-30)


def test_wide_range_sketch_strided(tk):
    dims, L = (64, 600, 30), 70
    A, At = tensor(dims, 9)
    M = ot.unfold(A.astype(np.float64), 1)
    Om = philox.gaussian_matrix(5, 1, M.shape[1], L)
    got = tk.range_sketch(At, dims, 1, L, seed=5, prec="bf16").double().cpu().numpy()
    assert rel(got, M @ Om) < 2e-4


def test_wide_rejects_what_it_cannot_take(tk):
    from paper_2303_11612_gb300 import _binding as B
    dims = (1024, 4, 4)
    A = torch.zeros(1024 * 16 + 1, device="cuda")[1:]                   # not 16-byte aligned for TMA
    st, _ = step(tk, A, dims, np.zeros((1024, 80), np.float32), "bf16")
    assert st == 6
    with pytest.raises(tk.TuckerError):                                   # stride 40: not a multiple of 32
        tk.range_sketch(torch.zeros(40 * 36 * 32, device="cuda"), (40, 36, 32), 1, 8, seed=1, prec="bf16")


DRIVER = [
    ((1024, 96, 40), (64, 16, 8), 16),
    ((600, 80, 60), (40, 10, 12), 10),
    ((640, 600, 8), (32, 32, 4), 16),       # the second mode strided (stride 32) with I_n = 600
]
FORMS = ["bf16x1", "bf16", "tf32"]


@pytest.mark.parametrize("which", ["ST", "T"])
@pytest.mark.parametrize("c", [0, 2000])
@pytest.mark.parametrize("dims,ranks,P", DRIVER)
def test_wide_drivers_against_the_oracle(tk, which, c, dims, ranks, P):
    """Whole decompositions whose first mode (and the gathered AMM samples) run
    through the tensor-core passes: relative error within 1e-3 of the oracle's
    in every tensor-core form, factors orthonormal."""
    A = synth.lowrank_noise(dims, [r + 2 for r in ranks], rel_noise=1e-2, seed=11)
    A64 = A.astype(np.float64)
    fn = ot.rthosvd if which == "T" else ot.rsthosvd
    Uo, Go = fn(A64, ranks, P=P, q=1, c=c, prob="uniform", seed=5)
    reo = ot.relative_error(A64, Uo, Go)
    At = torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()
    for prec in FORMS:
        U, G = tk.decompose(which, At, dims, ranks, P=P, q=1, c=c, prob="uniform", seed=5, prec=prec)
        U = [u.double().cpu().numpy() for u in U]
        G = synth.from_flat(G.double().cpu().numpy(), ranks)
        assert abs(ot.relative_error(A64, U, G) - reo) < 1e-3, prec
        for u in U:
            assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) < 1e-4, prec


@pytest.mark.parametrize("prec", ["bf16", "bf16x1"])
def test_wide_range_form_driver(tk, prec):
    """The range form with its first pass Y = A Omega on the tensor cores:
    relative error within 1e-3 of the oracle's range form."""
    dims, ranks = (1024, 64, 30), (48, 10, 8)
    A = synth.lowrank_noise(dims, [r + 2 for r in ranks], rel_noise=1e-2, seed=12)
    A64 = A.astype(np.float64)
    Uo, Go = ot.rsthosvd(A64, ranks, P=10, q=1, seed=9, form="range")
    reo = ot.relative_error(A64, Uo, Go)
    At = torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()
    U, G = tk.decompose("ST", At, dims, ranks, P=10, q=1, seed=9, form="range", prec=prec)
    U = [u.double().cpu().numpy() for u in U]
    G = synth.from_flat(G.double().cpu().numpy(), ranks)
    assert abs(ot.relative_error(A64, U, G) - reo) < 1e-3
