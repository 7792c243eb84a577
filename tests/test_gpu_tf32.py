"""Tensor-core power step with TF32 operands (tcgen05 kind::tf32, fp32
accumulation), against the FP64 oracle's unfoldings.

TF32 keeps 10 explicit mantissa bits: an operand is represented to 2^-11
relative when rounded to nearest and 2^-10 when truncated. The step rounds A
and X_in when they enter the first product and W = A^T X when it enters the
second, so against the exact product the Frobenius relative error is at most
about 3 x 2^-10 ~ 3e-3 (bar: 5e-3). The structural check is tighter: the same
product evaluated in float64 from TF32-rounded operands (A, X and the fp32 W)
must match to fp32 accumulation error (bar: 1e-4), under truncation or under
round-to-nearest, whichever the tensor cores apply; a transposed operand, a
wrong tile or a dropped fiber fails it by orders of magnitude.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from oracle import tucker as ot

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    import paper_2303_11612_gb300 as tk
    tk.lib()
    return tk


def tf32(x, nearest):
    u = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32)
    if nearest:
        u = u + np.uint32(0x1000)
    return (u & np.uint32(0xFFFFE000)).view(np.float32).astype(np.float64)


def colmajor(M):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(M, dtype=np.float32).T)).cuda().t()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def power_tf32(tk, At, dims, n, X):
    from paper_2303_11612_gb300 import _binding as B
    L = X.shape[1]
    out = tk.factor_tensor(dims[n], L, torch.float32, "cuda")
    o = B.make_opts(prec="tf32")
    st = B.lib().tucker_power_step(At.data_ptr(), 0, B._i64(dims), len(dims), n, colmajor(X).data_ptr(), L,
                                   out.data_ptr(), C.byref(o))
    return st, out


CASES = [
    ((400, 60, 50), 30),      # the bench's I_n and L_n, one ragged 64-fiber tile per CTA
    ((400, 160, 100), 30),    # 250 tiles: the sub-stage ring wraps within and across tiles
    ((400, 200, 160), 30),    # 500 tiles: 3-4 per CTA
    ((64, 200, 100), 17),     # small I_n (one sub-stage per tile), 313 tiles
    ((96, 24, 30), 24),       # I_n < 128
    ((512, 9, 33), 32),       # largest I_n and L_n (four full sub-stages)
    ((132, 70, 21), 13),      # I_n not a multiple of 32: zero-filled chunk tail
    ((4, 700, 3), 5),         # one chunk, mostly padding
]


@pytest.mark.parametrize("dims,L", CASES)
def test_tf32_power_step(tk, dims, L):
    A = synth.lowrank_noise(dims, [min(4, d) for d in dims], rel_noise=0.3, seed=5)
    At = torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()
    M = ot.unfold(A.astype(np.float64), 0)
    X = np.random.default_rng(1).standard_normal((dims[0], L)).astype(np.float32).astype(np.float64)
    st, out = power_tf32(tk, At, dims, 0, X)
    assert st == 0
    got = out.double().cpu().numpy()
    exact = M @ (M.T @ X)
    assert rel(got, exact) < 5e-3
    errs = []
    for nearest in (False, True):
        Mt, Xt = tf32(M, nearest), tf32(X, nearest)
        W = (Mt.T @ Xt).astype(np.float32)
        errs.append(rel(got, Mt @ tf32(W, nearest)))
    assert min(errs) < 1e-4, errs


def test_tf32_power_step_rejects_unsupported(tk):
    dims = (40, 36, 32)
    A = torch.randn(40 * 36 * 32, device="cuda")
    X = np.zeros((36, 8))
    assert power_tf32(tk, A, dims, 1, X)[0] == 6               # strided fibers
    assert power_tf32(tk, A, dims, 0, np.zeros((40, 130)))[0] == 6  # L > 128 (no tensor-core pass)
    dims = (42, 36, 32)
    A = torch.randn(42 * 36 * 32, device="cuda")
    assert power_tf32(tk, A, dims, 0, np.zeros((42, 8)))[0] == 6    # I_n not a multiple of 4
    dims = (40, 36, 32)
    A = torch.randn(40 * 36 * 32 + 1, device="cuda")[1:]      # not 16-byte aligned for TMA
    assert power_tf32(tk, A, dims, 0, np.zeros((40, 8)))[0] == 6


DRIVER_CASES = [
    dict(which="ST", c=0, prob="uniform", q=1),
    dict(which="T", c=0, prob="uniform", q=2),
    dict(which="ST", c=300, prob="nearly_optimal", q=1),
]


@pytest.mark.parametrize("case", DRIVER_CASES, ids=lambda c: "-".join(str(v) for v in c.values()))
@pytest.mark.parametrize("dims,ranks", [((120, 100, 90), (8, 6, 7)), ((40, 36, 32, 30), (4, 5, 3, 6))])
def test_tf32_driver_within_bar(tk, case, dims, ranks):
    """Whole decompositions in the TF32 form: relative error within 1e-3 of the
    oracle's (the bar the tensor-core forms are held to)."""
    case = dict(case)
    which = case.pop("which")
    A = synth.lowrank_noise(dims, ranks, rel_noise=1e-2, seed=31)
    A64 = A.astype(np.float64)
    fn = ot.rthosvd if which == "T" else ot.rsthosvd
    Uo, Go = fn(A64, ranks, P=5, seed=7, **case)
    U, G = tk.decompose(which, torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda(), dims, ranks, P=5,
                        seed=7, prec="tf32", **case)
    U = [u.double().cpu().numpy() for u in U]
    G = synth.from_flat(G.double().cpu().numpy(), ranks)
    assert abs(ot.relative_error(A64, U, G) - ot.relative_error(A64, Uo, Go)) < 1e-3
    for u, uo in zip(U, Uo):
        assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) < 1e-5
        assert np.linalg.norm(u @ u.T - uo @ uo.T, 2) < 1e-2
