"""Tensor-core (tcgen05, split-bf16 operands, fp32 accumulation) power step and
drivers, against the FP64 oracle.

Tolerances come from the arithmetic. A tile of A is held as a_hi + a_lo (two
bf16 words with 8 significant bits each, rounded to nearest: 2^-16 relative at
worst), W = A^T X likewise, and the dropped a_lo w_lo term is at most 2^-16;
sums accumulate in fp32. X_in is rounded to bf16 once (relative 2^-8 at
worst). Against M (M^T bf16(X)) in float64 the Frobenius relative error is
therefore a few times 1e-5 at most (bar: 1e-4). Against the exact product with
X unrounded it is about 2^-9 in the Frobenius norm (bar: 1.5e-2). For whole
decompositions the bar is the relative reconstruction error within 1e-3 of the
oracle's.
"""
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


def bf16(x):
    """Round float64 values to bf16 (nearest even) and back to float64."""
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.float32)))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def colmajor(M):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(M, dtype=np.float32).T)).cuda().t()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    ((400, 60, 50), 30),      # mode 1 of the bench shape (I = 400), ragged fiber tiles
    ((96, 24, 30), 24),       # I < 128
    ((512, 9, 33), 64),       # I = 512 (largest supported), L = 64
    ((130, 70, 21), 13),      # I not a multiple of 8 (scalar loads), L padded to 16
    ((40, 300, 37), 48),      # strided mode-2 fibers with I = 300
    ((17, 23, 19, 21), 5),    # 4th order, every mode
]


@pytest.mark.parametrize("dims,L", CASES)
def test_tc_power_step(tk, dims, L):
    A = synth.lowrank_noise(dims, [min(4, d) for d in dims], rel_noise=0.3, seed=3)
    At = torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()
    A64 = A.astype(np.float64)
    from paper_2303_11612_gb300 import _binding as B
    import ctypes as C
    for n in range(len(dims)):
        if dims[n] > 512:
            continue
        X = np.random.default_rng(n).standard_normal((dims[n], L)).astype(np.float32).astype(np.float64)
        M = ot.unfold(A64, n)
        exact = M @ (M.T @ X)
        ref = M @ (M.T @ bf16(X))
        out = tk.factor_tensor(dims[n], L, torch.float32, "cuda")
        o = B.make_opts(prec="bf16")
        st = B.lib().tucker_power_step(At.data_ptr(), 0, B._i64(dims), len(dims), n, colmajor(X).data_ptr(), L,
                                       out.data_ptr(), C.byref(o))
        assert st == 0, B.lib().tucker_status_string(st)
        got = out.double().cpu().numpy()
        assert rel(got, exact) < 1.5e-2, (dims, n)
        assert rel(got, ref) < 1e-4, (dims, n)


def test_tc_power_step_rejects_unsupported_sizes(tk):
    from paper_2303_11612_gb300 import _binding as B
    import ctypes as C
    dims = (4, 600, 4)
    A = torch.zeros(600 * 16, device="cuda")
    X = torch.zeros((8, 600), device="cuda").t()
    out = torch.zeros((8, 600), device="cuda").t()
    o = B.make_opts(prec="bf16")
    st = B.lib().tucker_power_step(A.data_ptr(), 0, B._i64(dims), 3, 1, X.data_ptr(), 8, out.data_ptr(), C.byref(o))
    assert st == 6                     # strided fibers with I_n > 512: no tensor-core pass takes them


DRIVER_CASES = [
    dict(which="ST", c=0, prob="uniform", q=1),
    dict(which="T", c=0, prob="uniform", q=2),
    dict(which="ST", c=300, prob="nearly_optimal", q=1),
]


@pytest.mark.parametrize("case", DRIVER_CASES, ids=lambda c: "-".join(str(v) for v in c.values()))
@pytest.mark.parametrize("dims,ranks", [((120, 100, 90), (8, 6, 7)), ((40, 36, 32, 30), (4, 5, 3, 6))])
def test_bf16_driver_within_bar(tk, case, dims, ranks):
    case = dict(case)
    which = case.pop("which")
    A = synth.lowrank_noise(dims, ranks, rel_noise=1e-2, seed=31)
    A64 = A.astype(np.float64)
    fn = ot.rthosvd if which == "T" else ot.rsthosvd
    Uo, Go = fn(A64, ranks, P=5, seed=7, **case)
    U, G = tk.decompose(which, torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda(), dims, ranks, P=5,
                        seed=7, prec="bf16", **case)
    U = [u.double().cpu().numpy() for u in U]
    G = synth.from_flat(G.double().cpu().numpy(), ranks)
    assert abs(ot.relative_error(A64, U, G) - ot.relative_error(A64, Uo, Go)) < 1e-3
    for u, uo in zip(U, Uo):
        assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) < 1e-5
        assert np.linalg.norm(u @ u.T - uo @ uo.T, 2) < 1e-2
