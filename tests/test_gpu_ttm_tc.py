"""Mode-n product on the tensor cores with split-bf16 operands (tucker_ttm with
prec BF16/TF32), against the FP64 oracle's unfolding.

Each operand x is held as hi + lo with hi = bf16(x) (8-bit significand,
rounded to nearest: relative error <= 2^-8) and lo = bf16(x - hi) (x - hi is
exact in FP32; lo carries it to 2^-8 of itself), so hi + lo is x to 2^-16. The
product keeps hi*hi + lo*hi + hi*lo; per term the error is at most about
3 x 2^-16 |a||m| (the two representation errors and the dropped lo*lo), the
bf16 x bf16 products are exact in FP32, and the FP32 accumulation of the 3 I_n
products adds at most 3 I_n 2^-24 sum |a||m|. The bound (with a factor 4 for
the second-order terms) is checked elementwise against sum_i |a_i||m_i|. The
structural check evaluates the same three products in float64 from the same
bf16 parts and must agree to the accumulation error alone; a wrong tile, a
transposed operand or a dropped unit fails it by orders of magnitude.
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
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.float32)))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def split(x):
    x32 = np.asarray(x, dtype=np.float32).astype(np.float64)
    hi = bf16(x32)
    lo = bf16((x32 - hi).astype(np.float32))
    return hi, lo


CASES = [
    ((400, 60, 50), 20),      # the bench's mode-1 shape on 3000 fibers: ragged 128-fiber tiles
    ((400, 200, 160), 20),    # 250 tiles: the unit rings wrap within and across tiles
    ((64, 300, 70), 32),      # one unit per tile, K_out = 32 (widest)
    ((132, 70, 21), 13),      # I_n not a multiple of 64: partial and wholly zero-filled boxes
    ((512, 9, 33), 32),       # largest I_n
    ((4, 700, 3), 1),         # one box, K_out = 1
]


@pytest.mark.parametrize("dims,K", CASES)
def test_split_bf16_mode_product(tk, dims, K):
    A = synth.lowrank_noise(dims, [min(4, d) for d in dims], rel_noise=0.3, seed=9)
    At = torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()
    U = np.random.default_rng(2).standard_normal((dims[0], K)).astype(np.float32)
    Ut = torch.from_numpy(np.ascontiguousarray(U.T)).cuda().t()          # I_n x K, column-major
    got = tk.ttm(At, dims, 0, Ut, transpose=True, prec="bf16").double().cpu().numpy()
    M = ot.unfold(A.astype(np.float64), 0)                                # I_n x J
    J = M.shape[1]
    got = got.reshape(J, K)                                               # out[j * K + o]
    exact = M.T @ U.astype(np.float64)
    absprod = np.abs(M.T) @ np.abs(U.astype(np.float64))
    I = dims[0]
    bound = (4 * 2.0 ** -16 + 4 * I * 2.0 ** -24) * absprod
    assert np.all(np.abs(got - exact) <= bound + 1e-30)
    Mh, Ml = split(M)
    Uh, Ul = split(U)
    emul = Mh.T @ Uh + Ml.T @ Uh + Mh.T @ Ul
    assert np.all(np.abs(got - emul) <= 4 * I * 2.0 ** -24 * absprod + 1e-30)


def test_split_bf16_mode_product_same_for_tf32_option(tk):
    dims, K = (96, 50, 40), 12
    A = torch.from_numpy(np.ascontiguousarray(synth.flat(synth.lowrank_noise(dims, (3, 3, 3), 0.1, seed=4)))).cuda()
    U = torch.randn(K, 96, device="cuda").t()
    assert torch.equal(tk.ttm(A, dims, 0, U, transpose=True, prec="bf16"),
                       tk.ttm(A, dims, 0, U, transpose=True, prec="tf32"))


def test_split_bf16_mode_product_rejects_unsupported(tk):
    dims = (40, 36, 32)
    A = torch.randn(40 * 36 * 32, device="cuda")
    with pytest.raises(tk.TuckerError):
        tk.ttm(A, dims, 1, torch.randn(8, 36, device="cuda").t(), transpose=True, prec="bf16")   # strided
    with pytest.raises(tk.TuckerError):
        tk.ttm(A, dims, 0, torch.randn(130, 40, device="cuda").t(), transpose=True, prec="bf16")  # K > 128
    with pytest.raises(tk.TuckerError):                                   # not 16-byte aligned for TMA
        tk.ttm(A[1:1 + 40 * 36 * 31], (40, 36, 31), 0, torch.randn(8, 40, device="cuda").t(), transpose=True,
               prec="bf16")
    A42 = torch.randn(42 * 36 * 32, device="cuda")
    with pytest.raises(tk.TuckerError):
        tk.ttm(A42, (42, 36, 32), 0, torch.randn(8, 42, device="cuda").t(), transpose=True, prec="bf16")
