"""Strategy B (remark after Algorithm 1) on the GPU: tucker_gram and the drivers
that use it.

- G = A_(n) A_(n)^T from the tensor-core pass, elementwise against the exact
  product (float64) within 4 * 2^-16 (|A_(n)| |A_(n)|^T)_ij (split bf16 drops the
  lo.lo term, ~2^-16 relative per product), and against the same three bf16
  products evaluated in float64 within 2e-6 of that scale (FP32 accumulation):
  contiguous fibers (mode 1) and strides that are multiples of 32, I_n from 32 to
  128, fiber counts with a ragged last chunk.
- Requests the kernel cannot take (I_n > 128, FP32 arithmetic, FP64 data) are
  refused with TUCKER_ERR_UNSUPPORTED.
- The drivers with q >= 2 in a tensor-core form (every mode the kernel can take
  goes the Gram route; tucker_plan_describe says so) match the oracle: RE within 1e-4
  and projectors within 1e-3 where the sketch has a gap at R_n."""
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


def bf16_parts(x):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    hi = t.to(torch.bfloat16).to(torch.float32)
    lo = (t - hi).to(torch.bfloat16).to(torch.float32)
    return hi.double().numpy(), lo.double().numpy()


@pytest.mark.parametrize("dims,mode", [((96, 300, 7), 0), ((128, 64, 33), 0), ((32, 1000, 3), 0), ((100, 50, 40), 0),
                                       ((64, 120, 30), 1), ((32, 20, 128), 2), ((64, 7, 90), 2)])
def test_gram_against_the_exact_product(tk, dims, mode):
    from paper_2303_11612_gb300 import _binding as B
    A = np.random.default_rng(sum(dims) + mode).standard_normal(dims).astype(np.float32)
    A[..., :1] *= 100.0                                 # uneven magnitudes across the fibers
    M = ot.unfold(A.astype(np.float64), mode)
    At = torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()
    G = B.gram(At, dims, mode).double().cpu().numpy()
    exact = M @ M.T
    scale = np.abs(M) @ np.abs(M).T
    assert np.all(np.abs(G - exact) <= 4 * 2.0 ** -16 * scale + 1e-30)
    hi, lo = bf16_parts(ot.unfold(A, mode))
    same = hi @ hi.T + lo @ hi.T + hi @ lo.T
    assert np.all(np.abs(G - same) <= 2e-6 * scale + 1e-30)
    assert np.allclose(G, G.T, rtol=0, atol=1e-6 * scale.max())


def test_gram_refuses_what_it_cannot_take(tk):
    from paper_2303_11612_gb300 import _binding as B
    A = torch.zeros(200 * 10 * 10, dtype=torch.float32, device="cuda")
    with pytest.raises(B.TuckerError):
        B.gram(A, (200, 10, 10), 0)                     # I_n > 128
    with pytest.raises(B.TuckerError):
        B.gram(A, (20, 100, 10), 0, prec="fp32")
    with pytest.raises(B.TuckerError):
        B.gram(A.double(), (20, 100, 10), 0)


@pytest.mark.parametrize("prec", ["bf16", "bf16x1", "tf32"])
@pytest.mark.parametrize("which", ["ST", "T"])
def test_drivers_with_strategy_b_match_the_oracle(tk, prec, which):
    dims, ranks = (96, 80, 64), (8, 6, 5)
    A = synth.lowrank_noise(dims, ranks, rel_noise=1e-2, seed=9)
    A64 = A.astype(np.float64)
    plan = tk.plan_describe(which, dims, ranks, P=6, q=2, prec=prec)
    # T-HOSVD: every mode of the input; ST-HOSVD: mode 1 only (the truncated tensor's
    # later modes have strides R_1 = 8 and 8 R_2, not multiples of 32: Strategy A there)
    assert plan.count("power=gram-split-bf16") == (3 if which == "T" else 1), plan
    At = torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()
    U, G = tk.decompose(which, At, dims, ranks, P=6, q=2, seed=4, prec=prec)
    fn = ot.rsthosvd if which == "ST" else ot.rthosvd
    info = {}
    Uo, Go = fn(A64, ranks, P=6, q=2, seed=4, info=info)
    Ud = [u.double().cpu().numpy() for u in U]
    re = ot.relative_error(A64, Ud, synth.from_flat(G.double().cpu().numpy(), ranks))
    reo = ot.relative_error(A64, Uo, Go)
    assert abs(re - reo) <= 1e-4, (re, reo)
    for n, (u, uo) in enumerate(zip(Ud, Uo)):
        assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) < 10 * u.shape[1] * 1.19e-7
        s = info["sigma_C"][n]
        if s[ranks[n] - 1] >= 1.5 * s[ranks[n]]:
            assert np.linalg.norm(u @ u.T - uo @ uo.T, 2) <= 1e-3, n
