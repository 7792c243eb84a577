"""Mode-1 and mode-2 fiber norms from one pass (tucker_fiber_norms12; the
nearly-optimal probabilities of the remark after Algorithm 3, for modes 1 and 2
of Algorithm 4).

- Against the oracle's squared fiber norms (FP64 sums of the exact squares)
  within 1e-11 relative, FP32 and FP64 data, orders 2 to 4, ragged extents.
- Mode 1 bitwise that of tucker_fiber_norms where that takes a warp per fiber
  (I_1 >= 64: the same summation order); mode 2 within 1e-12 relative of it.
- I_1 > 1024 and N < 2 are refused.
- Algorithm 4 with the nearly-optimal probabilities (which forms both modes'
  norms in this pass) matches the oracle, sampled fiber indices of every mode
  bit-exact."""
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


def flat_dev(A):
    return torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("dims", [(400, 300, 7), (64, 33, 20), (1024, 5, 3), (37, 50, 40, 3), (100, 80), (129, 1, 9),
                                  (1, 40, 30), (513, 70, 2, 2)])
def test_norms12_against_the_oracle_and_the_per_mode_kernel(tk, dims, dtype):
    A = synth.lowrank_noise(dims, [min(2, d) for d in dims], rel_noise=0.5, seed=len(dims), dtype=dtype)
    At = flat_dev(A)
    w1, w2 = tk.fiber_norms12(At, dims)
    A64 = A.astype(np.float64)
    for n, w in ((0, w1), (1, w2)):
        want = ot.fiber_weights(ot.unfold(A64, n), ot.PROB_NEARLY_OPTIMAL)
        got = w.cpu().numpy()
        assert got.shape == want.shape
        assert np.max(np.abs(got - want) / want) < 1e-11, n
    one1 = tk.fiber_norms(At, dims, 0).cpu().numpy()
    one2 = tk.fiber_norms(At, dims, 1).cpu().numpy()
    if dims[0] >= 64:
        assert np.array_equal(w1.cpu().numpy(), one1)
    else:
        assert np.max(np.abs(w1.cpu().numpy() - one1) / one1) < 1e-12
    assert np.max(np.abs(w2.cpu().numpy() - one2) / one2) < 1e-12


def test_norms12_refusals(tk):
    from paper_2303_11612_gb300 import _binding as B
    A = torch.zeros(1100 * 3 * 2, dtype=torch.float32, device="cuda")
    with pytest.raises(B.TuckerError) as e:
        tk.fiber_norms12(A, (1100, 3, 2))
    assert e.value.status == 6
    with pytest.raises((B.TuckerError, ValueError)):
        tk.fiber_norms12(A[:1100], (1100,))


@pytest.mark.parametrize("dims,ranks", [((400, 300, 20), (10, 8, 5)), ((60, 50, 40), (5, 4, 6)),
                                        ((30, 25, 20, 15), (4, 3, 3, 2))])
@pytest.mark.parametrize("q", [1, 2])
def test_algorithm4_nearly_optimal_matches_the_oracle(tk, dims, ranks, q):
    A = synth.lowrank_noise(dims, ranks, rel_noise=1e-2, seed=31)
    A64 = A.astype(np.float64)
    c = 300
    info = {}
    Uo, Go = ot.rthosvd(A64, ranks, P=5, q=q, c=c, prob="nearly_optimal", seed=9, info=info)
    U, G, re, samples = tk.decompose("T", flat_dev(A), dims, ranks, P=5, q=q, c=c, prob="nearly_optimal", seed=9,
                                     want_rel_error=True, want_samples=True)
    Ud = [u.double().cpu().numpy() for u in U]
    Gd = synth.from_flat(G.double().cpu().numpy(), ranks)
    assert abs(ot.relative_error(A64, Ud, Gd) - ot.relative_error(A64, Uo, Go)) < 1e-5
    for n in range(len(dims)):
        got = samples[n].cpu().numpy()[: len(info["idx"][n])]
        assert np.array_equal(got, info["idx"][n]), n
        s = info["sigma_C"][n]
        if s[ranks[n] - 1] >= 1.5 * s[ranks[n]]:
            assert np.linalg.norm(Ud[n] @ Ud[n].T - Uo[n] @ Uo[n].T, 2) < 1e-4, n


ORDER3 = [(400, 300, 7), (64, 33, 20), (1024, 5, 3), (129, 1, 9), (1, 40, 30), (513, 70, 2), (37, 50, 40),
          (100, 80, 1), (7, 300, 129), (257, 17, 65)]


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("dims", ORDER3)
def test_norms123_against_the_oracle_and_the_per_mode_kernel(tk, dims, dtype):
    """The three modes of an order-3 tensor from one pass (tucker_fiber_norms123):
    each against the oracle's squared fiber norms; mode 1 bitwise the per-mode
    kernel's where that takes a warp per fiber; modes 2 and 3 within 1e-12."""
    A = synth.lowrank_noise(dims, [min(2, d) for d in dims], rel_noise=0.5, seed=sum(dims), dtype=dtype)
    At = flat_dev(A)
    w1, w2, w3 = tk.fiber_norms123(At, dims)
    A64 = A.astype(np.float64)
    for n, w in ((0, w1), (1, w2), (2, w3)):
        want = ot.fiber_weights(ot.unfold(A64, n), ot.PROB_NEARLY_OPTIMAL)
        got = w.cpu().numpy()
        assert got.shape == want.shape
        assert np.max(np.abs(got - want) / want) < 1e-11, n
        one = tk.fiber_norms(At, dims, n).cpu().numpy()
        if n == 0 and dims[0] >= 64:
            assert np.array_equal(got, one)
        else:
            assert np.max(np.abs(got - one) / one) < 1e-12, n
    # the same bytes through a caller workspace of exactly the stated size
    nb = tk.fiber_norms123_workspace_size(dims)
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    again = tk.fiber_norms123(At, dims, workspace=scratch)
    for a, b in zip(again, (w1, w2, w3)):
        assert torch.equal(a, b)


def test_norms123_refusals(tk):
    from paper_2303_11612_gb300 import _binding as B
    A = torch.zeros(1100 * 3 * 2, dtype=torch.float32, device="cuda")
    with pytest.raises(B.TuckerError) as e:
        tk.fiber_norms123(A, (1100, 3, 2))
    assert e.value.status == 6
    with pytest.raises((B.TuckerError, ValueError)):
        tk.fiber_norms123(A, (1100, 3, 1, 2))
    dims = (40, 30, 20)
    A = flat_dev(synth.lowrank_noise(dims, (2, 2, 2), seed=3))
    small = torch.empty(tk.fiber_norms123_workspace_size(dims) - 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.TuckerError) as e:
        tk.fiber_norms123(A, dims, workspace=small)
    assert e.value.status == 1
