"""Autotuner: tuning happens in synchronous calls only, keeps one choice per
shape class, leaves the mode-n product bitwise unchanged (its candidates
compute every output in the same order), and tuned decompositions stay within
the oracle bars. The choices persist for the process, so this file runs after
the other GPU tests (only the allocation-free test, which does not depend on
them, sorts later)."""
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
    yield tk
    tk.autotune_enable(False)


def dev(A):
    return torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()


def test_mode_product_bitwise_unchanged_by_tuning(tk):
    dims = (96, 72, 40)
    A = dev(synth.lowrank_noise(dims, (4, 4, 4), rel_noise=0.3, seed=41))
    U = torch.randn(12, 72, device="cuda").t()
    tk.autotune_enable(False)
    plain = tk.ttm(A, dims, 1, U, transpose=True)
    n0 = len(tk.autotune_entries())
    tk.autotune_enable(True)
    tuned = tk.ttm(A, dims, 1, U, transpose=True)          # tunes this class
    again = tk.ttm(A, dims, 1, U, transpose=True)          # uses the kept choice
    entries = tk.autotune_entries()
    assert len(entries) == n0 + 1 and entries[-1].startswith("mode-n product")
    assert torch.equal(plain, tuned) and torch.equal(plain, again)


def test_asynchronous_calls_do_not_tune(tk):
    tk.autotune_enable(True)
    dims, ranks = (88, 52, 36), (5, 4, 3)
    A = dev(synth.lowrank_noise(dims, ranks, rel_noise=1e-2, seed=42))
    n0 = len(tk.autotune_entries())
    ws = torch.empty(tk.workspace_size("ST", dims, ranks, P=5, q=1), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    tk.rsthosvd(A, dims, ranks, P=5, q=1, seed=1, stream=s, workspace=ws, flags=tk.FLAG_ASYNC)
    s.synchronize()
    assert tk.last_device_status() == 0
    assert len(tk.autotune_entries()) == n0


@pytest.mark.parametrize("which", ["ST", "T"])
def test_tuned_decompositions_match_oracle(tk, which):
    tk.autotune_enable(True)
    dims, ranks = (120, 96, 80), (6, 5, 4)
    A = synth.lowrank_noise(dims, ranks, rel_noise=1e-2, seed=43)
    A64 = A.astype(np.float64)
    fn = ot.rthosvd if which == "T" else ot.rsthosvd
    Uo, Go = fn(A64, ranks, P=5, q=2, seed=3)
    reo = ot.relative_error(A64, Uo, Go)
    for _ in range(2):                                     # tunes on the first pass, reuses on the second
        U, G = tk.decompose(which, dev(A), dims, ranks, P=5, q=2, seed=3)
        U = [u.double().cpu().numpy() for u in U]
        G = synth.from_flat(G.double().cpu().numpy(), ranks)
        assert abs(ot.relative_error(A64, U, G) - reo) <= 1e-5
        for u, uo in zip(U, Uo):
            assert np.linalg.norm(u @ u.T - uo @ uo.T, 2) <= 1e-4
    assert any(e.startswith("FP32 power step") for e in tk.autotune_entries())
