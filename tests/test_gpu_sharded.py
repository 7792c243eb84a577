"""The steps of a slab-sharded call on the GPU (tucker_quantize_weights_max,
tucker_sample_fibers_slab, tucker_cholqr, tucker_leading_factor_chain,
tucker_sample_factor) and the sharded driver with the library as its step
provider on one rank (every GPU run here has one GPU, so more ranks are
covered on CPU ranks by test_sharded.py).

- Slab draws over a partition of the fibers reproduce tucker_sample_fibers bit
  for bit; quantising against the global maximum reproduces the integer weights.
- CholeskyQR then the factored extraction reproduce the driver's factor.
- The sharded driver on one rank equals tucker_rsthosvd: same sampled indices,
  projectors within 1e-5, relative error within 1e-6 (the same kernels run)."""
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


@pytest.mark.parametrize("parts", [1, 3])
def test_slab_draws_reproduce_the_global_draws(tk, parts):
    from paper_2303_11612_gb300 import _binding as B
    w = torch.from_numpy(np.abs(np.random.default_rng(3).standard_normal(5000)) ** 3).cuda()
    w[17] = 0.0
    T = 3000
    W = B.quantize_weights(w, "nearly_optimal")
    idx, scale = B.sample_fibers(W, T, seed=5, mode=1)
    bounds = np.linspace(0, w.numel(), parts + 1).astype(int)
    wmax = float(w.max())
    Ws = [B.quantize_weights_max(w[a:b].contiguous(), wmax) for a, b in zip(bounds[:-1], bounds[1:])]
    assert torch.equal(torch.cat(Ws), W)
    totals = [int(x.sum()) for x in Ws]
    gi = torch.full((T,), -1, dtype=torch.int64, device="cuda")
    gs = torch.zeros(T, dtype=torch.float64, device="cuda")
    for k, (a, b) in enumerate(zip(bounds[:-1], bounds[1:])):
        i, s = B.sample_fibers_slab(Ws[k], T, 5, 1, sum(totals[:k]), sum(totals), int(a))
        gi = torch.maximum(gi, i)
        gs = torch.maximum(gs, s)
    assert torch.equal(gi, idx) and torch.equal(gs, scale)


def test_cholqr_and_factored_extraction(tk):
    from paper_2303_11612_gb300 import _binding as B
    dims, ranks = (200, 60, 50), (12, 10, 8)
    A = synth.lowrank_noise(dims, ranks, rel_noise=1e-2, seed=2)
    At = torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()
    U_lib, _ = tk.rsthosvd(At, dims, ranks, P=6, q=2, seed=3)
    X = B.gaussian(200, 18, 3, 0, device="cuda")
    X = B.power_step(At, dims, 0, X)
    Q, F = B.cholqr(X)
    qd = Q.double()
    # one CholeskyQR pass: orthonormal to about cond(X)^2 times the Gram's rounding
    # (the factored form stays exact whatever it is: C = X_q F)
    assert float(torch.linalg.norm(qd.t() @ qd - torch.eye(18, dtype=torch.float64, device="cuda"))) < 1e-3
    X2 = B.power_step(At, dims, 0, Q)
    U = B.leading_factor_chain(X2, 12, [F])
    u, ul = U.double().cpu().numpy(), U_lib[0].double().cpu().numpy()
    assert np.linalg.norm(u @ u.T - ul @ ul.T, 2) < 1e-5


@pytest.mark.parametrize("c,prob,q", [(0, "uniform", 1), (0, "uniform", 2), (800, "nearly_optimal", 1),
                                      (800, "uniform", 2)])
def test_sharded_driver_one_rank_equals_the_library(tk, c, prob, q):
    from paper_2303_11612_gb300.sharded import rsthosvd_sharded, LibrarySteps
    dims, ranks = (120, 50, 40), (8, 6, 5)
    A = synth.lowrank_noise(dims, ranks, rel_noise=1e-2, seed=6)
    At = torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()
    U_lib, G_lib, smp = tk.rsthosvd(At, dims, ranks, P=5, q=q, c=c, prob=prob, seed=9, want_samples=True)
    samples = []
    U, G = rsthosvd_sharded(At, dims, ranks, P=5, q=q, c=c, prob=prob, seed=9, steps=LibrarySteps(),
                            samples=samples)
    A64 = A.astype(np.float64)
    re = ot.relative_error(A64, [u.double().cpu().numpy() for u in U], synth.from_flat(G.double().cpu().numpy(), ranks))
    re_lib = ot.relative_error(A64, [u.double().cpu().numpy() for u in U_lib],
                               synth.from_flat(G_lib.double().cpu().numpy(), ranks))
    assert abs(re - re_lib) < 1e-6
    for u, ul in zip(U, U_lib):
        ud, uld = u.double().cpu().numpy(), ul.double().cpu().numpy()
        assert np.linalg.norm(ud @ ud.T - uld @ uld.T, 2) < 1e-5
    if c:
        for s, sl in zip(samples, smp):
            assert torch.equal(s, sl)
