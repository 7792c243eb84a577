"""Batched launch (tucker_batch_*): a mixed batch of decompositions runs as one
CUDA graph, captured on the first run and replayed afterwards. Each request's
result must be bitwise that of the same request run alone, on the first run and
on every replay, and a replay must see inputs rewritten in place."""
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


def make_requests(n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n):
        N = 3 if rng.random() < 0.6 else 4
        hi = 80 if N == 3 else 24
        dims = tuple(int(x) for x in rng.integers(8, hi + 1, size=N))
        ranks = tuple(int(min(d, x)) for d, x in zip(dims, rng.integers(2, 9, size=N)))
        A = synth.lowrank_noise(dims, ranks, rel_noise=1e-2, seed=2000 + k)
        reqs.append(dict(which="ST" if rng.random() < 0.6 else "T", A0=A, dims=dims, ranks=ranks, P=5,
                         q=int(rng.integers(1, 3)), c=int(rng.choice([0, 0, 150])),
                         prob=str(rng.choice(["uniform", "nearly_optimal"])), seed=k))
    return reqs


def dev(A):
    return torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()


def alone(tk, r, A, prec):
    U, G = tk.decompose(r["which"], A, r["dims"], r["ranks"], P=r["P"], q=r["q"], c=r["c"], prob=r["prob"],
                        seed=r["seed"], prec=prec)
    return [u.contiguous().cpu() for u in U], G.cpu()


def same(got, want):
    U, G = got
    Ua, Ga = want
    return all(torch.equal(u.contiguous().cpu(), ua) for u, ua in zip(U, Ua)) and torch.equal(G.cpu(), Ga)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "tf32", "bf16x1"])
def test_batch_equals_requests_alone_and_replays(tk, prec):
    reqs = make_requests(12, seed=8)
    for r in reqs:
        r["A"] = dev(r["A0"])
    want = [alone(tk, r, r["A"], prec) for r in reqs]
    b = tk.Batch(reqs, prec=prec)
    n0 = tk.launch_count()
    out = b.run()                                        # capture + first launch
    n1 = tk.launch_count()
    for got, w in zip(out, want):
        assert same(got, w)
    s = torch.cuda.Stream()
    for _ in range(2):                                   # replays, synchronous and asynchronous
        for U, G in out:
            G.zero_()
            for u in U:
                u.zero_()
        torch.cuda.synchronize()
        out = b.run(stream=s, sync=False)
        s.synchronize()
        for got, w in zip(out, want):
            assert same(got, w)
    # every kernel of the graph is counted once per launch
    assert tk.launch_count() - n1 == 2 * (n1 - n0) > 0
    # the status word of each request's workspace slice is clear, at the offsets
    # the library's workspace sizes give
    sizes = [tk.workspace_size(r["which"], r["dims"], r["ranks"], P=r["P"], q=r["q"], c=r["c"], prec=prec)
             for r in reqs]
    offs = np.concatenate([[0], np.cumsum([(sz + 255) // 256 * 256 for sz in sizes])])
    assert b.workspace.numel() >= offs[-1] and b._offsets == [int(o) for o in offs[:-1]]
    assert b.status() == [0] * len(reqs)


def test_replay_reads_inputs_rewritten_in_place(tk):
    reqs = make_requests(6, seed=9)
    for r in reqs:
        r["A"] = dev(r["A0"])
    b = tk.Batch(reqs)
    b.run()
    # new contents in the same buffers: the cached graph must decompose them
    news = [synth.lowrank_noise(r["dims"], r["ranks"], rel_noise=3e-2, seed=3000 + k) for k, r in enumerate(reqs)]
    for r, A in zip(reqs, news):
        r["A"].copy_(dev(A))
    out = b.run()
    for r, A, got in zip(reqs, news, out):
        assert same(got, alone(tk, r, dev(A), "fp32"))
        # and against the oracle, within the same bars as single calls
        fn = ot.rthosvd if r["which"] == "T" else ot.rsthosvd
        A64 = A.astype(np.float64)
        if r["c"] == 0:
            Uo, Go = fn(A64, r["ranks"], P=r["P"], q=r["q"], seed=r["seed"])
            U = [u.double().cpu().numpy() for u in got[0]]
            G = synth.from_flat(got[1].double().cpu().numpy(), r["ranks"])
            assert abs(ot.relative_error(A64, U, G) - ot.relative_error(A64, Uo, Go)) <= 1e-5


def test_batch_argument_errors(tk):
    dims, ranks = (16, 12, 10), (3, 3, 3)
    A = dev(synth.lowrank_noise(dims, ranks, rel_noise=1e-2, seed=4))
    with pytest.raises(tk.TuckerError):
        tk.Batch([dict(which="ST", A=A, dims=dims, ranks=(3, 30, 3))])       # R_n > I_n
    b = tk.Batch([dict(which="ST", A=A, dims=dims, ranks=ranks)])
    b.workspace = b.workspace[:128]                                           # too small
    with pytest.raises(tk.TuckerError):
        b.run()
    b2 = tk.Batch([dict(which="ST", A=A.cpu(), dims=dims, ranks=ranks)])     # host input and outputs
    b2.workspace = torch.empty(b2.workspace.numel(), dtype=torch.uint8, device="cuda")
    with pytest.raises(tk.TuckerError):
        b2.run()
