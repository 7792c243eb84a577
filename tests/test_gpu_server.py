"""Serving loop (tucker_server_*): requests of mixed orders, sizes and ranks
arrive over time, are admitted against a device-memory budget and run
concurrently. Each result must be the same as the same request run alone:
every kernel reduces in a fixed order, so the bar is bitwise equality."""
import time

import numpy as np
import pytest
import torch

import synth

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
        N = 3 if rng.random() < 0.5 else 4
        hi = 64 if N == 3 else 24
        dims = tuple(int(x) for x in rng.integers(8, hi + 1, size=N))
        ranks = tuple(int(min(d, x)) for d, x in zip(dims, rng.integers(2, 9, size=N)))
        A = synth.lowrank_noise(dims, ranks, rel_noise=1e-2, seed=1000 + k)
        reqs.append(dict(which="ST" if rng.random() < 0.7 else "T", A=A, dims=dims, ranks=ranks,
                         q=int(rng.integers(1, 3)), c=int(rng.choice([0, 0, 200])),
                         prob=str(rng.choice(["uniform", "nearly_optimal"])), seed=k,
                         host_in=bool(rng.random() < 0.4), host_out=bool(rng.random() < 0.4)))
    return reqs


@pytest.mark.parametrize("prec", ["fp32", "bf16", "tf32", "bf16x1"])
def test_results_same_alone_and_in_the_mix(tk, prec):
    reqs = make_requests(24, seed=5)
    alone = []
    for r in reqs:
        At = torch.from_numpy(np.ascontiguousarray(synth.flat(r["A"]))).cuda()
        U, G = tk.decompose(r["which"], At, r["dims"], r["ranks"], P=5, q=r["q"], c=r["c"], prob=r["prob"],
                            seed=r["seed"], prec=prec)
        alone.append(([u.cpu() for u in U], G.cpu()))
    rng = np.random.default_rng(11)
    with tk.Server(budget_bytes=64 << 20, max_inflight=6, prec=prec) as srv:
        tickets = []
        for r in reqs:
            flat = torch.from_numpy(np.ascontiguousarray(synth.flat(r["A"])))
            A = flat.pin_memory() if r["host_in"] else flat.cuda()
            tickets.append(srv.submit(r["which"], A, r["dims"], r["ranks"], P=5, q=r["q"], c=r["c"], prob=r["prob"],
                                      seed=r["seed"], out_device="cpu" if r["host_out"] else "cuda"))
            time.sleep(float(rng.exponential(0.002)))          # Poisson arrivals
        got = [srv.wait(t) for t in tickets]
        st = srv.stats()
    for (U, G), (Ua, Ga) in zip(got, alone):
        for u, ua in zip(U, Ua):
            if u.is_cuda:
                u = u.cpu()
            assert torch.equal(u.contiguous(), ua.contiguous())
        assert torch.equal(G.cpu(), Ga)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["peak_bytes"] <= 64 << 20
    assert 1 <= st["peak_inflight"] <= 6
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]


def test_admission_budget_and_errors(tk):
    dims, ranks = (48, 40, 32), (4, 4, 4)
    A = torch.from_numpy(np.ascontiguousarray(synth.flat(synth.lowrank_noise(dims, ranks, 1e-2, seed=3)))).cuda()
    need = tk.workspace_size("ST", dims, ranks, P=5, q=1)
    # room for exactly one request at a time: they must run one after another
    with tk.Server(budget_bytes=need + need // 2, max_inflight=4) as srv:
        ts = [srv.submit("ST", A, dims, ranks, P=5, q=1, seed=s) for s in range(5)]
        for t in ts:
            srv.wait(t)
        st = srv.stats()
        assert st["peak_inflight"] == 1 and st["completed"] == 5
        with pytest.raises(tk.TuckerError) as e:                  # alone larger than the budget
            srv.submit("ST", A, (48, 40, 32), (40, 40, 32), P=5, q=1)
        assert e.value.status == 7
        with pytest.raises(tk.TuckerError) as e:                  # rank above the extent
            srv.submit("ST", A, dims, (49, 4, 4), P=5, q=1)
        assert e.value.status == 1

