"""Work-list batches (tucker_batch_run with TUCKER_FLAG_WORKLIST): every stage of
every request becomes items of one persistent kernel launch per step, and the
orthonormalisations of all requests run as grouped launches.

- Each request's factors and core are bitwise those of the same request run
  alone through the driver (the items run the stages' own block programs, the
  grouped launches the extraction's), in FP32 and FP64, for ST- and T-HOSVD,
  q = 1 and 2, orders 3 and 4, ragged extents up to 256 and ranks up to 32; on
  the first run and on graph replays, synchronous and asynchronous; and a replay
  sees inputs rewritten in place.
- A request's results do not depend on the batch around it (alone in a batch of
  one, and in a mix of 16).
- Against the oracle: RE within 1e-5 (FP32) / 1e-10 (FP64) of the oracle's, and
  projectors within 1e-4 where the sketch has a gap at R_n.
- The batch takes a few launches per step whatever the number of requests.
- A dependency wait that runs out (a two-item list whose second item waits for
  an item never listed, through tucker_check_wait_timeout) returns the timeout
  status, the context stays usable and a work-list batch after it is exact."""
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


def make_requests(n, seed, dtype=np.float32, hi3=200, hi4=40):
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n):
        N = 3 if rng.random() < 0.7 else 4
        hi = hi3 if N == 3 else hi4
        dims = tuple(int(x) for x in rng.integers(16, hi + 1, size=N))
        ranks = tuple(int(min(d, x)) for d, x in zip(dims, rng.integers(2, 33, size=N)))
        A = synth.lowrank_noise(dims, ranks, rel_noise=1e-2, seed=4000 + k + seed, dtype=dtype)
        reqs.append(dict(which="ST" if rng.random() < 0.6 else "T", A0=A, dims=dims, ranks=ranks,
                         P=int(rng.integers(0, 9)), q=int(rng.integers(1, 3)), seed=k))
    return reqs


def dev(A):
    return torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()


def alone(tk, r, A):
    U, G = tk.decompose(r["which"], A, r["dims"], r["ranks"], P=r["P"], q=r["q"], seed=r["seed"])
    return [u.contiguous().cpu() for u in U], G.cpu()


def same(got, want):
    U, G = got
    Ua, Ga = want
    return all(torch.equal(u.contiguous().cpu(), ua) for u, ua in zip(U, Ua)) and torch.equal(G.cpu(), Ga)


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
def test_worklist_equals_requests_alone_and_replays(tk, dtype):
    reqs = make_requests(10, seed=3, dtype=dtype)
    for r in reqs:
        r["A"] = dev(r["A0"])
    want = [alone(tk, r, r["A"]) for r in reqs]
    b = tk.Batch(reqs, worklist=True)
    out = b.run()
    for k, (got, w) in enumerate(zip(out, want)):
        assert same(got, w), k
    assert b.status() == [0] * len(reqs)
    s = torch.cuda.Stream()
    for _ in range(2):
        for U, G in out:
            G.zero_()
            for u in U:
                u.zero_()
        torch.cuda.synchronize()
        out = b.run(stream=s, sync=False)
        s.synchronize()
        for got, w in zip(out, want):
            assert same(got, w)
    # inputs rewritten in place: the replay decomposes the new tensors
    for r in reqs:
        r["A"].mul_(-0.5)
    want2 = [alone(tk, r, r["A"]) for r in reqs]
    out = b.run()
    for got, w in zip(out, want2):
        assert same(got, w)


def test_worklist_equals_stream_batch_and_is_independent_of_the_mix(tk):
    reqs = make_requests(16, seed=11)
    for r in reqs:
        r["A"] = dev(r["A0"])
    mixed = tk.Batch(reqs, worklist=True).run()
    streams = tk.Batch(reqs).run()
    for got, w in zip(mixed, streams):
        assert same(got, ([u.contiguous().cpu() for u in w[0]], w[1].cpu()))
    for k in (0, 7, 15):
        single = tk.Batch([reqs[k]], worklist=True).run()[0]
        assert same(single, ([u.contiguous().cpu() for u in mixed[k][0]], mixed[k][1].cpu()))


@pytest.mark.parametrize("dtype,re_tol", [(np.float32, 1e-5), (np.float64, 1e-10)], ids=["f32", "f64"])
def test_worklist_matches_the_oracle(tk, dtype, re_tol):
    specs = [("ST", (96, 80, 64), (8, 6, 5), 2), ("T", (64, 56, 48), (6, 5, 4), 1),
             ("ST", (40, 36, 32, 28), (4, 4, 3, 3), 1), ("T", (256, 33, 17), (32, 8, 6), 2)]
    reqs = []
    for k, (which, dims, ranks, q) in enumerate(specs):
        A = synth.lowrank_noise(dims, ranks, rel_noise=1e-2, seed=70 + k, dtype=dtype)
        reqs.append(dict(which=which, A0=A, A=dev(A), dims=dims, ranks=ranks, P=6, q=q, seed=k + 1))
    out = tk.Batch(reqs, worklist=True).run()
    for r, (U, G) in zip(reqs, out):
        A64 = r["A0"].astype(np.float64)
        fn = ot.rsthosvd if r["which"] == "ST" else ot.rthosvd
        info = {}
        Uo, Go = fn(A64, r["ranks"], P=r["P"], q=r["q"], seed=r["seed"], info=info)
        Ud = [u.double().cpu().numpy() for u in U]
        re = ot.relative_error(A64, Ud, synth.from_flat(G.double().cpu().numpy(), r["ranks"]))
        reo = ot.relative_error(A64, Uo, Go)
        assert abs(re - reo) <= re_tol, (r["which"], r["dims"], re, reo)
        for n, (u, uo) in enumerate(zip(Ud, Uo)):
            s = info["sigma_C"][n]
            if s[r["ranks"][n] - 1] >= 1.5 * s[r["ranks"][n]]:
                assert np.linalg.norm(u @ u.T - uo @ uo.T, 2) <= 1e-4, (r["dims"], n)


def test_worklist_launches_per_step_not_per_request(tk):
    counts = []
    for n in (16, 48):
        reqs = make_requests(n, seed=5, hi3=64, hi4=24)
        for r in reqs:
            r["which"], r["q"], r["dims"] = "ST", 1, (40, 36, 32, 20)
            r["ranks"] = (4, 4, 3, 2)
            r["A"] = dev(synth.lowrank_noise(r["dims"], r["ranks"], rel_noise=1e-2, seed=r["seed"]))
        wl = tk.Batch(reqs, worklist=True)
        n0 = tk.launch_count()
        wl.run()
        counts.append(tk.launch_count() - n0)
    st = tk.Batch(reqs)
    n0 = tk.launch_count()
    st.run()
    n_st = tk.launch_count() - n0
    # 4 lanes of 4 modes: per lane 4 power steps + 1 core step and 4 grouped extractions of
    # 8 launches (with their CholeskyQR passes), whatever the number of requests
    assert counts == [4 * 37, 4 * 37], counts
    assert n_st >= 5 * counts[1], (n_st, counts)


def test_worklist_wait_times_out_and_the_context_survives(tk):
    from paper_2303_11612_gb300 import _binding as B
    assert B.check_wait_timeout(1000, worklist=True) == 5          # TUCKER_ERR_TIMEOUT
    assert B.check_wait_timeout(1, worklist=True) == 5
    reqs = make_requests(3, seed=21)
    for r in reqs:
        r["A"] = dev(r["A0"])
    out = tk.Batch(reqs, worklist=True).run()
    for r, got in zip(reqs, out):
        assert same(got, alone(tk, r, r["A"]))
