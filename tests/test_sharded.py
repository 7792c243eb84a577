"""The slab-sharded ST-HOSVD driver (paper_2303_11612_gb300.sharded) on CPU
ranks (gloo, world sizes 2 and 4), against the single-rank oracle.

Each rank holds its slab of the last mode; the local steps are the oracle's
FP64 steps (a test-only provider), so what is tested is the sharded logic
itself: one all-reduce of the I_n x L power-step product per step, the global
maximum of the fiber weights, each rank's CDF range and fiber offset, the
assembly of the sampled indices and of C', slab-local truncations and the
all-gather before the last mode. Against the same driver on one rank the
factors and the relative error agree to the FP64 summation order (1e-10);
against the oracle, which evaluates (A A^T)^q Omega directly rather than in
factored form, within the FP32 bars (projectors 1e-4, RE 1e-8 here); the
sampled fiber indices are the oracle's, bit for bit."""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import philox  # noqa: E402
from oracle import tucker as ot  # noqa: E402


class OracleSteps:
    """Local steps on the CPU in FP64, following the oracle (test only)."""

    @staticmethod
    def _t(A, dims):
        return synth.from_flat(A.numpy(), dims)

    def gaussian(self, I, L, seed, mode, dtype, device):
        return torch.from_numpy(philox.gaussian_matrix(seed, mode, I, L))

    def power(self, A, dims, n, X):
        M = ot.unfold(self._t(A, dims), n)
        return torch.from_numpy(M @ (M.T @ X.numpy()))

    def cholqr(self, X):
        Q, R = np.linalg.qr(X.numpy())
        s = np.sign(np.diag(R))
        s[s == 0] = 1.0
        return torch.from_numpy(Q * s), torch.from_numpy(s[:, None] * R)

    def factor(self, X, R, factors):
        C = X.numpy()
        for F in reversed(factors):
            C = C @ F.numpy()
        return torch.from_numpy(ot.leading_left_singular_vectors(C, R)[0])

    def fiber_norms(self, A, dims, n):
        return torch.from_numpy(ot.fiber_weights(ot.unfold(self._t(A, dims), n), ot.PROB_NEARLY_OPTIMAL))

    def quantize_max(self, w, wmax):
        return torch.from_numpy(ot.quantize_weights(w.numpy(), wmax=wmax).astype(np.int64))

    def sample_slab(self, W, T, seed, n, S_offset, S_total, fiber_offset):
        i, s = ot.randsample_slab(W.numpy().astype(np.uint64), T, seed, n, S_offset, S_total, fiber_offset)
        return torch.from_numpy(i), torch.from_numpy(s)

    def gather(self, A, dims, n, idx, scale):
        return torch.from_numpy(ot.amm_matrix(ot.unfold(self._t(A, dims), n), idx.numpy(), scale.numpy()))

    def sample_factor(self, Cp, R, P, q, seed, n):
        I = Cp.shape[0]
        C = ot.sketch_paper(Cp.numpy(), min(R + P, I), q, seed, n)
        return torch.from_numpy(ot.leading_left_singular_vectors(C, R)[0])

    def ttm(self, A, dims, n, U):
        return torch.from_numpy(synth.flat(ot.ttm(self._t(A, dims), U.numpy().T, n)))


CASES = {
    "q1": dict(dims=(30, 24, 20), ranks=(5, 4, 3), q=1, c=0, prob="uniform"),
    "q2": dict(dims=(30, 24, 20), ranks=(5, 4, 3), q=2, c=0, prob="uniform"),
    "amm_nearly_optimal": dict(dims=(30, 24, 20), ranks=(5, 4, 3), q=1, c=300, prob="nearly_optimal"),
    "amm_uniform_q2": dict(dims=(30, 24, 20), ranks=(5, 4, 3), q=2, c=300, prob="uniform"),
    "order4": dict(dims=(10, 9, 8, 11), ranks=(3, 3, 2, 4), q=1, c=100, prob="nearly_optimal"),
}


def tensor(dims, ranks):
    # core of exactly the target ranks: a gap at R_n, so the subspaces are well determined
    return synth.lowrank_noise(dims, ranks, rel_noise=0.05, seed=4, dtype=np.float64)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out_dir, name):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2303_11612_gb300.sharded import rsthosvd_sharded, slab_bounds
    case = CASES[name]
    A = tensor(case["dims"], case["ranks"])
    a, b = slab_bounds(case["dims"][-1], world, rank)
    slab = torch.from_numpy(synth.flat(A[..., a:b]))
    samples = []
    Us, G = rsthosvd_sharded(slab, case["dims"], case["ranks"], P=3, q=case["q"], c=case["c"], prob=case["prob"],
                             seed=11, steps=OracleSteps(), samples=samples)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"U": [u.numpy().tolist() for u in Us], "G": G.numpy().tolist(),
                   "idx": [None if s is None else s.numpy().tolist() for s in samples]}, f)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("name", list(CASES))
def test_sharded_equals_single_rank(tmp_path, world, name):
    case = CASES[name]
    mp.start_processes(worker, args=(world, free_port(), str(tmp_path), name), nprocs=world, start_method="spawn")
    outs = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    A = tensor(case["dims"], case["ranks"])
    info = {}
    Uo, Go = ot.rsthosvd(A, case["ranks"], P=3, q=case["q"], c=case["c"], prob=case["prob"], seed=11, info=info)
    reo = ot.relative_error(A, Uo, Go)
    for o in outs:
        assert o["U"] == outs[0]["U"] and o["G"] == outs[0]["G"]          # identical on every rank
    U = [np.array(u) for u in outs[0]["U"]]
    G = synth.from_flat(np.array(outs[0]["G"]), case["ranks"])
    # the same driver on one rank: only the summation order of the power steps differs
    from paper_2303_11612_gb300.sharded import rsthosvd_sharded
    U1, G1 = rsthosvd_sharded(torch.from_numpy(synth.flat(A)), case["dims"], case["ranks"], P=3, q=case["q"],
                              c=case["c"], prob=case["prob"], seed=11, steps=OracleSteps())
    for u, u1 in zip(U, U1):
        assert np.linalg.norm(u @ u.T - u1.numpy() @ u1.numpy().T, 2) < 1e-10
    assert abs(ot.relative_error(A, U, G) - ot.relative_error(A, [u.numpy() for u in U1],
                                                               synth.from_flat(G1.numpy(), case["ranks"]))) < 1e-12
    # the oracle's direct (A A^T)^q Omega against the factored form: the FP32 bars
    for u, uo in zip(U, Uo):
        assert np.linalg.norm(u @ u.T - uo @ uo.T, 2) < 1e-4
    assert abs(ot.relative_error(A, U, G) - reo) < 1e-8
    if case["c"]:
        for n, s in enumerate(outs[0]["idx"]):
            assert s is not None and np.array_equal(np.array(s), info["idx"][n]), n
