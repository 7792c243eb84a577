"""Parity at the full sizes of the benchmarked and listed workloads, in the
launch configuration the benchmark uses (caller workspace, asynchronous calls
on side streams, several decompositions in flight).

- 400^3 FP32 (the benchmark's tensors), randomized ST-HOSVD R = 20, P = 10:
  FP32 form |RE - RE_oracle| <= 1e-5 and projectors <= 1e-4 on the low-rank
  tensor (gap at R), split-BF16 within 1e-4 and single-pass BF16 within 1e-3;
  on the Hilbert tensor per-form bars against the oracle (see the test), and
  the FP64 data path never worse than the oracle by more than 1e-5;
  orthonormal factors throughout; sampled fiber indices of mode 1 equal to the
  oracle's.
- 96^4 FP32 with a geometrically decaying core, ST-HOSVD R = 16, P = 8, q = 2.
- 1024 x 1024 x 512 FP32 video-like tensor (2.1 GB), ST-HOSVD R = (64, 64, 32),
  P = 16, q = 1, with and without AMM (c = 20000): against the FP64 oracle run
  on the same bytes, in all four arithmetic forms.
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


def dev(A):
    return torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()


def in_flight(tk, jobs, prec):
    """Runs every job asynchronously on its own stream with its own workspace,
    all in flight together, as the benchmark does."""
    main = torch.cuda.current_stream()
    outs = []
    streams = [torch.cuda.Stream() for _ in jobs]
    for st in streams:
        st.wait_stream(main)
    for (A, dims, ranks, kw), st in zip(jobs, streams):
        ws = torch.empty(tk.workspace_size("ST", dims, ranks, prec=prec, **{k: kw[k] for k in ("P", "q", "c")}),
                         dtype=torch.uint8, device="cuda")
        c = kw.get("c", 0)
        res = tk.rsthosvd(A, dims, ranks, stream=st, workspace=ws, flags=tk.FLAG_ASYNC, prec=prec,
                          want_samples=bool(c), **kw)
        outs.append((res, ws))
    for st in streams:
        main.wait_stream(st)
    torch.cuda.synchronize()
    assert tk.last_device_status() == 0
    return [r for r, _ in outs]


@pytest.fixture(scope="module")
def bench_tensors():
    dims, ranks = (400, 400, 400), (20, 20, 20)
    low = synth.lowrank_noise(dims, ranks, rel_noise=1e-2, seed=0)
    hil = synth.hilbert(dims)
    return dims, ranks, low, hil


@pytest.mark.parametrize("prec", ["fp32", "bf16", "tf32", "bf16x1"])
def test_benchmark_workload_400cubed(tk, bench_tensors, prec):
    dims, ranks, low, hil = bench_tensors
    variants = [
        (low, dict(P=10, q=1, c=0, prob="uniform", seed=0)),
        (low, dict(P=10, q=1, c=4000, prob="nearly_optimal", seed=0)),
        (hil, dict(P=10, q=2, c=0, prob="uniform", seed=0)),
        (hil, dict(P=10, q=1, c=4000, prob="uniform", seed=0)),
    ]
    jobs = [(dev(A), dims, ranks, kw) for A, kw in variants]
    got = in_flight(tk, jobs, prec)
    for (A, kw), res in zip(variants, got):
        U = [u.double().cpu().numpy() for u in res[0]]
        G = synth.from_flat(res[1].double().cpu().numpy(), ranks)
        info = {}
        A64 = A.astype(np.float64)
        Uo, Go = ot.rsthosvd(A64, ranks, info=info, **kw)
        re, reo = ot.relative_error(A64, U, G), ot.relative_error(A64, Uo, Go)
        for u in U:
            assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) < 10 * u.shape[1] * 1.19e-7
        if A is low:
            if prec == "fp32":
                # gap at R = 20 (core 20^3, noise 1e-2): the FP32 bars
                assert abs(re - reo) <= 1e-5, (kw, re, reo)
                for u, uo in zip(U, Uo):
                    assert np.linalg.norm(u @ u.T - uo @ uo.T, 2) <= 1e-4
            else:
                # tensor-core forms: the sketch's rounding moves RE only to second
                # order and the mode-1 product (split bf16, ~2^-16) to about 1e-6;
                # the single-pass bf16 sketch (2^-8) is held to the 1e-3 bar
                bar = 1e-3 if prec == "bf16x1" else 1e-4
                assert abs(re - reo) <= bar, (kw, re, reo)
        else:
            # Hilbert: its mode-n singular values fall by orders of magnitude per
            # index. Bars against the oracle, per form (measured in brackets):
            #   q = 2, no sampling: a full power step carries sigma_i^2, so FP32
            #   loses the directions with sigma_i / sigma_1 below ~2^-12 the FP64
            #   oracle keeps: FP32 1.2e-4 (8e-5), tensor-core forms 2e-4 (1.2-1.4e-4);
            #   q = 1 with AMM: the sample is sketched in orthonormalised half steps
            #   and the factored extraction never forms C_n, so every form resolves
            #   directions the oracle's explicit FP64 C_n loses: never worse than the
            #   oracle, within 2.5e-4 of it (1.7e-4 better)
            if kw["c"]:
                assert re <= reo + 1e-5 and abs(re - reo) <= 2.5e-4, (prec, kw, re, reo)
            else:
                assert abs(re - reo) <= (1.2e-4 if prec == "fp32" else 2e-4), (prec, kw, re, reo)
        if kw["c"]:
            # mode 1 samples the input tensor itself: identical weights, identical draws
            assert np.array_equal(res[2][0].cpu().numpy(), info["idx"][0]), kw


@pytest.mark.parametrize("kw", [dict(P=10, q=2, c=0, prob="uniform", seed=0),
                                dict(P=10, q=1, c=4000, prob="uniform", seed=0)], ids=["q2", "amm4000"])
def test_hilbert_400cubed_fp64_matches_oracle(tk, bench_tensors, kw):
    dims, ranks, _, hil = bench_tensors
    A64 = hil.astype(np.float64)
    Uo, Go = ot.rsthosvd(A64, ranks, **kw)
    U, G = tk.rsthosvd(torch.from_numpy(np.ascontiguousarray(synth.flat(A64))).cuda(), dims, ranks, **kw)
    U = [u.cpu().numpy() for u in U]
    G = synth.from_flat(G.cpu().numpy(), ranks)
    # never worse than the oracle by more than 1e-5. At q = 2 the GPU is far
    # better (RE ~5e-6 against 9.1e-5): its factored power scheme loses only
    # directions whose (sigma_i / sigma_1)^2 falls below FP64 rounding, the
    # oracle's direct (A A^T)^2 Omega those whose (sigma_i / sigma_1)^4 does
    assert ot.relative_error(A64, U, G) <= ot.relative_error(A64, Uo, Go) + 1e-5


def test_fourth_order_96(tk):
    dims, ranks = (96, 96, 96, 96), (16, 16, 16, 16)
    A = synth.decaying_core(dims, 16, ratio=0.8, seed=0)
    A64 = A.astype(np.float64)
    Uo, Go = ot.rsthosvd(A64, ranks, P=8, q=2, seed=0)
    reo = ot.relative_error(A64, Uo, Go)
    for prec, bar in (("fp32", 1e-5), ("bf16", 1e-3), ("tf32", 1e-3), ("bf16x1", 1e-3)):
        (res,) = in_flight(tk, [(dev(A), dims, ranks, dict(P=8, q=2, c=0, prob="uniform", seed=0))], prec)
        U = [u.double().cpu().numpy() for u in res[0]]
        G = synth.from_flat(res[1].double().cpu().numpy(), ranks)
        assert abs(ot.relative_error(A64, U, G) - reo) <= bar, prec


@pytest.fixture(scope="module")
def video():
    dims, ranks = (1024, 1024, 512), (64, 64, 32)
    A = synth.video_like(dims, terms=50, noise_var=1e-2, seed=0)
    return dims, ranks, A


VIDEO_VARIANTS = [dict(P=16, q=1, c=0, prob="uniform", seed=0), dict(P=16, q=1, c=20000, prob="uniform", seed=0)]


@pytest.fixture(scope="module")
def video_oracle(video):
    """The FP64 oracle on the same bytes (a few seconds per variant on the host)."""
    dims, ranks, A = video
    A64 = A.astype(np.float64)
    nA = ot.frobenius(A64)
    out = []
    for kw in VIDEO_VARIANTS:
        info = {}
        Uo, Go = ot.rsthosvd(A64, ranks, info=info, **kw)
        reo = np.sqrt(max(0.0, 1.0 - ot.frobenius(Go) ** 2 / nA ** 2))   # exact: the reconstruction is a projection
        out.append((Uo, Go, reo, info))
    return out


@pytest.mark.parametrize("prec", ["fp32", "bf16", "tf32", "bf16x1"])
def test_video_like_1024_against_the_oracle(tk, video, video_oracle, prec):
    """The 1024 x 1024 x 512 video-like workload (2.15 GB), both variants in
    flight together as the benchmark runs them: relative error within 1e-5 of
    the oracle's in the FP32 form and 1e-3 in the tensor-core forms; projectors
    within 1e-4 (FP32) / 1e-2 where the oracle's sketch has a gap at R_n
    (sigma_R / sigma_{R+1} >= 1.5); orthonormal factors; mode-1 sampled fibers
    identical to the oracle's; and the identity RE^2 = 1 - ||G||^2 / ||A||^2
    against the explicit reconstruction error computed on the device."""
    dims, ranks, A = video
    Ad = dev(A)
    jobs = [(Ad, dims, ranks, kw) for kw in VIDEO_VARIANTS]
    got = in_flight(tk, jobs, prec)
    for kw, res, (Uo, Go, reo, info) in zip(VIDEO_VARIANTS, got, video_oracle):
        re = tk.relative_error(Ad, dims, ranks, res[0], res[1])              # explicit, on the device
        U = [u.double().cpu().numpy() for u in res[0]]
        G = res[1].double().cpu().numpy()
        re_id = np.sqrt(max(0.0, 1.0 - float(np.sum(G * G)) / float(np.sum(A.astype(np.float64) ** 2))))
        assert abs(re - reo) <= (1e-5 if prec == "fp32" else 1e-3), (prec, kw["c"], re, reo)
        # the identity is as accurate as the core: a relative error d of ||G||^2
        # moves it by about d / (2 RE); the tensor-core forms' mode products are
        # split bf16 (d ~ 2^-15), the FP32 form's exact FP32
        assert abs(re_id - re) <= (1e-4 if prec == "fp32" else 2.0 ** -15 / (2 * re) + 1e-5), (re_id, re)
        for n, (u, uo) in enumerate(zip(U, Uo)):
            assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) < 10 * u.shape[1] * 1.19e-7
            s = info["sigma_C"][n]
            R = ranks[n]
            if len(s) > R and s[R - 1] >= 1.5 * s[R]:
                assert np.linalg.norm(u @ u.T - uo @ uo.T, 2) <= (1e-4 if prec == "fp32" else 1e-2), (prec, n)
        if kw["c"]:
            assert np.array_equal(res[2][0].cpu().numpy(), info["idx"][0])
