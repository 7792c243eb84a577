"""tucker_power_step_noalloc: the power step for callers that cannot allocate
device memory while they run. It must give the same result as
tucker_power_step (within the power-step tolerance of the other tests, 2e-5
relative in the Frobenius norm; only the number of partial sums may differ)
on consecutive calls that share its fixed scratch block, and reject a
problem whose partial sums do not fit in that block.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _colmajor(M):
    return torch.from_numpy(np.ascontiguousarray(M.T)).cuda().t()


def test_noalloc_power_step_matches_allocating_entry_point():
    import paper_2303_11612_gb300 as tk
    from paper_2303_11612_gb300 import _binding as B
    tk.lib()
    cases = [((130, 70, 90), 13), ((600, 20, 18), 24)]
    for rep in range(2):                                   # two calls in a row per case
        for dims, L in cases:
            A = torch.from_numpy(np.ascontiguousarray(synth.flat(
                synth.lowrank_noise(dims, (4, 4, 4), rel_noise=0.3, seed=1)))).cuda()
            for n in range(3):
                X = _colmajor(np.random.default_rng(10 * rep + n).standard_normal((dims[n], L)).astype(np.float32))
                want = B.power_step(A, dims, n, X)
                got = B.power_step_noalloc(A, dims, n, X)
                torch.cuda.synchronize()
                assert _rel(got, want) < 2e-5, (rep, dims, n)


def test_noalloc_power_step_caps_partials_to_the_block_fp64_and_side_stream():
    """Cases that reach the entry point's own paths: an FP32 problem whose
    1024 x 1024 partial is 4 MiB, so only two partials fit in the 8 MiB block
    (the number of partials is capped); FP64 data (I_n <= 512); and a call on
    a non-default stream. Each twice in a row against tucker_power_step."""
    from paper_2303_11612_gb300 import _binding as B
    B.lib()
    side = torch.cuda.Stream()
    cases = [((1024, 24, 20), 0, 1024, torch.float32, None),
             ((96, 300, 40), 1, 40, torch.float64, None),
             ((256, 60, 70), 0, 48, torch.float32, side)]
    for rep in range(2):
        for dims, mode, L, dt, stream in cases:
            A = torch.from_numpy(np.ascontiguousarray(synth.flat(
                synth.lowrank_noise(dims, (4, 4, 4), rel_noise=0.3, seed=2 + rep)))).to("cuda", dt)
            X = _colmajor(np.random.default_rng(7 + rep).standard_normal((dims[mode], L))).to(dt)
            torch.cuda.synchronize()
            want = B.power_step(A, dims, mode, X)
            with torch.cuda.stream(side if stream is not None else torch.cuda.current_stream()):
                got = B.power_step_noalloc(A, dims, mode, X, stream=stream)
            torch.cuda.synchronize()
            tol = 2e-5 if dt == torch.float32 else 1e-12
            assert _rel(got, want) < tol, (rep, dims, mode, L, dt)


def test_noalloc_power_step_rejects_tensor_core_forms():
    """Only the exact FMA arithmetic is served: a tensor-core form is refused
    (before any launch) instead of silently computed in FP32."""
    from paper_2303_11612_gb300 import _binding as B
    lib = B.lib()
    dims = (64, 8, 8)
    A = torch.zeros(64 * 64, dtype=torch.float32, device="cuda")
    X = torch.zeros((8, 64), dtype=torch.float32, device="cuda").t()
    out = torch.zeros((8, 64), dtype=torch.float32, device="cuda").t()
    for prec in ("tf32", "bf16", "bf16x1"):
        o = B.make_opts(prec=prec)
        st = lib.tucker_power_step_noalloc(A.data_ptr(), 0, B._i64(dims), 3, 0, X.data_ptr(), 8, out.data_ptr(),
                                           C.byref(o))
        assert st == 6, prec      # TUCKER_ERR_UNSUPPORTED


def test_noalloc_power_step_rejects_oversized_partials():
    from paper_2303_11612_gb300 import _binding as B
    lib = B.lib()
    dims = (1024, 2, 1)
    L = 4096                                   # one 1024 x 4096 FP32 partial = 16 MiB > 8 MiB
    A = torch.zeros(2048, dtype=torch.float32, device="cuda")
    X = torch.zeros((L, 1024), dtype=torch.float32, device="cuda").t()
    out = torch.zeros((L, 1024), dtype=torch.float32, device="cuda").t()
    o = B.make_opts()
    st = lib.tucker_power_step_noalloc(A.data_ptr(), 0, B._i64(dims), 3, 0, X.data_ptr(), L, out.data_ptr(),
                                       C.byref(o))
    assert st == 6      # TUCKER_ERR_UNSUPPORTED, before any launch
