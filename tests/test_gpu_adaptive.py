"""Fixed-precision ranks (Problem 2) on the GPU: tucker_rsthosvd_adaptive
against the oracle's rsthosvd_adaptive on the same tensors.

- The ranks equal the oracle's wherever its decision has a margin (every case
  here keeps |budget - remainder| above 2.8e-5 ||B||^2 at the chosen rank and
  the one before, far above the FP32 energies' rounding).
- The relative error meets the tolerance and agrees with the oracle's (FP64
  data to 1e-10, FP32 to 1e-6); factors are orthonormal.
- tendiag follows the closed form of its ranks; exact multilinear ranks are
  recovered; eps = 0 keeps every direction.
- Invalid requests give TUCKER_ERR_INVALID_ARG."""
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


def dev(A, dtype):
    return torch.from_numpy(np.ascontiguousarray(synth.flat(A.astype(dtype)))).cuda()


def check(tk, A, eps, q, seed, L0, dtype, re_tol, **kw):
    A64 = A.astype(np.float64) if dtype == np.float64 else A.astype(np.float32).astype(np.float64)
    Qo, Go, ro = ot.rsthosvd_adaptive(A64, eps, q=q, seed=seed, L0=L0)
    U, G, r, re_dev = tk.rsthosvd_adaptive(dev(A, dtype), A.shape, eps, q=q, L0=L0, seed=seed,
                                           want_rel_error=True, **kw)
    assert r == ro, (r, ro)
    Ud = [u.double().cpu().numpy() for u in U]
    Gd = synth.from_flat(G.double().cpu().numpy(), r)
    re, reo = ot.relative_error(A64, Ud, Gd), ot.relative_error(A64, Qo, Go)
    assert re <= eps * (1 + 1e-6) + re_tol, (re, eps)
    assert abs(re - reo) <= re_tol, (re, reo)
    # the call's own RE comes from ||G||^2 / ||A||^2, as accurate as the core's norm
    assert abs(re_dev ** 2 - re ** 2) <= (1e-6 if dtype == np.float32 else 1e-12), (re_dev, re)
    for u in Ud:
        tol = 1e-5 if dtype == np.float32 else 1e-12
        assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) < tol
    return r


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("eps", [0.2, 0.1, 0.06])
def test_noisy_tensor_matches_the_oracle(tk, dtype, eps):
    B = synth.lowrank_noise((24, 20, 18), (6, 5, 4), rel_noise=0.05, seed=6, dtype=np.float64)
    check(tk, B, eps, 2, 2, 2, dtype, 1e-10 if dtype == np.float64 else 1e-6)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_tendiag_closed_form(tk, dtype):
    v = 0.6 ** np.arange(12)
    A = synth.tendiag(v, (20, 18, 16), seed=3)
    eps = 0.05
    # at q = 3 the sketch grades its directions as v_i^6 (0.6^66 across the 12), so
    # FP32 resolves the weak ones only to its rounding: RE within 1e-4 of the
    # oracle's (measured 6e-5), the ranks exactly
    r = check(tk, A, eps, 3, 4, 2, dtype, 1e-10 if dtype == np.float64 else 1e-4)
    total = float(np.sum(v ** 2))
    spent, m, want = 0.0, len(v), []
    for n in range(3):
        budget = (eps ** 2 * total - spent) / (3 - n)
        tail = [float(np.sum(v[k:m] ** 2)) for k in range(m + 1)]
        k = next(k for k in range(1, m + 1) if tail[k] <= budget)
        want.append(k)
        spent += tail[k]
        m = k
    assert r == want


def test_exact_ranks_recovered(tk):
    A = synth.lowrank_noise((24, 20, 18), (4, 3, 5), rel_noise=0.0, seed=5, dtype=np.float64)
    assert check(tk, A, 1e-9, 1, 1, 4, np.float64, 1e-10) == [4, 3, 5]
    assert check(tk, A, 1e-2, 1, 1, 4, np.float32, 1e-6) == [4, 3, 5]


@pytest.mark.parametrize("kw", [dict(), dict(prec="bf16"), dict(prec="bf16x1"), dict(form="range")],
                         ids=["fp32", "bf16", "bf16x1", "range"])
def test_larger_tensor_in_every_form(tk, kw):
    """200 x 150 x 120 of multilinear rank (10, 8, 6) plus 1e-3 noise, eps = 1e-2:
    the widening reaches L = 16 in mode 1; ranks (10, 8, 6) in every form."""
    A = synth.lowrank_noise((200, 150, 120), (10, 8, 6), rel_noise=1e-3, seed=7, dtype=np.float64)
    U, G, r = tk.rsthosvd_adaptive(dev(A, np.float32), A.shape, 1e-2, q=1, L0=8, seed=0, **kw)
    assert r == [10, 8, 6]
    if not kw:
        check(tk, A, 1e-2, 1, 0, 8, np.float32, 1e-6)
    else:
        Ud = [u.double().cpu().numpy() for u in U]
        re = ot.relative_error(A, Ud, synth.from_flat(G.double().cpu().numpy(), r))
        assert re <= 1e-2


def test_zero_tolerance_keeps_every_direction(tk):
    A = np.random.default_rng(3).standard_normal((6, 5, 4))
    U, G, r = tk.rsthosvd_adaptive(dev(A, np.float64), A.shape, 0.0, q=1, L0=2, seed=1)
    assert r == [6, 5, 4]
    Ud = [u.cpu().numpy() for u in U]
    assert ot.relative_error(A, Ud, synth.from_flat(G.cpu().numpy(), r)) < 1e-12


def test_invalid_requests(tk):
    from paper_2303_11612_gb300 import _binding as B
    A = torch.zeros(6 * 5 * 4, dtype=torch.float32, device="cuda")
    with pytest.raises(B.TuckerError):
        tk.rsthosvd_adaptive(A, (6, 5, 4), -1.0)
    with pytest.raises(B.TuckerError):
        tk.rsthosvd_adaptive(A, (6, 5, 4), 0.1, q=0)
    with pytest.raises(B.TuckerError):
        tk.rsthosvd_adaptive(A, (6, 5, 4), 0.1, L0=0)
    with pytest.raises(B.TuckerError):
        tk.rsthosvd_adaptive(A.cpu(), (6, 5, 4), 0.1)
