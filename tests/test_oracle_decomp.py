"""Pins of the oracle's decompositions (Algorithms 1, 2, 4, 5) against exact
recovery, closed forms, the paper's bounds and library special cases."""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import tucker as ot

ALGS = [("T", 0, ot.PROB_UNIFORM), ("ST", 0, ot.PROB_UNIFORM),
        ("T", 150, ot.PROB_NEARLY_OPTIMAL), ("ST", 150, ot.PROB_NEARLY_OPTIMAL),
        ("ST", 150, ot.PROB_UNIFORM)]


def _run(kind, A, ranks, P=5, q=1, c=0, prob=ot.PROB_UNIFORM, seed=0, form=ot.FORM_PAPER, info=None):
    f = ot.rthosvd if kind == "T" else ot.rsthosvd
    return f(A, ranks, P=P, q=q, c=c, prob=prob, seed=seed, form=form, info=info)


def _proj_dist(U, V):
    return np.linalg.norm(U @ U.T - V @ V.T, 2)


@pytest.mark.parametrize("kind,c,prob", ALGS)
@pytest.mark.parametrize("form", [ot.FORM_PAPER, ot.FORM_RANGE])
def test_exact_multilinear_rank_is_recovered(kind, c, prob, form):
    A = synth.lowrank_noise((20, 18, 16), (4, 3, 5), rel_noise=0.0, seed=1, dtype=np.float64)
    Us, G = _run(kind, A, (4, 3, 5), c=c, prob=prob, form=form)
    # the sketch squares the spectrum, so rounding enters as eps * cond^2
    assert ot.relative_error(A, Us, G) < 1e-9
    for U, R in zip(Us, (4, 3, 5)):
        assert U.shape[1] == R
        assert np.allclose(U.T @ U, np.eye(R), atol=1e-12)
    assert G.shape == (4, 3, 5)


def test_sign_rule():
    A = synth.lowrank_noise((15, 14, 13), (3, 3, 3), rel_noise=1e-2, seed=2, dtype=np.float64)
    Us, _ = ot.rsthosvd(A, (3, 3, 3), P=4, q=1)
    for U in Us:
        for r in range(U.shape[1]):
            k = np.argmax(np.abs(U[:, r]))
            assert U[k, r] > 0


def test_tendiag_closed_form():
    """Section 6.3 tensor: superdiagonal v times orthogonal factors. Every unfolding
    has singular values |v_i|, so deterministic T-HOSVD's error is the tail of v."""
    v = 0.9 ** np.arange(24)
    A = synth.tendiag(v, (24, 24, 24), seed=3)
    for mu in (4, 9, 15):
        Us, G = ot.thosvd(A, (mu,) * 3)
        want = np.sqrt(np.sum(v[mu:] ** 2) / np.sum(v ** 2))
        assert abs(ot.relative_error(A, Us, G) - want) < 1e-12
        Us, G = ot.sthosvd(A, (mu,) * 3)
        assert abs(ot.relative_error(A, Us, G) - want) < 1e-12
        # randomized: never below the optimum, falling toward it as q grows
        res = [ot.relative_error(A, *ot.rsthosvd(A, (mu,) * 3, P=5, q=q)) for q in (1, 2, 4, 8)]
        assert all(r >= want - 1e-12 for r in res)
        assert all(res[i + 1] < res[i] for i in range(3))
        assert res[-1] - want < 5e-3
    # with a gap of 10 at mu = 8 the power scheme reaches the optimum
    v = np.concatenate([np.ones(8), 0.1 * 0.9 ** np.arange(16)])
    A = synth.tendiag(v, (24, 24, 24), seed=4)
    want = np.sqrt(np.sum(v[8:] ** 2) / np.sum(v ** 2))
    for alg in (ot.rthosvd, ot.rsthosvd):
        Us, G = alg(A, (8,) * 3, P=5, q=3)
        assert abs(ot.relative_error(A, Us, G) - want) < 1e-8


def test_tendiag_with_the_papers_spectrum_shape():
    """Section 6.3's v, scaled from 600 to 48 entries: a flat block of ones
    (50 there, 8 here) followed by (i - 49)^-2 (here (i - 7)^-2). For mu at or
    beyond the flat block the leading directions are unique, and deterministic
    T- and ST-HOSVD reach the closed-form error of the tail of v, which no
    multilinear rank-(mu, mu, mu) approximation beats; the randomized
    algorithms with two power steps stay within 1.5 times it (the gap at
    mu = 20 is only v_20 / v_21 = 1.16)."""
    k, n = 8, 48
    i = np.arange(1, n + 1)
    v = np.where(i <= k, 1.0, np.maximum(i - (k - 1), 1).astype(float) ** -2.0)
    A = synth.tendiag(v, (n, n, n), seed=5)
    for mu in (k, 12, 20):
        want = np.sqrt(np.sum(v[mu:] ** 2) / np.sum(v ** 2))
        for alg in (ot.thosvd, ot.sthosvd):
            Us, G = alg(A, (mu,) * 3)
            assert abs(ot.relative_error(A, Us, G) - want) < 1e-12, (alg.__name__, mu)
        for alg in (ot.rthosvd, ot.rsthosvd):
            re = ot.relative_error(A, *alg(A, (mu,) * 3, P=5, q=2))
            assert want - 1e-12 <= re <= 1.5 * want, (alg.__name__, mu, re, want)


def test_matrix_case_is_eckart_young():
    """N = 2: T-HOSVD is the truncated SVD; compare with eigenvalues of A A^T from
    a symmetric eigensolver (a different routine from the oracle's SVD)."""
    rng = np.random.default_rng(4)
    A = rng.standard_normal((30, 8)) @ rng.standard_normal((8, 25)) + 1e-3 * rng.standard_normal((30, 25))
    lam = np.sort(scipy.linalg.eigh(A @ A.T, eigvals_only=True))[::-1]
    for R in (3, 8):
        Us, G = ot.thosvd(A, (R, R))
        want = np.sqrt(max(np.sum(lam[R:]), 0.0) / np.sum(lam))
        assert abs(ot.relative_error(A, Us, G) - want) < 1e-9
        # column space of U_1: the leading eigenvectors of A A^T
        _, V = scipy.linalg.eigh(A @ A.T)
        V = V[:, ::-1][:, :R]
        assert _proj_dist(Us[0], V) < 1e-8


def test_thosvd_bound_eq5():
    """Eq. 5: ||A - A_hat||^2 <= sum_n ||A - A x_n U_n U_n^T||^2, and for the
    deterministic factors the right side is the tail energy of every unfolding."""
    A = synth.lowrank_noise((16, 15, 14), (4, 4, 4), rel_noise=0.2, seed=5, dtype=np.float64)
    ranks = (3, 4, 5)
    nA2 = ot.frobenius(A) ** 2
    for Us, G in (ot.thosvd(A, ranks), ot.rthosvd(A, ranks, P=3, q=1)):
        lhs = ot.relative_error(A, Us, G) ** 2 * nA2
        rhs = sum(ot.frobenius(A - ot.ttm(A, U @ U.T, n)) ** 2 for n, U in enumerate(Us))
        assert lhs <= rhs * (1 + 1e-12)
    Us, G = ot.thosvd(A, ranks)
    assert ot.relative_error(A, Us, G) ** 2 * nA2 <= ot.tail_energy_bound(A, ranks) * (1 + 1e-12)


def test_sthosvd_bound_eq23_and_lemma8():
    """Eq. 23: the ST error is bounded by the sum of the per-step truncation errors
    of the partially truncated tensors; Lemma 8: truncation never increases the
    singular values of a later unfolding."""
    A = synth.lowrank_noise((16, 15, 14), (4, 4, 4), rel_noise=0.2, seed=6, dtype=np.float64)
    ranks = (3, 4, 5)
    for Us, G in (ot.sthosvd(A, ranks), ot.rsthosvd(A, ranks, P=3, q=1)):
        lhs = ot.relative_error(A, Us, G) ** 2 * ot.frobenius(A) ** 2
        rhs, B = 0.0, A
        for n, U in enumerate(Us):
            rhs += ot.frobenius(ot.ttm(B, np.eye(U.shape[0]) - U @ U.T, n)) ** 2
            sB = np.linalg.svd(ot.unfold(B, n), compute_uv=False)
            sA = np.linalg.svd(ot.unfold(A, n), compute_uv=False)
            k = min(len(sA), len(sB))
            assert np.all(sB[:k] <= sA[:k] * (1 + 1e-12) + 1e-12)
            B = ot.ttm(B, U.T, n)
        assert lhs <= rhs * (1 + 1e-10)
    Us, G = ot.sthosvd(A, ranks)
    assert (ot.relative_error(A, Us, G) ** 2 * ot.frobenius(A) ** 2
            <= ot.tail_energy_bound(A, ranks) * (1 + 1e-12))


@pytest.mark.parametrize("kind,c,prob", ALGS)
def test_randomized_close_to_deterministic_on_noisy_lowrank(kind, c, prob):
    """Section 3.3 / 6.2: the randomized algorithms reach RE comparable to
    deterministic T/ST-HOSVD on low-rank-plus-noise tensors."""
    A = synth.lowrank_noise((24, 22, 20), (5, 5, 5), rel_noise=1e-2, seed=7, dtype=np.float64)
    det = ot.relative_error(A, *ot.sthosvd(A, (5, 5, 5)))
    Us, G = _run(kind, A, (5, 5, 5), P=5, q=1, c=c, prob=prob)
    assert ot.relative_error(A, Us, G) <= 1.5 * det + 1e-6


@pytest.mark.parametrize("form", [ot.FORM_PAPER, ot.FORM_RANGE])
def test_power_scheme_converges_to_deterministic_subspace(form):
    """More power steps sharpen the sketch: the distance between the randomized
    and the deterministic leading subspace falls as q grows (gapped spectrum),
    for the paper's (A A^T)^q Omega and for the range form's subspace
    iteration alike."""
    A = synth.lowrank_noise((40, 30, 20), (6, 6, 6), rel_noise=0.3, seed=8, dtype=np.float64)
    Ud, _ = ot.thosvd(A, (6, 6, 6))
    d = []
    for q in (1, 2, 3, 4):
        Us, _ = ot.rthosvd(A, (6, 6, 6), P=2, q=q, seed=1, form=form)
        d.append(_proj_dist(Us[0], Ud[0]))
    assert all(d[i + 1] < d[i] for i in range(3))
    assert d[-1] < 1e-3


def test_paper_sketch_equals_gram_power():
    """Strategy A (C' = M^T X; X = M C') and Strategy B (Gram first) give the same C."""
    M = np.random.default_rng(9).standard_normal((12, 50))
    from oracle import philox
    for q in (1, 2, 3):
        C = ot.sketch_paper(M, 5, q, seed=3, mode=1)
        Om = philox.gaussian_matrix(3, 1, 12, 5)
        assert np.allclose(C, np.linalg.matrix_power(M @ M.T, q) @ Om, rtol=1e-10)


def test_st_core_is_last_truncated_tensor_and_t_core_is_projection():
    A = synth.lowrank_noise((12, 11, 10), (3, 3, 3), rel_noise=0.1, seed=10, dtype=np.float64)
    Us, G = ot.rthosvd(A, (3, 3, 3), P=2, q=1)
    want = A
    for n, U in enumerate(Us):
        want = ot.ttm(want, U.T, n)
    assert np.allclose(G, want)
    # RE identity for orthogonal projections: RE^2 = 1 - ||G||^2 / ||A||^2
    re = ot.relative_error(A, Us, G)
    assert abs(re ** 2 - (1 - ot.frobenius(G) ** 2 / ot.frobenius(A) ** 2)) < 1e-12


def test_sample_counts_and_argument_checks():
    assert ot.sample_count(4000, 0.0, 400) == 400
    assert ot.sample_count(10, 0.0, 400) == 10
    assert ot.sample_count(0, 0.2, 401) == 81
    assert ot.sample_count(0, 0.0, 401) == 0
    A = np.zeros((4, 5, 6))
    with pytest.raises(ValueError):
        ot.rsthosvd(A, (5, 2, 2))
    with pytest.raises(ValueError):
        ot.rsthosvd(A, (2, 2, 2), q=0)


def test_amm_indices_drawn_only_from_nonzero_fibers():
    A = synth.lowrank_noise((10, 12, 14), (3, 3, 3), rel_noise=0.0, seed=11, dtype=np.float64)
    A[:, 3, :] = 0.0                          # a slab of zero mode-1 fibers
    info = {}
    ot.rsthosvd(A, (3, 3, 3), P=2, q=1, c=60, prob=ot.PROB_NEARLY_OPTIMAL, info=info)
    idx = info["idx"][0]
    cols = ot.unfold(A, 0)[:, idx]
    assert np.all(np.linalg.norm(cols, axis=0) > 0)


# ---------------------------------------------------------------- related forms (Algorithms 6 and 7)
def _mode_residual(M, U):
    return float(np.linalg.norm(M - U @ (U.T @ M)))


@pytest.mark.parametrize("kind", ["T", "ST"])
def test_related_form_is_optimal_within_the_sketch_span(kind):
    """Algorithms 6/7 take, inside span(C_n) = span(P_n), the R_n-dimensional
    subspace that best approximates the (current) unfolding: the left singular
    vectors of P_n^T A_(n). So per mode its projection error is never larger
    than the paper form's factor (which lies in the same span) nor than random
    R_n-dimensional subspaces of span(P_n)."""
    A = synth.lowrank_noise((24, 20, 18), (6, 5, 4), rel_noise=0.3, seed=8, dtype=np.float64)
    ranks = (4, 3, 3)
    rng = np.random.default_rng(1)
    B = A.copy()
    for n in range(3):
        M = ot.unfold(B, n)
        info_r, info_p = {}, {}
        Ur = ot._factor(M, ranks[n], 4, 1, 0, ot.PROB_UNIFORM, 3, n, ot.FORM_RELATED, info_r)
        Up = ot._factor(M, ranks[n], 4, 1, 0, ot.PROB_UNIFORM, 3, n, ot.FORM_PAPER, info_p)
        assert np.allclose(Ur.T @ Ur, np.eye(ranks[n]), atol=1e-12)
        e_r = _mode_residual(M, Ur)
        assert e_r <= _mode_residual(M, Up) + 1e-12
        Pn, _ = np.linalg.qr(ot.sketch_paper(M, info_r["L"][n], 1, 3, n))
        assert np.linalg.norm(Ur - Pn @ (Pn.T @ Ur)) < 1e-12           # inside span(P_n)
        for _ in range(20):
            V = Pn @ np.linalg.qr(rng.standard_normal((Pn.shape[1], ranks[n])))[0]
            assert e_r <= _mode_residual(M, V) + 1e-12
        if kind == "ST":
            B = ot.ttm(B, Up.T, n)


def test_related_form_without_oversampling_spans_the_sketch():
    """With K = 0 the sketch has R_n columns: both forms return a basis of
    span(C_n), hence the same projector."""
    A = synth.lowrank_noise((20, 18, 16), (5, 4, 4), rel_noise=0.2, seed=3, dtype=np.float64)
    Ur, _ = ot.rsthosvd(A, (4, 3, 3), P=0, q=1, seed=2, form=ot.FORM_RELATED)
    Up, _ = ot.rsthosvd(A, (4, 3, 3), P=0, q=1, seed=2, form=ot.FORM_PAPER)
    for a, b in zip(Ur, Up):
        assert _proj_dist(a, b) < 1e-10


def test_related_form_recovers_exact_rank_and_rejects_amm():
    A = synth.lowrank_noise((20, 18, 16), (4, 3, 5), rel_noise=0.0, seed=1, dtype=np.float64)
    for kind in ("T", "ST"):
        Us, G = _run(kind, A, (4, 3, 5), form=ot.FORM_RELATED)
        assert ot.relative_error(A, Us, G) < 1e-9
        for U in Us:
            k = np.argmax(np.abs(U), axis=0)
            assert np.all(U[k, np.arange(U.shape[1])] > 0)      # the sign rule holds on Q_n
    with pytest.raises(ValueError):
        _run("ST", A, (4, 3, 5), c=50, form=ot.FORM_RELATED)


# ---------------------------------------------------------------- fixed precision (Problem 2)
def test_adaptive_ranks_meet_the_tolerance_and_recover_exact_ranks():
    """Problem 2: the returned decomposition meets ||A - Ahat|| <= eps ||A||; on a
    tensor of exact multilinear rank the ranks found are that rank."""
    A = synth.lowrank_noise((24, 20, 18), (4, 3, 5), rel_noise=0.0, seed=5, dtype=np.float64)
    Qs, G, ranks = ot.rsthosvd_adaptive(A, 1e-9, q=1, seed=1, L0=4)
    assert ranks == [4, 3, 5]
    assert ot.relative_error(A, Qs, G) <= 1e-9
    B = synth.lowrank_noise((24, 20, 18), (6, 5, 4), rel_noise=0.05, seed=6, dtype=np.float64)
    for eps in (0.2, 0.1, 0.06):
        Qs, G, ranks = ot.rsthosvd_adaptive(B, eps, q=2, seed=2, L0=2)
        assert ot.relative_error(B, Qs, G) <= eps * (1 + 1e-12), (eps, ranks)
        for Q in Qs:
            assert np.allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-12)


def test_adaptive_ranks_on_tendiag_follow_the_closed_form():
    """tendiag: every unfolding has singular values |v_i| exactly (Section 6.3),
    and after truncating modes 1..n-1 to r_1..r_{n-1} the next unfolding keeps
    v_1..v_min(r). So the ranks are the closed-form minimal r meeting each
    mode's budget: with budget_n = (eps^2 sum v^2 - spent) / (N - n + 1), r_n =
    the least r with sum_{r < i <= m} v_i^2 <= budget_n over the m values left."""
    v = 0.6 ** np.arange(12)
    A = synth.tendiag(v, (20, 18, 16), seed=3)
    eps = 0.05
    _, _, ranks = ot.rsthosvd_adaptive(A, eps, q=3, seed=4, L0=2)
    total = float(np.sum(v ** 2))
    spent, m, want = 0.0, len(v), []
    for n in range(3):
        budget = (eps ** 2 * total - spent) / (3 - n)
        tail = [float(np.sum(v[r:m] ** 2)) for r in range(m + 1)]
        r = next(r for r in range(1, m + 1) if tail[r] <= budget)
        want.append(r)
        spent += tail[r]
        m = r
    assert ranks == want
