"""Pins of the oracle's AMM sampler (RANDSAMPLE / BasicMatrixMultiplication, Section 3.2)."""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import synth
from oracle import philox
from oracle import tucker as ot


def test_quantize_weights_hand_values():
    w = np.array([0.0, 1.0, 0.5, 1e-9, 0.25 + 2.0 ** -30])
    W = ot.quantize_weights(w)
    assert W.tolist() == [0, 1 << 24, 1 << 23, 1, (1 << 22) + 1]
    assert ot.quantize_weights(np.zeros(5)).tolist() == [1] * 5


def _bucket_table(W):
    """Brute force: the index owning each integer v in [0, S)."""
    table = []
    for j, wj in enumerate(W.tolist()):
        table += [j] * int(wj)
    return table


@pytest.mark.parametrize("kind", ["mixed", "spiky", "ones"])
def test_inverse_cdf_against_expanded_table(kind):
    W = synth.sample_weights(40, seed=3, kind=kind) % np.uint64(50)   # keep S small
    if int(W.sum()) == 0:
        W[0] = 1
    table = _bucket_table(W)
    S = len(table)
    T = 300
    idx, scale = ot.randsample(W, T, seed=5, mode=1)
    words = philox.sampling_words(5, 1, T)
    for t in range(T):
        v = (words[t] * S) >> 64
        assert idx[t] == table[v]
        p = int(W[idx[t]]) / S
        assert scale[t] == 1.0 / math.sqrt(T * p)
        assert W[idx[t]] > 0       # zero-weight fibers are never drawn


def test_sampled_frequencies_follow_p():
    W = np.array([1, 2, 3, 4, 0, 10], dtype=np.uint64)
    T = 20000
    idx, _ = ot.randsample(W, T, seed=11, mode=0)
    counts = np.bincount(idx, minlength=len(W))
    p = W.astype(float) / W.sum()
    mask = p > 0
    chi = stats.chisquare(counts[mask], T * p[mask])
    assert chi.pvalue > 1e-4
    assert counts[4] == 0


@pytest.mark.parametrize("prob", [ot.PROB_NEARLY_OPTIMAL, ot.PROB_UNIFORM])
@pytest.mark.parametrize("T", [2, 3])
def test_amm_unbiased_by_enumeration(prob, T):
    """E[C' C'^T] = M M^T exactly: enumerate every index tuple with its probability."""
    M = np.random.default_rng(2).standard_normal((3, 4))
    M[:, 2] *= 0.01                          # uneven fiber norms
    W = ot.quantize_weights(ot.fiber_weights(M, prob))
    S = int(W.sum())
    p = W.astype(np.float64) / S
    acc = np.zeros((3, 3))
    for tup in itertools.product(range(4), repeat=T):
        pr = np.prod([p[j] for j in tup])
        if pr == 0:
            continue
        scale = np.array([1.0 / math.sqrt(T * p[j]) for j in tup])
        C = ot.amm_matrix(M, np.array(tup), scale)
        acc += pr * (C @ C.T)
    assert np.allclose(acc, M @ M.T, rtol=1e-13, atol=1e-13)


def test_amm_error_shrinks_like_inverse_sqrt_T():
    """Corollary 1 / Lemmas 5-6: E||M M^T - C'C'^T||_F decays like 1/sqrt(T)."""
    rng = np.random.default_rng(0)
    M = rng.standard_normal((20, 400)) * (1 + 5 * rng.random(400))
    ref = M @ M.T
    Ts = [25, 100, 400]
    errs = []
    for T in Ts:
        W = ot.quantize_weights(ot.fiber_weights(M, ot.PROB_NEARLY_OPTIMAL))
        e = []
        for seed in range(120):
            idx, scale = ot.randsample(W, T, seed=seed, mode=0)
            C = ot.amm_matrix(M, idx, scale)
            e.append(np.linalg.norm(ref - C @ C.T))
        errs.append(np.mean(e))
    slope = np.polyfit(np.log(Ts), np.log(errs), 1)[0]
    assert -0.6 < slope < -0.4


def test_nearly_optimal_beats_uniform_on_skewed_fibers():
    rng = np.random.default_rng(1)
    M = rng.standard_normal((10, 500))
    M[:, :10] *= 50.0                        # a few heavy fibers
    ref = M @ M.T
    out = {}
    for prob in (ot.PROB_NEARLY_OPTIMAL, ot.PROB_UNIFORM):
        W = ot.quantize_weights(ot.fiber_weights(M, prob))
        e = []
        for seed in range(40):
            idx, scale = ot.randsample(W, 100, seed=seed, mode=0)
            C = ot.amm_matrix(M, idx, scale)
            e.append(np.linalg.norm(ref - C @ C.T))
        out[prob] = np.mean(e)
    assert out[ot.PROB_NEARLY_OPTIMAL] < out[ot.PROB_UNIFORM]


def test_fiber_weights_hand_values():
    """Nearly-optimal weights are the squared fiber norms (remark after
    Algorithm 3 with B = A^T): columns (3, 4), (0, 0), (1, 1) of a 2 x 3
    unfolding have squared norms 25, 0 and 2; uniform weights are all one."""
    M = np.array([[3.0, 0.0, 1.0],
                  [4.0, 0.0, 1.0]])
    assert ot.fiber_weights(M, ot.PROB_NEARLY_OPTIMAL).tolist() == [25.0, 0.0, 2.0]
    assert ot.fiber_weights(M, ot.PROB_UNIFORM).tolist() == [1.0, 1.0, 1.0]
    # quantised: the largest weight maps to 2^24, 2/25 of it rounds up
    W = ot.quantize_weights(ot.fiber_weights(M, ot.PROB_NEARLY_OPTIMAL))
    assert W.tolist() == [1 << 24, 0, math.ceil(2 / 25 * (1 << 24))]


def _expected_amm_error(M, p):
    """E ||M M^T - C' C'^T||_F^2 for one sample (T = 1) with probabilities p,
    by enumerating the J outcomes; with T samples the error is this over T."""
    ref = M @ M.T
    e = 0.0
    for j in range(M.shape[1]):
        if p[j] == 0:
            continue
        c = M[:, j:j + 1] / math.sqrt(p[j])
        e += p[j] * float(np.sum((ref - c @ c.T) ** 2))
    return e


def test_nearly_optimal_weights_minimise_the_enumerated_amm_error():
    """The probabilities the oracle derives for the nearly-optimal scheme are
    the minimiser of the AMM estimator's expected squared error (Lemma 5 and
    the remark after Algorithm 3 with B = A^T: p_j proportional to the squared
    fiber norm). Enumerated, not from a closed form: every random perturbation
    of p, and the unsquared-norm probabilities, give a larger error."""
    rng = np.random.default_rng(4)
    M = rng.standard_normal((3, 6)) * np.array([0.2, 1.0, 3.0, 0.5, 1.5, 0.05])[None, :]
    W = ot.quantize_weights(ot.fiber_weights(M, ot.PROB_NEARLY_OPTIMAL))
    p = W.astype(np.float64) / float(W.sum())
    best = _expected_amm_error(M, p)
    for k in range(40):
        d = rng.standard_normal(p.shape)
        q = p * np.exp(0.05 * d)
        q /= q.sum()
        assert _expected_amm_error(M, q) > best
    norms = np.linalg.norm(M, axis=0)
    assert _expected_amm_error(M, norms / norms.sum()) > best * 1.01
    u = np.full(p.shape, 1.0 / p.size)
    assert _expected_amm_error(M, u) > best * 1.01


@pytest.mark.parametrize("parts", [1, 2, 3, 5])
def test_slab_draws_partition_the_global_draws(parts):
    """RANDSAMPLE resolved part by part over a partition of the fibers (each
    part quantised against the global largest weight, its CDF range offset by
    the earlier parts' totals) gives, over the parts, exactly the single-call
    indices and scales: the sharded sampler's definition."""
    w = np.abs(np.random.default_rng(7).standard_normal(50)) ** 3
    w[[3, 17]] = 0.0
    T = 400
    W = ot.quantize_weights(w)
    idx, scale = ot.randsample(W, T, seed=9, mode=2)
    bounds = np.linspace(0, w.size, parts + 1).astype(int)
    Ws = [ot.quantize_weights(w[a:b], wmax=float(np.max(w))) for a, b in zip(bounds[:-1], bounds[1:])]
    assert np.array_equal(np.concatenate(Ws), W)
    totals = [int(x.sum()) for x in Ws]
    got_i = np.full(T, -1, dtype=np.int64)
    got_s = np.zeros(T)
    for k, (a, b) in enumerate(zip(bounds[:-1], bounds[1:])):
        i, s = ot.randsample_slab(Ws[k], T, 9, 2, sum(totals[:k]), sum(totals), a)
        mine = i >= 0
        assert not np.any(got_i[mine] >= 0)                 # every draw resolved by one part only
        got_i[mine], got_s[mine] = i[mine], s[mine]
    assert np.array_equal(got_i, idx)
    assert np.array_equal(got_s, scale)
