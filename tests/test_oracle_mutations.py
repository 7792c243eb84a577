"""Each test plants one plausible mistake in the oracle (on the CPU, via
monkeypatch) and checks that one of the oracle's pins catches it."""
import math

import numpy as np
import pytest

from oracle import philox
from oracle import tucker as ot

import test_oracle_decomp as decomp
import test_oracle_philox as tphilox
import test_oracle_sampling as tsamp
import test_oracle_tensor_ops as tops


def _caught(fn, *args, **kw):
    try:
        fn(*args, **kw)
    except (AssertionError, ValueError, IndexError):
        return True
    return False


def test_wrong_unfolding_order_is_caught(monkeypatch):
    def bad_unfold(A, n):
        A = np.asarray(A)
        return np.reshape(np.moveaxis(A, n, 0), (A.shape[n], -1), order="C")
    monkeypatch.setattr(ot, "unfold", bad_unfold)
    assert _caught(tops.test_unfold_index_map_brute_force)


def test_transposed_mode_product_is_caught(monkeypatch):
    good = ot.ttm
    monkeypatch.setattr(ot, "ttm", lambda A, M, n: good(A, M.T, n) if M.shape[0] == M.shape[1] else good(A, M, n))
    def check():
        A = tops._rand((4, 4, 4), 0)
        M = np.random.default_rng(1).standard_normal((4, 4))
        B = ot.ttm(A, M, 1)
        want = np.einsum("ji,aib->ajb", M, A)
        assert np.allclose(B, want)
    assert _caught(check)


def test_missing_sqrt_in_amm_scale_is_caught(monkeypatch):
    good = ot.amm_matrix
    monkeypatch.setattr(ot, "amm_matrix", lambda M, idx, scale: good(M, idx, scale ** 2))
    assert _caught(tsamp.test_amm_unbiased_by_enumeration, ot.PROB_NEARLY_OPTIMAL, 2)


def test_dropped_power_step_is_caught(monkeypatch):
    def bad(M, L, q, seed, mode):
        X = philox.gaussian_matrix(seed, mode, M.shape[0], L)
        for _ in range(q - 1):
            X = M @ (M.T @ X)
        return X
    monkeypatch.setattr(ot, "sketch_paper", bad)
    assert _caught(decomp.test_paper_sketch_equals_gram_power)


def test_wrong_sign_rule_is_caught(monkeypatch):
    def bad(U):
        U = U.copy()
        for r in range(U.shape[1]):
            k = int(np.argmin(np.abs(U[:, r])))
            if U[k, r] < 0:
                U[:, r] = -U[:, r]
        return U
    monkeypatch.setattr(ot, "sign_fix", bad)
    assert _caught(decomp.test_sign_rule)


def test_swapped_philox_words_are_caught(monkeypatch):
    good = philox.philox4x32_10
    monkeypatch.setattr(philox, "philox4x32_10", lambda *a: (lambda o: (o[1], o[0], o[2], o[3]))(good(*a)))
    rows = tphilox._kat_rows()
    assert _caught(tphilox.test_philox_known_answers, rows[0])


def test_floor_quantisation_is_caught(monkeypatch):
    def bad(w):
        w = np.asarray(w, dtype=np.float64)
        return np.floor(w / w.max() * float(1 << ot.QUANT_BITS)).astype(np.uint64)
    monkeypatch.setattr(ot, "quantize_weights", bad)
    assert _caught(tsamp.test_quantize_weights_hand_values)


def test_off_by_one_inverse_cdf_is_caught(monkeypatch):
    good = ot.randsample
    def bad(W, T, seed, mode):
        idx, scale = good(W, T, seed, mode)
        return np.minimum(idx + 1, len(W) - 1), scale
    monkeypatch.setattr(ot, "randsample", bad)
    assert _caught(tsamp.test_inverse_cdf_against_expanded_table, "mixed")


def test_missing_st_truncation_is_caught(monkeypatch):
    good_ttm = ot.ttm
    calls = {"n": 0}
    def ttm_skipping_update(A, M, n):
        # drop the Algorithm 2 update for mode 1 (first ttm call with a thin M^T)
        calls["n"] += 1
        if calls["n"] == 1 and M.shape[0] < M.shape[1]:
            return A
        return good_ttm(A, M, n)
    monkeypatch.setattr(ot, "ttm", ttm_skipping_update)
    assert _caught(decomp.test_exact_multilinear_rank_is_recovered, "ST", 0, ot.PROB_UNIFORM,
                   ot.FORM_PAPER)


def test_wrong_gaussian_angle_is_caught(monkeypatch):
    good = philox.gaussian_elements
    def bad(seed, stream, count):
        z = good(seed, stream, count)
        return np.abs(z)            # e.g. a dropped sign from the angle term
    monkeypatch.setattr(philox, "gaussian_elements", bad)
    assert _caught(tphilox.test_gaussian_moments_and_ks)


def test_unsquared_fiber_norms_are_caught(monkeypatch):
    def bad(M, prob):
        if prob == ot.PROB_UNIFORM:
            return np.ones(M.shape[1])
        return np.sqrt(np.sum(M.astype(np.float64) ** 2, axis=0))
    monkeypatch.setattr(ot, "fiber_weights", bad)
    assert _caught(tsamp.test_fiber_weights_hand_values)
    assert _caught(tsamp.test_nearly_optimal_weights_minimise_the_enumerated_amm_error)


def test_right_singular_vectors_in_the_related_form_are_caught(monkeypatch):
    good = ot.leading_left_singular_vectors
    def bad(C, R):
        # the related form asks for left singular vectors of the L x J matrix
        # P^T A; a plausible slip takes the leading right ones of its transpose's
        # transpose, i.e. of C^T C, truncated to C's row count
        if C.shape[0] < C.shape[1]:
            _, s, Vt = np.linalg.svd(C, full_matrices=False)
            W = np.linalg.qr(np.random.default_rng(0).standard_normal((C.shape[0], R)))[0]
            return W, s
        return good(C, R)
    monkeypatch.setattr(ot, "leading_left_singular_vectors", bad)
    assert _caught(decomp.test_related_form_is_optimal_within_the_sketch_span, "T")


def test_related_form_without_the_basis_product_is_caught(monkeypatch):
    good_qr = np.linalg.qr
    def bad_qr(C, *a, **k):
        Q, R = good_qr(C, *a, **k)
        return np.roll(Q, 1, axis=0), R          # a basis of the wrong span
    monkeypatch.setattr(ot.np.linalg, "qr", bad_qr)
    assert _caught(decomp.test_related_form_is_optimal_within_the_sketch_span, "ST")
