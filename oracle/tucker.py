"""FP64 CPU oracle for randomized T-HOSVD / ST-HOSVD with the power scheme and
approximate matrix multiplication (Che, Wei, Yan, arXiv 2303.11612).

TEST INFRASTRUCTURE: only tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline leg may import this package. It shares no code with the CUDA
library; the two meet only in the seeded input tensors (``synth``) and in the
specification of the Philox stream (``oracle.philox`` implements it on the CPU).

Everything is plain numpy in float64, written to be checked against the paper
by eye. Library routines used as single steps: matrix products, QR (range
form only) and the SVD (factor extraction, the remark after Algorithm 5).

Notation (paper -> here): mu_n -> R_n (target rank), K -> P (oversampling),
T_n -> T (AMM sample count), G_n (Gaussian) -> Omega, Q_n -> U_n, core -> G.
Tensors are numpy arrays of shape (I_1, ..., I_N), i_1 fastest (Fortran order).

Readings where the paper is silent or ambiguous:
  * L_n = min(R_n + P, I_n) columns in the sketch.
  * T_n = min(c, J_n) when c > 0; T_n = ceil(alpha J_n) when c == 0 and alpha > 0
    (the parameter rule of Section 3.3); no AMM otherwise.
  * Nearly-optimal probabilities for A_(n) A_(n)^T are p_j proportional to the
    squared norm of fiber j (the optimal probabilities of the remark after
    Algorithm 3 with B = A^T); uniform p_j = 1 / J_n.
  * Probabilities are quantised to integer weights
    W_j = ceil(w_j / max_k w_k * 2^24) for w_j > 0 (0 otherwise); the sampled
    index solves CDF_{j-1} <= v < CDF_j for v = floor(r * S / 2^64), r a 64-bit
    Philox word and S = sum W. The rescaling 1/sqrt(T p_j) uses the quantised
    p_j = W_j / S, so E[C' C'^T] = A_(n) A_(n)^T holds exactly. A tensor whose
    fibers are all zero is sampled uniformly.
  * Extraction: U_n = the R_n leading left singular vectors of C_n (the remark
    after Algorithm 5), each column's largest-magnitude entry made positive
    (first such entry on ties).
  * "Related form" (Algorithms 6 and 7, the related forms of Algorithms 1 and 2):
    the sketch C_n as in the paper form, its thin QR C_n = P_n R, the R_n leading
    left singular vectors U of P_n^T A_(n), and Q_n = P_n U (sign rule applied to
    Q_n). Defined without AMM only.
  * "Range form" (optional, from the comparison in the introduction, item (c)):
    Y = A_(n) Omega with Omega J_n x L_n, then q times Y = A_(n) (A_(n)^T orth(Y));
    U_n = leading left singular vectors of Y.
"""
from __future__ import annotations

import math

import numpy as np

from . import philox

FORM_PAPER = "paper"
FORM_RANGE = "range"
FORM_RELATED = "related"
PROB_NEARLY_OPTIMAL = "nearly_optimal"
PROB_UNIFORM = "uniform"
QUANT_BITS = 24


# ---------------------------------------------------------------- Section 2 basics
def unfold(A: np.ndarray, n: int) -> np.ndarray:
    """Mode-n unfolding A_(n) (I_n x J_n). Column index follows Section 2:
    j = i_1 + (i_2-1) I_1 + ... with i_n skipped, i.e. the remaining indices in
    increasing mode order, the lowest fastest."""
    A = np.asarray(A)
    return np.reshape(np.moveaxis(A, n, 0), (A.shape[n], -1), order="F")


def fold(M: np.ndarray, n: int, dims) -> np.ndarray:
    """Inverse of ``unfold`` for a tensor of shape ``dims`` (dims[n] = rows of M)."""
    dims = tuple(int(d) for d in dims)
    rest = dims[:n] + dims[n + 1:]
    T = np.reshape(M, (dims[n],) + rest, order="F")
    return np.moveaxis(T, 0, n)


def ttm(A: np.ndarray, M: np.ndarray, n: int) -> np.ndarray:
    """Mode-n product A x_n M (Section 2): (A x_n M)_(n) = M A_(n), M is J x I_n."""
    dims = list(A.shape)
    out = M @ unfold(A, n)
    dims[n] = M.shape[0]
    return fold(out, n, dims)


def frobenius(A: np.ndarray) -> float:
    return float(np.sqrt(np.sum(np.asarray(A, dtype=np.float64) ** 2)))


# ---------------------------------------------------------------- AMM (Section 3.2)
def fiber_weights(M: np.ndarray, prob: str) -> np.ndarray:
    """w_j for the columns (mode-n fibers) of M: squared norms, or ones (uniform)."""
    if prob == PROB_UNIFORM:
        return np.ones(M.shape[1])
    return np.sum(M.astype(np.float64) ** 2, axis=0)


def quantize_weights(w: np.ndarray, wmax: float = None) -> np.ndarray:
    """Integer weights W_j = ceil(w_j / max(w) * 2^24) (0 for w_j = 0); all ones
    when every w_j is zero. With `wmax` given, that value replaces max(w): the
    largest weight over every part of a partitioned set of fibers."""
    w = np.asarray(w, dtype=np.float64)
    if wmax is None:
        wmax = float(np.max(w)) if w.size else 0.0
    if wmax <= 0.0:
        return np.ones(w.shape, dtype=np.uint64)
    W = np.ceil((w / wmax) * float(1 << QUANT_BITS))
    W[w <= 0.0] = 0.0
    return W.astype(np.uint64)


def randsample(W: np.ndarray, T: int, seed: int, mode: int):
    """RANDSAMPLE(T, p) of Section 3.2 with p_j = W_j / S: T indices drawn with
    replacement and the nonzero entries 1/sqrt(T p_xi) of the sampling matrix."""
    W = np.asarray(W, dtype=np.uint64)
    cdf = [0] * len(W)
    acc = 0
    for j, wj in enumerate(W.tolist()):
        acc += int(wj)
        cdf[j] = acc
    S = acc
    words = philox.sampling_words(seed, mode, T)
    idx = np.empty(T, dtype=np.int64)
    scale = np.empty(T, dtype=np.float64)
    for t, r in enumerate(words):
        v = (r * S) >> 64                       # floor(r * S / 2^64), exact integers
        # smallest j with CDF_j > v
        lo, hi = 0, len(cdf) - 1
        while lo < hi:
            mid = (lo + hi) // 2
            if cdf[mid] > v:
                hi = mid
            else:
                lo = mid + 1
        idx[t] = lo
        p = float(int(W[lo])) / float(S)
        scale[t] = 1.0 / math.sqrt(float(T) * p)
    return idx, scale


def randsample_slab(W: np.ndarray, T: int, seed: int, mode: int, S_offset: int, S_total: int,
                    fiber_offset: int):
    """RANDSAMPLE (Section 3.2) resolved by one part of a partition of the
    fibers: this part holds global fibers fiber_offset .. fiber_offset + len(W) - 1
    whose weights W cover [S_offset, S_offset + sum W) of the total S_total.
    Draw t lands here when S_offset <= v_t < S_offset + sum W, v_t as in
    randsample; it then gets its global index and 1/sqrt(T p); other draws get
    index -1 and scale 0 (another part resolves them)."""
    W = np.asarray(W, dtype=np.uint64)
    cdf, acc = [], 0
    for wj in W.tolist():
        acc += int(wj)
        cdf.append(acc)
    words = philox.sampling_words(seed, mode, T)
    idx = np.full(T, -1, dtype=np.int64)
    scale = np.zeros(T, dtype=np.float64)
    for t, r in enumerate(words):
        v = (r * S_total) >> 64
        if not (S_offset <= v < S_offset + acc):
            continue
        u = v - S_offset
        lo, hi = 0, len(cdf) - 1
        while lo < hi:
            mid = (lo + hi) // 2
            if cdf[mid] > u:
                hi = mid
            else:
                lo = mid + 1
        idx[t] = lo + fiber_offset
        p = float(int(W[lo])) / float(S_total)
        scale[t] = 1.0 / math.sqrt(float(T) * p)
    return idx, scale


def sample_count(c: int, alpha: float, J: int) -> int:
    if c > 0:
        return int(min(c, J))
    if alpha > 0:
        return int(min(math.ceil(alpha * J), J))
    return 0


def amm_matrix(M: np.ndarray, idx: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """C' = M S (Algorithms 4/5): the sampled columns, each times its scale."""
    return M[:, idx] * scale[None, :]


# ---------------------------------------------------------------- sketches (Alg 1, Strategy A)
def sketch_paper(M: np.ndarray, L: int, q: int, seed: int, mode: int) -> np.ndarray:
    """C = (M M^T)^q Omega with Omega I x L standard Gaussian, evaluated as in
    Strategy A (C' = M^T X, X = M C', q times)."""
    X = philox.gaussian_matrix(seed, mode, M.shape[0], L)
    for _ in range(q):
        X = M @ (M.T @ X)
    return X


def sketch_range(M: np.ndarray, L: int, q: int, seed: int, mode: int) -> np.ndarray:
    """Y = M Omega with Omega J x L standard Gaussian; then q times
    Y = M (M^T Q) with Q an orthonormal basis of range(Y)."""
    Om = philox.gaussian_matrix(seed, mode, M.shape[1], L)
    Y = M @ Om
    for _ in range(q):
        Q, _ = np.linalg.qr(Y)
        Y = M @ (M.T @ Q)
    return Y


def sign_fix(U: np.ndarray) -> np.ndarray:
    """Make the largest-magnitude entry of every column positive (first on ties)."""
    U = U.copy()
    for r in range(U.shape[1]):
        k = int(np.argmax(np.abs(U[:, r])))
        if U[k, r] < 0:
            U[:, r] = -U[:, r]
    return U


def leading_left_singular_vectors(C: np.ndarray, R: int):
    """(U(:, 1:R), sigma) from the thin SVD of C (remark after Algorithm 5)."""
    Uc, s, _ = np.linalg.svd(C, full_matrices=False)
    if Uc.shape[1] < R:   # fewer sketch columns than R: pad with an orthonormal complement
        Qf, _ = np.linalg.qr(np.hstack([Uc, np.eye(C.shape[0])[:, :R]]))
        Uc = np.hstack([Uc, Qf[:, Uc.shape[1]:R]])
    return sign_fix(Uc[:, :R]), s


# ---------------------------------------------------------------- drivers (Alg 1, 2, 4, 5)
def _factor(M, R, P, q, T, prob, seed, mode, form, info):
    """One mode's factor from the current unfolding M (I_n x J_n)."""
    I, J = M.shape
    L = min(R + P, I)
    if T > 0:
        W = quantize_weights(fiber_weights(M, prob))
        idx, scale = randsample(W, T, seed, mode)
        M = amm_matrix(M, idx, scale)
        info.setdefault("idx", {})[mode] = idx
        info.setdefault("scale", {})[mode] = scale
        info.setdefault("W", {})[mode] = W
    if form == FORM_RELATED:
        if T > 0:
            raise ValueError("the related forms (Algorithms 6 and 7) are defined without AMM")
        C = sketch_paper(M, L, q, seed, mode)
        Pn, _ = np.linalg.qr(C)                          # thin QR, P_n orthonormal I x L
        Ul, s = leading_left_singular_vectors(Pn.T @ M, R)
        U = sign_fix(Pn @ Ul)
        info.setdefault("L", {})[mode] = L
        info.setdefault("T", {})[mode] = T
        info.setdefault("sigma_C", {})[mode] = s
        return U
    if form == FORM_RANGE:
        C = sketch_range(M, L, q, seed, mode)
    else:
        C = sketch_paper(M, L, q, seed, mode)
    U, s = leading_left_singular_vectors(C, R)
    info.setdefault("L", {})[mode] = L
    info.setdefault("T", {})[mode] = T
    info.setdefault("sigma_C", {})[mode] = s
    return U


def _check(A, ranks, P, q):
    if A.ndim < 1 or A.ndim != len(ranks):
        raise ValueError("ranks must give one R_n per mode")
    for I, R in zip(A.shape, ranks):
        if R < 1 or R > I:
            raise ValueError("need 1 <= R_n <= I_n")
    if q < 1 or P < 0:
        raise ValueError("need q >= 1 and P >= 0")


def rthosvd(A, ranks, P=10, q=1, c=0, prob=PROB_UNIFORM, seed=0, alpha=0.0, form=FORM_PAPER,
            info=None):
    """Algorithm 1 (c == 0 and alpha == 0) or Algorithm 4 (AMM): every factor from
    the unfolding of the input tensor, then G = A x_1 U_1^T ... x_N U_N^T."""
    A = np.asarray(A, dtype=np.float64)
    _check(A, ranks, P, q)
    info = {} if info is None else info
    Us = []
    for n in range(A.ndim):
        M = unfold(A, n)
        T = sample_count(c, alpha, M.shape[1])
        Us.append(_factor(M, ranks[n], P, q, T, prob, seed, n, form, info))
    G = A
    for n, U in enumerate(Us):
        G = ttm(G, U.T, n)
    return Us, G


def rsthosvd(A, ranks, P=10, q=1, c=0, prob=PROB_UNIFORM, seed=0, alpha=0.0, form=FORM_PAPER,
             info=None):
    """Algorithm 2 (c == 0 and alpha == 0) or Algorithm 5 (AMM): modes in the order
    1..N; after U_n the tensor is replaced by B x_n U_n^T; the last B is the core."""
    B = np.asarray(A, dtype=np.float64)
    _check(B, ranks, P, q)
    info = {} if info is None else info
    Us = []
    for n in range(B.ndim):
        M = unfold(B, n)
        T = sample_count(c, alpha, M.shape[1])
        U = _factor(M, ranks[n], P, q, T, prob, seed, n, form, info)
        Us.append(U)
        B = ttm(B, U.T, n)
    return Us, B


# ---------------------------------------------------------------- deterministic (Section 2.1, 4)
def thosvd(A, ranks):
    """Truncated HOSVD: U_n = leading left singular vectors of A_(n)."""
    A = np.asarray(A, dtype=np.float64)
    Us = [leading_left_singular_vectors(unfold(A, n), ranks[n])[0] for n in range(A.ndim)]
    G = A
    for n, U in enumerate(Us):
        G = ttm(G, U.T, n)
    return Us, G


def sthosvd(A, ranks):
    """Sequentially truncated HOSVD with processing order 1..N."""
    B = np.asarray(A, dtype=np.float64)
    Us = []
    for n in range(B.ndim):
        U = leading_left_singular_vectors(unfold(B, n), ranks[n])[0]
        Us.append(U)
        B = ttm(B, U.T, n)
    return Us, B


# ---------------------------------------------------------------- evaluation (Eq. 8)
def reconstruct(G, Us):
    X = np.asarray(G, dtype=np.float64)
    for n, U in enumerate(Us):
        X = ttm(X, U, n)
    return X


def relative_error(A, Us, G) -> float:
    """RE = ||A - G x_1 U_1 ... x_N U_N||_F / ||A||_F (Eq. 8)."""
    A = np.asarray(A, dtype=np.float64)
    return frobenius(A - reconstruct(G, Us)) / frobenius(A)


def tail_energy_bound(A, ranks) -> float:
    """Right side of the T-HOSVD bound (Eq. 5 with optimal single-mode factors):
    sum_n sum_{i > R_n} sigma_i(A_(n))^2."""
    A = np.asarray(A, dtype=np.float64)
    tot = 0.0
    for n in range(A.ndim):
        s = np.linalg.svd(unfold(A, n), compute_uv=False)
        tot += float(np.sum(s[ranks[n]:] ** 2))
    return tot


# ---------------------------------------------------------------- fixed precision (Problem 2)
def rsthosvd_adaptive(A, eps, P=0, q=1, seed=0, L0=8, form=FORM_PAPER):
    """Problem 2 (concluding section): multilinear ranks and factors with
    ||A - A x_1 Q_1 Q_1^T ... x_N Q_N Q_N^T||_F <= eps ||A||_F.

    Reading (the paper poses the problem only): ST-HOSVD order 1..N. The
    truncation error is the sum of the energies the modes discard (the equality
    behind Eq. 23 / Lemma 8), so mode n may discard
        budget_n = (eps^2 ||A||^2 - discarded so far) / (N - n + 1).
    For mode n a sketch of L columns (L = L0, doubled up to I_n) gives U_L (all
    L leading left singular vectors of the paper form's sketch), the exact
    energies e_k = ||u_k^T B_(n)||^2 and the smallest r with
    ||B||^2 - sum_{k<=r} e_k <= budget_n; without such r the sketch is widened,
    and at L = I_n nothing is discarded. Q_n = U_L(:, 1:r), B <- B x_n Q_n^T.
    Returns (Qs, G, ranks)."""
    B = np.asarray(A, dtype=np.float64)
    N = B.ndim
    total = frobenius(B) ** 2
    allowed = (eps ** 2) * total
    spent = 0.0
    Qs, ranks = [], []
    for n in range(N):
        M = unfold(B, n)
        I = M.shape[0]
        normB = float(np.sum(M * M))
        budget = (allowed - spent) / (N - n)
        L = min(L0, I)
        while True:
            info = {}
            U = _factor(M, L, 0, q, 0, PROB_UNIFORM, seed, n, form, info)    # all L vectors of an L-column sketch
            e = np.sum((U.T @ M) ** 2, axis=1)
            resid = normB - np.cumsum(e)
            ok = np.nonzero(resid <= budget)[0]
            if ok.size or L == I:
                r = int(ok[0]) + 1 if ok.size else I
                break
            L = min(2 * L, I)
        Q = U[:, :r]
        spent += normB - float(np.sum(e[:r]))
        Qs.append(Q)
        ranks.append(r)
        B = ttm(B, Q.T, n)
    return Qs, B, ranks
