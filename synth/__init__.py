"""Seeded synthetic input tensors shaped like the paper's workloads.

This module is shared by the FP64 oracle, the tests and the benchmark. It holds
none of the decomposition's arithmetic: it only builds input tensors from a
seeded numpy generator (PCG64). The random numbers the method itself draws (the
Gaussian test matrices and the fiber-sampling uniforms) do not come from here;
each side implements the counter-based Philox4x32-10 stream for those.

Layout convention: every tensor is returned as a numpy array of shape
(I_1, ..., I_N) in Fortran order, i.e. i_1 varies fastest in memory, which is
the element order implied by the mode-n unfolding index map of Section 2. The
flat buffer handed to the CUDA library is ``flat(A)``.

Workload recipes (Section 6 shapes, scaled):
  * ``lowrank_noise``: G x_1 U_1 ... x_N U_N + noise, G i.i.d. N(0,1) (or U(0,1),
    Eq. 9), U_n orthonormal from the QR of a Gaussian matrix with diag(R) > 0,
    noise scaled to a stated relative Frobenius norm (Section 6.2 / Eq. 9).
  * ``hilbert``: a_{i_1..i_N} = 1 / (i_1 + ... + i_N - N + 1), 1-based indices.
  * ``decaying_core``: core entries N(0,1) * ratio**(i_1+...+i_N) (0-based),
    orthonormal factors, no noise (exact multilinear rank = core size).
  * ``video_like``: sum of separable sinusoids with random frequencies plus
    Gaussian noise (a stand-in for the hyperspectral / video tensors of
    Section 6.4, whose datasets are not available).
  * ``tendiag``: superdiagonal core v x_n A_n with square orthogonal A_n
    (Section 6.3).
  * ``sparse_rank1_sum``: sum of weighted outer products of sparse vectors
    (Section 6.1).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "flat", "from_flat", "orthonormal", "mode_product", "lowrank_noise", "hilbert",
    "decaying_core", "video_like", "tendiag", "sparse_rank1_sum", "serving_requests",
    "sample_weights",
]


def flat(A: np.ndarray) -> np.ndarray:
    """The tensor's memory as a 1-D array, i_1 fastest."""
    return np.ravel(A, order="F")


def from_flat(buf: np.ndarray, dims) -> np.ndarray:
    """Inverse of ``flat``: view a 1-D buffer (i_1 fastest) as shape ``dims``."""
    return np.reshape(np.asarray(buf), tuple(int(d) for d in dims), order="F")


def orthonormal(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """Q factor of the QR of a rows x cols standard Gaussian, signs set so diag(R) > 0."""
    B = rng.standard_normal((rows, cols))
    Q, R = np.linalg.qr(B)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def mode_product(T: np.ndarray, M: np.ndarray, n: int) -> np.ndarray:
    """T x_n M for building inputs (M is J x I_n). Used only to synthesise tensors."""
    Tm = np.moveaxis(T, n, 0)
    out = np.tensordot(M, Tm, axes=([1], [0]))
    return np.asfortranarray(np.moveaxis(out, 0, n))


def _with_noise(rng, B, rel_noise, dtype):
    if rel_noise > 0:
        E = rng.standard_normal(B.shape)
        B = B + (rel_noise * np.linalg.norm(B) / np.linalg.norm(E)) * E
    return np.asfortranarray(B.astype(dtype))


def lowrank_noise(dims, core_dims, rel_noise=1e-3, seed=0, dtype=np.float32,
                  core_dist="normal"):
    """G x_1 U_1 ... x_N U_N + E with ||E||_F = rel_noise * ||G x U||_F."""
    rng = np.random.default_rng(seed)
    dims = tuple(int(d) for d in dims)
    core_dims = tuple(int(r) for r in core_dims)
    if core_dist == "uniform":
        G = rng.random(core_dims)
    else:
        G = rng.standard_normal(core_dims)
    B = np.asfortranarray(G)
    for n, (I, R) in enumerate(zip(dims, core_dims)):
        B = mode_product(B, orthonormal(rng, I, R), n)
    return _with_noise(rng, B, rel_noise, dtype)


def hilbert(dims, dtype=np.float32):
    """Hilbert-type tensor a = 1 / (i_1 + ... + i_N - N + 1) with 1-based indices."""
    dims = tuple(int(d) for d in dims)
    grids = np.meshgrid(*[np.arange(1, d + 1, dtype=np.float64) for d in dims], indexing="ij")
    s = sum(grids) - len(dims) + 1
    return np.asfortranarray((1.0 / s).astype(dtype))


def decaying_core(dims, core, ratio=0.8, seed=0, dtype=np.float32):
    """Core N(0,1) * ratio**(sum of 0-based indices), orthonormal factors, no noise."""
    rng = np.random.default_rng(seed)
    dims = tuple(int(d) for d in dims)
    core_dims = (int(core),) * len(dims) if np.isscalar(core) else tuple(int(c) for c in core)
    G = rng.standard_normal(core_dims)
    idx = np.meshgrid(*[np.arange(c) for c in core_dims], indexing="ij")
    G = G * ratio ** sum(idx)
    B = np.asfortranarray(G)
    for n, (I, R) in enumerate(zip(dims, core_dims)):
        B = mode_product(B, orthonormal(rng, I, R), n)
    return np.asfortranarray(B.astype(dtype))


def video_like(dims, terms=50, noise_var=1e-2, seed=0, dtype=np.float32):
    """Sum of ``terms`` separable sinusoids (frequencies U(0, 0.05)*2*pi per mode,
    phases U(0, 2*pi), amplitudes N(0,1)) plus N(0, noise_var) noise."""
    rng = np.random.default_rng(seed)
    dims = tuple(int(d) for d in dims)
    amps = rng.standard_normal(terms)
    facs = []
    for d in dims:
        w = rng.random(terms) * 0.05 * 2 * np.pi
        ph = rng.random(terms) * 2 * np.pi
        facs.append(np.sin(np.outer(np.arange(d), w) + ph))  # d x terms
    # Khatri-Rao of the trailing factors (first trailing index fastest), then one GEMM.
    kr = facs[1]
    for F in facs[2:]:
        kr = (F[:, None, :] * kr[None, :, :]).reshape(-1, terms)
    body = ((facs[0] * amps).astype(np.float32) @ kr.T.astype(np.float32))
    out = body.reshape(-1, order="F")
    out += rng.standard_normal(out.size, dtype=np.float32) * np.float32(np.sqrt(noise_var))
    out = out.astype(dtype, copy=False)
    return from_flat(out, dims)


def tendiag(v, dims, seed=0, dtype=np.float64):
    """Superdiagonal tensor with diagonal v, multiplied in every mode by a square
    orthogonal matrix (Q of a Gaussian, diag(R) > 0)."""
    rng = np.random.default_rng(seed)
    dims = tuple(int(d) for d in dims)
    k = len(v)
    D = np.zeros((k,) * len(dims))
    for i, vi in enumerate(v):
        D[(i,) * len(dims)] = vi
    B = np.asfortranarray(D)
    for n, I in enumerate(dims):
        B = mode_product(B, orthonormal(rng, I, I)[:, :k], n)
    return np.asfortranarray(B.astype(dtype))


def sparse_rank1_sum(dims, terms, gamma=1000.0, lead=50, density=0.05, seed=0, dtype=np.float32):
    """sum_i w_i x_i o y_i o ... with sparse vectors; w_i = gamma/i^2 for i <= lead,
    1/i^2 otherwise (1-based i)."""
    rng = np.random.default_rng(seed)
    dims = tuple(int(d) for d in dims)
    A = np.zeros(dims)
    for i in range(1, terms + 1):
        w = (gamma if i <= lead else 1.0) / i ** 2
        vecs = []
        for d in dims:
            x = rng.standard_normal(d) * (rng.random(d) < density)
            vecs.append(x)
        t = w * vecs[0]
        for x in vecs[1:]:
            t = np.multiply.outer(t, x)
        A += t
    return np.asfortranarray(A.astype(dtype))


def serving_requests(count, seed=0, dim_range=(32, 256), rank_range=(4, 32), orders=(3, 4),
                     rate=None):
    """Request specs of the serving workload: order 3 or 4 (equal odds), every dim
    uniform in dim_range, ranks uniform in rank_range (clamped to the dim), and
    Poisson arrival times when ``rate`` (requests/s) is given."""
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for k in range(count):
        N = int(rng.choice(orders))
        dims = tuple(int(d) for d in rng.integers(dim_range[0], dim_range[1] + 1, size=N))
        ranks = tuple(int(min(r, d)) for r, d in
                      zip(rng.integers(rank_range[0], rank_range[1] + 1, size=N), dims))
        if rate:
            t += float(rng.exponential(1.0 / rate))
        reqs.append({"id": k, "dims": dims, "ranks": ranks, "seed": int(rng.integers(0, 2**31)),
                     "arrival_s": t})
    return reqs


def sample_weights(J, seed=0, kind="mixed"):
    """Synthetic uint64 sampling weights (for testing the sampler alone):
    'mixed' = heavy-tailed with zeros, 'ones' = all 1, 'spiky' = few large."""
    rng = np.random.default_rng(seed)
    if kind == "ones":
        return np.ones(J, dtype=np.uint64)
    if kind == "spiky":
        W = rng.integers(0, 4, size=J).astype(np.uint64)
        W[rng.integers(0, J, size=max(1, J // 100))] = np.uint64(1 << 24)
        return W
    W = (rng.pareto(1.5, size=J) * 1000).astype(np.uint64)
    W[rng.random(J) < 0.1] = 0
    W = np.minimum(W, np.uint64(1 << 24))
    if W.sum() == 0:
        W[0] = 1
    return W
