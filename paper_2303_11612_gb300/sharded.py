"""Slab-sharded randomized ST-HOSVD (Algorithm 2, and Algorithm 5 with AMM)
over the ranks of a torch.distributed process group, one GPU per rank.

Partitioning: the tensor is split along its last mode N into slabs, rank r
holding indices i_N in [a_r, b_r) (balanced) as its own dense tensor with i_1
fastest. Mode N is the most significant part of every mode-n fiber index
(n < N), so a slab's fibers are the consecutive global fibers
a_r * J_n / I_N .. b_r * J_n / I_N - 1.

For every mode n < N (processing order 1..N, Section 4):
  * sketch: the mode-n power step of Strategy A is a sum over the slabs,
    A_(n) (A_(n)^T X) = sum_r A_r (A_r^T X): each step's I_n x L product is
    all-reduced (one collective of I_n L values per power step); the CholeskyQR
    factors between steps and the extraction (remark after Algorithm 5) run on
    identical inputs, so every rank obtains the same U_n;
  * AMM (Algorithm 5): the largest fiber weight is all-reduced (max) so every
    slab quantises against it, the slabs' weight totals are all-gathered, and
    each rank resolves the draws of RANDSAMPLE (Section 3.2) that land in its
    range of the CDF; one all-reduce (max) assembles the global indices and
    scales, the owners gather their sampled fibers and one all-reduce (sum)
    assembles C' (columns of other ranks are zeros), from which every rank
    computes U_n;
  * the truncation B <- B x_n U_n^T (Algorithm 2) is slab-local.
Before mode N the tensor is R_1 ... R_{N-1} x I_N: its slabs are all-gathered
(concatenation in rank order along the slowest mode) and mode N is computed on
every rank, as is the core.

The result equals a single-rank call up to the summation order of the power
steps' partial products; the sampled fiber indices are the same, bit for bit.
The local steps come from a provider object: ``LibrarySteps`` runs them through
the library's C ABI on the rank's GPU (collectives then use NCCL tensors on the
device); any object with the same methods can stand in.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence, Tuple

import torch


def slab_bounds(extent: int, world: int, rank: int) -> Tuple[int, int]:
    """[a, b) of the last mode held by `rank` (balanced, earlier ranks larger)."""
    base, extra = divmod(extent, world)
    a = rank * base + min(rank, extra)
    return a, a + base + (1 if rank < extra else 0)


def sample_count(c: int, J: int) -> int:
    """T_n = min(c, J_n) for c > 0 (AMM), else 0."""
    return int(min(c, J)) if c > 0 else 0


class Comm:
    """The collectives the sharded driver uses, over a torch.distributed group
    (or a single rank when no group is initialised)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        self.group = group
        self.rank = self.dist.get_rank(group) if self.dist else 0
        self.size = self.dist.get_world_size(group) if self.dist else 1

    def sum_(self, t: torch.Tensor) -> torch.Tensor:
        if self.dist and self.size > 1:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t

    def max_(self, t: torch.Tensor) -> torch.Tensor:
        if self.dist and self.size > 1:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return t

    def gather_ints(self, x: int, device) -> List[int]:
        """Every rank's integer, in rank order."""
        t = torch.zeros(self.size, dtype=torch.int64, device=device)
        t[self.rank] = int(x)
        return [int(v) for v in self.sum_(t).tolist()]

    def gather_flat(self, t: torch.Tensor) -> torch.Tensor:
        """The concatenation, in rank order, of every rank's 1-D tensor."""
        if not (self.dist and self.size > 1):
            return t
        n = self.gather_ints(t.numel(), t.device)
        m = max(n)
        buf = torch.zeros(m, dtype=t.dtype, device=t.device)
        buf[:t.numel()] = t
        parts = [torch.empty_like(buf) for _ in range(self.size)]
        self.dist.all_gather(parts, buf, group=self.group)
        return torch.cat([p[:k] for p, k in zip(parts, n)])


class LibrarySteps:
    """Local steps through the library's C ABI on the rank's GPU."""

    def __init__(self, prec: str = "fp32", stream=None):
        from . import _binding as B
        self.B = B
        self.prec = prec
        self.stream = stream

    def gaussian(self, I, L, seed, mode, dtype, device):
        return self.B.gaussian(I, L, seed, (0 << 8) | mode, dtype=dtype, device=device, stream=self.stream)

    def power(self, A, dims, n, X):
        return self.B.power_step(A, dims, n, X, stream=self.stream, prec=self.prec)

    def cholqr(self, X):
        return self.B.cholqr(X, stream=self.stream)

    def factor(self, X, R, factors):
        return self.B.leading_factor_chain(X, R, factors, stream=self.stream)

    def fiber_norms(self, A, dims, n):
        return self.B.fiber_norms(A, dims, n, stream=self.stream)

    def quantize_max(self, w, wmax):
        return self.B.quantize_weights_max(w, wmax, stream=self.stream)

    def sample_slab(self, W, T, seed, n, S_offset, S_total, fiber_offset):
        return self.B.sample_fibers_slab(W, T, seed, n, S_offset, S_total, fiber_offset, stream=self.stream)

    def gather(self, A, dims, n, idx, scale):
        return self.B.gather_fibers(A, dims, n, idx, scale, stream=self.stream)

    def sample_factor(self, Cp, R, P, q, seed, n):
        return self.B.sample_factor(Cp, R, P, q, seed, n, stream=self.stream)

    def ttm(self, A, dims, n, U):
        return self.B.ttm(A, dims, n, U, transpose=True, stream=self.stream, prec=self.prec).reshape(-1)


def _mode_factor(comm: Comm, steps, cur, cur_dims, n, R, P, q, c, prob, seed, fiber_offset, J_global):
    """U_n for the current (local) tensor; collectives over `comm`. Returns
    (U_n, sampled global fiber indices or None)."""
    I = cur_dims[n]
    L = min(R + P, I)
    J_local = cur.numel() // I
    T = sample_count(c, J_global)
    dev = cur.device
    if T == 0:
        X = steps.gaussian(I, L, seed, n, cur.dtype, dev)
        factors = []
        for k in range(q):
            if k > 0:
                X, F = steps.cholqr(X)
                factors.append(F)
            # I x L column-major: its transpose is the contiguous block the all-reduce sums
            Y = steps.power(cur, cur_dims, n, X) if J_local else torch.zeros((L, I), dtype=cur.dtype, device=dev).t()
            X = comm.sum_(Y.t().contiguous()).t()
        return steps.factor(X, R, factors), None
    # RANDSAMPLE over all slabs
    if prob == "nearly_optimal" and J_local:
        w = steps.fiber_norms(cur, cur_dims, n)
        wmax = comm.max_(torch.tensor([float(w.max())], dtype=torch.float64, device=dev)).item()
        W = steps.quantize_max(w, wmax)
    elif prob == "nearly_optimal":
        comm.max_(torch.zeros(1, dtype=torch.float64, device=dev))
        W = torch.zeros(0, dtype=torch.int64, device=dev)
    else:
        W = torch.ones(J_local, dtype=torch.int64, device=dev)
    totals = comm.gather_ints(int(W.sum().item()) if J_local else 0, dev)
    S_off, S_tot = sum(totals[:comm.rank]), sum(totals)
    if J_local and totals[comm.rank] > 0:
        idx, scale = steps.sample_slab(W, T, seed, n, S_off, S_tot, fiber_offset)
    else:
        idx = torch.full((T,), -1, dtype=torch.int64, device=dev)
        scale = torch.zeros(T, dtype=torch.float64, device=dev)
    idx = comm.max_(idx.clone())
    scale = comm.max_(scale.clone())
    own = (idx >= fiber_offset) & (idx < fiber_offset + J_local)
    if J_local:
        Cp = steps.gather(cur, cur_dims, n, torch.where(own, idx - fiber_offset, torch.zeros_like(idx)),
                          torch.where(own, scale, torch.zeros_like(scale)))
    else:
        Cp = torch.zeros((T, I), dtype=cur.dtype, device=dev).t()
    Cp = comm.sum_(Cp.t().contiguous()).t()                 # each column from its owner, zeros elsewhere
    return steps.sample_factor(Cp, R, P, q, seed, n), idx


def rsthosvd_sharded(A_local: torch.Tensor, dims: Sequence[int], ranks: Sequence[int], P: int = 10, q: int = 1,
                     c: int = 0, prob: str = "uniform", seed: int = 0, steps=None, group=None,
                     samples: Optional[list] = None):
    """Randomized ST-HOSVD of a tensor of shape `dims` whose last-mode slab
    slab_bounds(dims[-1], world, rank) this rank holds in A_local (flat, i_1
    fastest). Returns (factors U_n, core G flat), the same on every rank. When
    `samples` is a list it receives each mode's sampled global fiber indices."""
    comm = Comm(group)
    steps = steps or LibrarySteps()
    dims = [int(d) for d in dims]
    ranks = [int(r) for r in ranks]
    N = len(dims)
    if N < 2 or len(ranks) != N:
        raise ValueError("need an order >= 2 tensor and one rank per mode")
    if dims[-1] < comm.size:
        raise ValueError("the last mode must have at least one index per rank")
    a, b = slab_bounds(dims[-1], comm.size, comm.rank)
    if A_local.numel() != math.prod(dims[:-1]) * (b - a):
        raise ValueError("A_local must hold exactly this rank's slab")
    cur = A_local.reshape(-1)
    cur_dims = dims[:-1] + [b - a]
    full_dims = list(dims)
    Us = []
    for n in range(N - 1):
        J_global = math.prod(full_dims) // full_dims[n]
        fiber_offset = a * (J_global // full_dims[-1])
        U, idx = _mode_factor(comm, steps, cur, cur_dims, n, ranks[n], P, q, c, prob, seed, fiber_offset, J_global)
        if samples is not None:
            samples.append(idx)
        Us.append(U)
        cur = steps.ttm(cur, cur_dims, n, U)
        cur_dims[n] = ranks[n]
        full_dims[n] = ranks[n]
    # the small tensor R_1 ... R_{N-1} x I_N: slabs concatenated along the slowest mode
    B = comm.gather_flat(cur.contiguous())
    single = Comm.__new__(Comm)
    single.dist, single.group, single.rank, single.size = None, None, 0, 1
    n = N - 1
    U, idx = _mode_factor(single, steps, B, full_dims, n, ranks[n], P, q, c, prob, seed, 0,
                          math.prod(full_dims) // full_dims[n])
    if samples is not None:
        samples.append(idx)
    Us.append(U)
    G = steps.ttm(B, full_dims, n, U)
    return Us, G
