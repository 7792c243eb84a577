"""Seeded synthetic tensors generated on a CUDA device with torch, following the
same recipes as the numpy generators of this package (used where many large
distinct inputs are needed quickly, e.g. one tensor per slot of a batch).

The values are NOT bitwise equal to the numpy generators' for the same seed:
the random draws of the noise and of the factors come from torch's device
generator. Parameters that are small (sinusoid amplitudes, frequencies and
phases) are drawn with numpy exactly as the numpy recipe draws them. Nothing
here holds any of the decomposition's arithmetic.
"""
from __future__ import annotations

import numpy as np


def _gen(torch, seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def video_like(torch, dims, terms=50, noise_var=1e-2, seed=0, device="cuda"):
    """The recipe of ``synth.video_like``: a sum of ``terms`` separable sinusoids
    (frequencies U(0, 0.05) 2 pi per mode, phases U(0, 2 pi), amplitudes N(0,1))
    plus N(0, noise_var) noise; flat FP32, i_1 fastest."""
    rng = np.random.default_rng(seed)
    dims = tuple(int(d) for d in dims)
    amps = rng.standard_normal(terms)
    facs = []
    for d in dims:
        w = rng.random(terms) * 0.05 * 2 * np.pi
        ph = rng.random(terms) * 2 * np.pi
        facs.append(torch.from_numpy(np.sin(np.outer(np.arange(d), w) + ph)).to(device, torch.float32))
    kr = facs[1]
    for F in facs[2:]:
        kr = (F[:, None, :] * kr[None, :, :]).reshape(-1, terms)
    f0 = facs[0] * torch.from_numpy(amps).to(device, torch.float32)[None, :]
    out = (kr @ f0.t()).reshape(-1)          # element (i_1, j) at j * I_1 + i_1
    del kr
    noise = torch.randn(out.numel(), device=device, generator=_gen(torch, seed, device))
    out.add_(noise, alpha=float(np.sqrt(noise_var)))
    return out


def tucker_tensor(torch, dims, core_dims, rel_noise=1e-2, seed=0, core_scale=None, device="cuda"):
    """G x_1 U_1 ... x_N U_N with a N(0,1) core (times ``core_scale`` entrywise if
    given, an array of the core's shape, i_1 fastest), U_n orthonormal from the
    QR of Gaussian matrices, plus Gaussian noise at ``rel_noise`` relative
    Frobenius norm (none if 0); flat FP32, i_1 fastest."""
    g = _gen(torch, seed, device)
    N = len(dims)
    X = torch.randn(*reversed(core_dims), device=device, generator=g)
    if core_scale is not None:
        X = X * torch.from_numpy(np.ascontiguousarray(np.asarray(core_scale).T)).to(device, torch.float32)
    for m in range(N):                       # X x_m U_m; i_1 fastest means torch axis N-1-m
        Um = torch.linalg.qr(torch.randn(dims[m], core_dims[m], device=device, generator=g))[0]
        X = torch.movedim(torch.tensordot(X, Um, dims=([N - 1 - m], [1])), -1, N - 1 - m)
    X = X / X.norm()
    if rel_noise > 0:
        E = torch.randn(X.shape, device=device, generator=g)
        X = X + rel_noise * E / E.norm()
    return X.contiguous().view(-1)


def tucker_tensor_lean(torch, dims, core_dims, rel_noise=1e-2, seed=0, device="cuda", chunk=1 << 27):
    """The recipe of ``tucker_tensor`` for tensors of many GB: the mode products
    are applied from the last mode to the first, so that the first lands on the
    innermost axis and the result is built contiguous without a copy, and the
    noise is drawn in chunks from per-chunk generators (one pass for its norm, a
    second, re-seeded, to add it), so that the peak footprint is the tensor
    itself plus one chunk. Flat FP32, i_1 fastest."""
    g = _gen(torch, seed, device)
    N = len(dims)
    X = torch.randn(*reversed(core_dims), device=device, generator=g)
    Us = [torch.linalg.qr(torch.randn(dims[m], core_dims[m], device=device, generator=g))[0] for m in range(N)]
    for m in reversed(range(N)):                   # mode m is torch axis N-1-m
        X = torch.tensordot(X, Us[m], dims=([N - 1 - m], [1]))
        if m > 0:
            X = torch.movedim(X, -1, N - 1 - m)
    X = X.reshape(-1)
    X /= X.norm()
    if rel_noise > 0:
        n = X.numel()
        starts = range(0, n, chunk)
        ss = 0.0
        for k, a in enumerate(starts):
            e = torch.randn(min(chunk, n - a), device=device, generator=_gen(torch, seed * 1_000_003 + k + 1, device))
            ss += float(torch.dot(e, e))
        scale = rel_noise / float(np.sqrt(ss))
        for k, a in enumerate(starts):
            e = torch.randn(min(chunk, n - a), device=device, generator=_gen(torch, seed * 1_000_003 + k + 1, device))
            X[a:a + e.numel()].add_(e, alpha=scale)
    return X
