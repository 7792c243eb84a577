"""Algorithms 6 and 7 (the related forms of Algorithms 1 and 2, form RELATED)
on the GPU, against the FP64 oracle's related form on the same bytes.

Per mode: the paper form's sketch, P_n = its orthonormal basis (CholeskyQR2),
one more power step Z = A_(n) (A_(n)^T P_n), H = P_n^T Z, the leading
eigenvectors U of H (= the leading left singular vectors of P_n^T A_(n)), and
Q_n = P_n U with the sign rule. Bars as for the paper form: FP32 relative
error within 1e-5 of the oracle's and projectors within 1e-4 (the tensors
have a gap at R_n); tensor-core forms within 1e-3; orthonormal factors; every
column's largest-magnitude entry positive."""
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


@pytest.mark.parametrize("which", ["T", "ST"])
@pytest.mark.parametrize("q", [1, 2])
@pytest.mark.parametrize("dims,ranks,P", [((120, 100, 90), (8, 6, 7), 5), ((1024, 96, 40), (64, 16, 8), 16)])
def test_related_form_against_the_oracle(tk, which, q, dims, ranks, P):
    A = synth.lowrank_noise(dims, ranks, rel_noise=1e-2, seed=21)
    A64 = A.astype(np.float64)
    fn = ot.rthosvd if which == "T" else ot.rsthosvd
    Uo, Go = fn(A64, ranks, P=P, q=q, seed=4, form=ot.FORM_RELATED)
    reo = ot.relative_error(A64, Uo, Go)
    At = torch.from_numpy(np.ascontiguousarray(synth.flat(A))).cuda()
    for prec in ("fp32", "bf16", "bf16x1"):
        U, G = tk.decompose(which, At, dims, ranks, P=P, q=q, seed=4, form="related", prec=prec)
        U = [u.double().cpu().numpy() for u in U]
        G = synth.from_flat(G.double().cpu().numpy(), ranks)
        re = ot.relative_error(A64, U, G)
        assert abs(re - reo) <= (1e-5 if prec == "fp32" else 1e-3), (prec, re, reo)
        for u, uo in zip(U, Uo):
            assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) < 10 * u.shape[1] * 1.19e-7
            k = np.argmax(np.abs(u), axis=0)
            assert np.all(u[k, np.arange(u.shape[1])] > 0)
            if prec == "fp32":
                assert np.linalg.norm(u @ u.T - uo @ uo.T, 2) <= 1e-4


def test_related_form_rejects_amm(tk):
    dims = (40, 36, 32)
    A = torch.randn(40 * 36 * 32, device="cuda")
    with pytest.raises(tk.TuckerError) as e:
        tk.rsthosvd(A, dims, (4, 4, 4), P=3, c=100, form="related")
    assert e.value.status == 6
