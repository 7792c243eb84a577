"""Argument checks of the Python binding that run before any call into the C
ABI (so without a GPU): the ABI reads N extents and N ranks and the tensor as
dense memory with i_1 fastest, so mismatched lengths, non-contiguous tensors
and mis-shaped outputs must be refused here rather than read out of bounds."""
import pytest
import torch

from paper_2303_11612_gb300 import _binding as B


def test_problem_checks():
    A = torch.zeros(4 * 5 * 6)
    assert B._problem("ST", A, (4, 5, 6), (2, 2, 2)) == ([4, 5, 6], [2, 2, 2])
    with pytest.raises(ValueError):
        B._problem("X", A, (4, 5, 6), (2, 2, 2))                  # neither T nor ST
    with pytest.raises(ValueError):
        B._problem("T", A, (4, 5, 6), (2, 2))                     # fewer ranks than extents
    with pytest.raises(ValueError):
        B._problem("T", A, (), ())
    with pytest.raises(ValueError):
        B._problem("T", A, (4, 5, 7), (2, 2, 2))                  # numel mismatch
    with pytest.raises(ValueError):
        B._problem("T", torch.zeros(6, 5, 4).permute(2, 1, 0), (4, 5, 6), (2, 2, 2))   # not dense
    with pytest.raises(TypeError):
        B._problem("T", torch.zeros(120, dtype=torch.int32), (4, 5, 6), (2, 2, 2))


def test_output_checks():
    A = torch.zeros(4 * 5 * 6)
    U, G = B._outputs(None, A, [4, 5, 6], [2, 3, 1], "cpu")
    assert [tuple(u.shape) for u in U] == [(4, 2), (5, 3), (6, 1)] and all(u.stride(0) == 1 for u in U)
    assert G.numel() == 6
    assert B._outputs((U, G), A, [4, 5, 6], [2, 3, 1], "cpu")[1] is G
    with pytest.raises(ValueError):                                # row-major factor
        B._outputs(([torch.zeros(4, 2)] + U[1:], G), A, [4, 5, 6], [2, 3, 1], "cpu")
    with pytest.raises(ValueError):                                # a factor missing
        B._outputs((U[:2], G), A, [4, 5, 6], [2, 3, 1], "cpu")
    with pytest.raises(ValueError):                                # core of the wrong size
        B._outputs((U, torch.zeros(5)), A, [4, 5, 6], [2, 3, 1], "cpu")
    with pytest.raises(ValueError):                                # dtype differs from A's
        B._outputs((U, G.double()), A, [4, 5, 6], [2, 3, 1], "cpu")


def test_public_calls_refuse_bad_arguments_before_the_library():
    A = torch.zeros(4 * 5 * 6)
    with pytest.raises(ValueError):
        B.decompose("ST", A, (4, 5, 6), (2, 2))
    with pytest.raises(ValueError):
        B.decompose("Q", A, (4, 5, 6), (2, 2, 2))
    with pytest.raises(ValueError):
        B.workspace_size("Q", (4, 5, 6), (2, 2, 2))
    with pytest.raises(ValueError):
        B.Batch([dict(which="ST", A=A, dims=(4, 5, 6), ranks=(2, 2))])
