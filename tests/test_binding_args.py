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


def test_step_wrappers_refuse_mis_shaped_operands():
    """Every step wrapper checks the shapes the C ABI will read (an X with fewer
    than I_n rows, an M of the wrong extent, index/scale vectors of other
    types) before calling it."""
    dims = (4, 5, 6)
    A = torch.zeros(120)
    with pytest.raises(ValueError):
        B.power_step(A, dims, 3, torch.zeros(4, 2))                 # mode out of range
    with pytest.raises(ValueError):
        B.power_step(A, dims, 1, torch.zeros(4, 2).t().contiguous().t())   # 4 rows, I_n = 5
    with pytest.raises(ValueError):
        B.power_step(A, dims, 0, torch.zeros(4, 2, dtype=torch.float64))   # dtype differs from A's
    with pytest.raises(ValueError):
        B.power_step_noalloc(A[:119], dims, 0, torch.zeros(4, 2))   # numel mismatch
    with pytest.raises(ValueError):
        B.ttm(A, dims, 1, torch.zeros(3, 4), transpose=False)       # K x I_n needs I_n = 5 columns
    with pytest.raises(ValueError):
        B.ttm(A, dims, 1, torch.zeros(4, 3), transpose=True)        # I_n x K needs I_n = 5 rows
    with pytest.raises(ValueError):
        B.gather_fibers(A, dims, 0, torch.zeros(3), torch.zeros(3, dtype=torch.float64))   # float indices
    with pytest.raises(ValueError):
        B.gather_fibers(A, dims, 0, torch.zeros(3, dtype=torch.int64), torch.zeros(2, dtype=torch.float64))
    with pytest.raises(ValueError):
        B.fiber_norms(A, dims, -1)
    with pytest.raises(ValueError):
        B.range_sketch(A.view(6, 5, 4).transpose(0, 2), dims, 0, 3, seed=0)   # not dense
    with pytest.raises(ValueError):
        B.quantize_weights(torch.zeros(10, dtype=torch.float32))
    with pytest.raises(ValueError):
        B.sample_fibers(torch.zeros(10, dtype=torch.float64), 4, seed=0, mode=0)
    U = [B.factor_tensor(I, 2, torch.float32, "cpu") for I in dims]
    with pytest.raises(ValueError):
        B.relative_error(A, dims, (2, 2, 2), U[:2], torch.zeros(8))
    with pytest.raises(ValueError):
        B.relative_error(A, dims, (2, 2, 2), U, torch.zeros(7))


def test_binding_flags_match_the_header():
    """The binding's TUCKER_FLAG_* values are the header's."""
    import re
    from pathlib import Path
    from paper_2303_11612_gb300 import _binding as B
    text = (Path(__file__).resolve().parents[1] / "include" / "tucker.h").read_text()
    flags = {m.group(1): int(m.group(2), 16) for m in re.finditer(r"#define TUCKER_FLAG_(\w+) (0x[0-9a-fA-F]+)u", text)}
    assert flags == {"ASYNC": B.FLAG_ASYNC, "WORKLIST": B.FLAG_WORKLIST}


def test_norms123_workspace_size_arguments():
    """tucker_fiber_norms123_workspace_size: order 3 only, I_1 <= 1024; the size
    covers the band partials (8 bytes per mode-2 entry and band) at least."""
    from paper_2303_11612_gb300 import _binding as B
    n = B.fiber_norms123_workspace_size((400, 300, 7))
    assert n >= 400 * 7 * 8 * ((300 + 15) // 16)
    with pytest.raises(B.TuckerError) as e:
        B.fiber_norms123_workspace_size((1100, 4, 4))
    assert e.value.status == 6
    with pytest.raises(B.TuckerError) as e:
        B.fiber_norms123_workspace_size((10, 4, 4, 4))
    assert e.value.status == 1
