"""GB300 (sm_103a) randomized Tucker decompositions: randomized T-HOSVD and
ST-HOSVD with the power scheme and approximate matrix multiplication
(Che, Wei, Yan, arXiv 2303.11612).

The compute path is the CUDA library libtucker.so (C ABI in include/tucker.h);
this package only marshals torch tensors into it. There is no CPU fallback:
importing the binding builds the library if needed and raises if it cannot be
loaded.
"""
from ._binding import (  # noqa: F401
    TuckerError, decompose, rthosvd, rsthosvd, rsthosvd_adaptive, workspace_size, plan_describe, factor_tensor,
    gaussian, power_step, range_sketch, fiber_norms, fiber_norms12, fiber_norms123, fiber_norms123_workspace_size, quantize_weights, sample_fibers, gather_fibers, leading_factor,
    ttm, gram, cholqr, leading_factor_chain, sample_factor, quantize_weights_max, sample_fibers_slab,
    relative_error, last_device_status, lib, exported_symbols, FLAG_ASYNC, launch_count, profile_enable, batch_describe,
    profile_read, Server, Batch, autotune_enable, autotune_entries,
)

__all__ = ["rthosvd", "rsthosvd", "rsthosvd_adaptive", "decompose", "workspace_size", "plan_describe", "TuckerError", "Server", "Batch"]
