"""FP64 CPU oracle for the computation-aware Kalman filter and smoother.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
it is used by `tests/`, by `__graft_entry__.smoke()` and by the `cpu_baseline`
/ `--impl reference` legs of `bench.py`.  It shares no code with the CUDA path.
"""
from .cakf import (  # noqa: F401
    kernel_matrix, matern, Model, model_from, filter_run, smoother_run, nll_terms, nll_total,
    truncate, nll_grad_fd, FilterResult, update_iterative, update_batch, coordinate_actions,
    sample_run, interpolate_run, smoother_messages,
)
