"""GB300-native computation-aware Kalman filter and smoother (arXiv 2405.08971).

The compute path is libcakf.so (CUDA kernels for sm_103a behind the C ABI in
include/cakf.h); `binding` marshals arguments to it.  Importing the package does
not load the library; the first call does, and fails loudly if it is missing.
"""
from .binding import (  # noqa: F401
    Context, CakfError, make_problem, problem_from_workload, cakf_filter, cakf_smooth, cakf_nll,
    cakf_nll_backward, cakf_get_actions, cakf_gram_matmul, cakf_gram_matmul_noalloc, cakf_eig_topk, cakf_get_stats,
    cakf_set_profiling, cakf_probe_peaks, cakf_factor_gemm, cakf_get_diagnostics, cakf_sample, cakf_interpolate, cakf_set_wait_limit,
    cakf_set_device_memory_limit, pack_actions, lib,
    FP64, FP32, TF32, BF16, FP16X3, TF32X3, MATERN12, MATERN32, MATERN52,
)
