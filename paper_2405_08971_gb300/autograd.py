"""torch.autograd.Function wrapper of the CAKF negative log likelihood.

forward(theta) runs cakf_filter + cakf_nll for theta = (log l_x, log l_t, log sf2, log sn2);
backward returns grad_output * cakf_nll_backward (the gradient with the actions and truncation
rotations of that forward run held fixed).  All compute happens in libcakf.so.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class _NLL(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, data, precision, stream):
        th = theta.detach().to("cpu", torch.float64).numpy()
        prob = B.make_problem(data["coords"], data["kernel"], th[0], th[1], th[2], th[3], data["T"], data["dt"],
                              data["obs_ptr"], data["obs_idx"], data["y"], data["budget_i"], data["rank_r"],
                              precision=precision, prior_mean=data.get("prior_mean"))
        c, _, _ = B.cakf_filter(prob, None, want_outputs=False, stream=stream)
        nll = B.cakf_nll(c)
        ctx.cakf = c
        ctx.device = theta.device
        return torch.tensor(nll, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        g = B.cakf_nll_backward(ctx.cakf)
        ctx.cakf.close()
        return grad_out * torch.as_tensor(g, dtype=torch.float64, device=ctx.device), None, None, None


def cakf_neg_log_likelihood(theta: torch.Tensor, data: dict, precision: str = "fp32", stream=None) -> torch.Tensor:
    """NLL of the projected data as a differentiable function of theta (shape (4,))."""
    return _NLL.apply(theta, data, precision, stream)


def workload_data(w) -> dict:
    """The fields cakf_neg_log_likelihood needs, from a synth.Workload-like object."""
    return {"coords": w.coords, "kernel": w.kernel, "T": w.T, "dt": w.dt, "obs_ptr": w.obs_ptr,
            "obs_idx": w.obs_idx, "y": w.y, "budget_i": w.budget_i, "rank_r": w.rank_r,
            "prior_mean": w.prior_mean}
