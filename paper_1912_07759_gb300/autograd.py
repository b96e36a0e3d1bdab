"""torch.autograd.Function over the batched forward model and its hand-written adjoint.

TransitSpectrum.apply(theta, model) returns the binned transit depths [B][n_bin] of the
parameter vectors theta [B][n_theta] (float64, CUDA); its backward calls tr_adjoint_transit in
vector-Jacobian-product mode with the upstream gradient.  Both directions run in the
library's CUDA kernels.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import torch

from . import transit as T


@dataclasses.dataclass
class BatchModel:
    """Everything fixed across calls: context, tables, bins, batch description, layer counts."""
    ctx: T.TransitContext
    tables: T.XsecTables
    bins: T.Bins
    spec: T.BatchSpec
    nlayers: Optional[torch.Tensor] = None


class TransitSpectrum(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta: torch.Tensor, model: BatchModel):
        binned, status = T.forward_transit_batch(model.ctx, model.tables, model.spec,
                                                 theta.contiguous(), model.nlayers, model.bins)
        fctx.save_for_backward(theta)
        fctx.model = model
        fctx.mark_non_differentiable(status)
        return binned, status

    @staticmethod
    def backward(fctx, grad_binned, grad_status):
        (theta,) = fctx.saved_tensors
        m = fctx.model
        _, grad, _, _ = T.adjoint_transit(m.ctx, m.tables, m.spec, theta.contiguous(), m.nlayers,
                                          m.bins, gbin=grad_binned.contiguous().double(),
                                          want_binned=False)
        return grad, None


def spectrum(theta: torch.Tensor, model: BatchModel):
    """Differentiable binned spectra and per-item status."""
    return TransitSpectrum.apply(theta, model)


def chi2_and_grad(theta: torch.Tensor, model: BatchModel, obs: torch.Tensor,
                  sigma_obs: torch.Tensor):
    """chi^2 [B] and d chi^2 / d theta [B][n_theta] in one adjoint call (no autograd tape)."""
    chi2, grad, binned, status = T.adjoint_transit(model.ctx, model.tables, model.spec,
                                                   theta.contiguous(), model.nlayers, model.bins,
                                                   obs=obs, sigma_obs=sigma_obs)
    return chi2, grad, binned, status
