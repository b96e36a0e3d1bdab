"""torch.autograd.Function over the batched forward model and its hand-written adjoint.

TransitSpectrum.apply(theta, model) returns the binned transit depths [B][n_bin] of the
parameter vectors theta [B][n_theta] (float64, CUDA); its backward calls tr_adjoint_transit in
vector-Jacobian-product mode with the upstream gradient.  That backward call does not repeat
the forward's optical-depth contraction and binning: it rebuilds the geometry and the opacity
K (the quantities the reverse pass needs) and runs the backward kernels.  Both directions run
in the library's CUDA kernels.

jacobian() returns dD_bin/dtheta of every item from one library call, and fisher_matrix()
turns it into the Fisher information of a Gaussian likelihood with per-bin uncertainties.
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
    precision: int = T.TR_PREC_FP32


class TransitSpectrum(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta: torch.Tensor, model: BatchModel):
        binned, status = T.forward_transit_batch(model.ctx, model.tables, model.spec,
                                                 theta.contiguous(), model.nlayers, model.bins,
                                                 precision=model.precision)
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
                                          precision=m.precision, want_binned=False)
        return grad, None


def spectrum(theta: torch.Tensor, model: BatchModel):
    """Differentiable binned spectra and per-item status."""
    return TransitSpectrum.apply(theta, model)


def chi2_and_grad(theta: torch.Tensor, model: BatchModel, obs: torch.Tensor,
                  sigma_obs: torch.Tensor):
    """chi^2 [B] and d chi^2 / d theta [B][n_theta] in one adjoint call (no autograd tape)."""
    chi2, grad, binned, status = T.adjoint_transit(model.ctx, model.tables, model.spec,
                                                   theta.contiguous(), model.nlayers, model.bins,
                                                   obs=obs, sigma_obs=sigma_obs,
                                                   precision=model.precision)
    return chi2, grad, binned, status


def jacobian(theta: torch.Tensor, model: BatchModel):
    """(binned [B][n_bin], jac [B][n_bin][n_theta] = dD_bin/dtheta, status [B]) from one
    tr_adjoint_transit call (one forward, then one backward pass per bin over that bin's
    wavenumbers)."""
    _, _, binned, status, jac = T.adjoint_transit(model.ctx, model.tables, model.spec,
                                                  theta.contiguous(), model.nlayers, model.bins,
                                                  precision=model.precision, want_grad=False,
                                                  want_jac=True)
    return binned, jac, status


def fisher_matrix(theta: torch.Tensor, model: BatchModel, sigma_obs: torch.Tensor):
    """Fisher information F[b] = J_b^T diag(1/sigma^2) J_b [B][n_theta][n_theta] of the
    Gaussian likelihood of binned depths with uncertainties sigma_obs [n_bin] (or
    [B][n_bin]), from the library's Jacobian; also returns the per-item status.  The small
    J^T W J product is plain post-processing of the Jacobian the kernels computed."""
    _, jac, status = jacobian(theta, model)
    w = 1.0 / sigma_obs.to(jac.dtype) ** 2
    if w.dim() == 1:
        w = w.expand(jac.shape[0], -1)
    fisher = torch.einsum("bjk,bj,bjl->bkl", jac, w, jac)
    return fisher, status
