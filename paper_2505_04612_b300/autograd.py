"""The direct epipolar objective as a ``torch.autograd.Function``.

Forward evaluates L = (1/Z) sum_m w_m rho(x~2_m^T E_n x~1_m) (Sec. 3.3, Eq. 7
for rho = |r|; Eqs. 8-9 for rho = r^2 with IRLS weights) at the epipolar-stage
parameters [N, 9] (6D rotation, translation per camera); backward is the
library's hand-written adjoint: dL/dE_n per image pair, the chain rule
through E_n = [t^_ij]_x R_j R_i^T to both cameras, the fixed-order
per-camera sum and the 6D map's adjoint.  Both passes run in the C ABI
(``fm_ea_forward`` / ``fm_ea_backward``); this module only allocates the
outputs and passes pointers.

Modes (what forward keeps for backward):
  ``"recompute"``  nothing; backward re-reads every keypoint pair and
                   recomputes its residual (16 B per pair again);
  ``"stored"``     the per-pair coefficient w rho'(r) (4 B per pair written,
                   then 4 + 16 B per pair read by backward);
  ``"fused"``      dL/dE_n per image pair (9 floats): forward does all the
                   per-pair work, backward only the per-image-pair and
                   per-camera parts.

The problem's loss (L1 or L2) and weights are the ones set on it; they must
not change between a forward call and its backward call.  The problem is
bound to the CUDA stream it was created on, which should be the stream torch
runs the surrounding graph on.
"""
from __future__ import annotations

import torch

from . import fastmap as F

MODES = {"recompute": F.FM_EA_SAVE_NONE, "stored": F.FM_EA_SAVE_COEF, "fused": F.FM_EA_SAVE_DLDE}


def _saved_buffer(problem, save, device):
    if save == F.FM_EA_SAVE_COEF:
        return torch.empty(max(problem.n_kp, 1), dtype=torch.float32, device=device)
    if save == F.FM_EA_SAVE_DLDE:
        return torch.empty(max(problem.n_pairs, 1) * 9, dtype=torch.float32, device=device)
    return None


class EpipolarLoss(torch.autograd.Function):
    """loss = EpipolarLoss.apply(params [N, 9] CUDA float32, problem, mode)."""

    @staticmethod
    def forward(ctx, params, problem, mode="recompute"):
        if mode not in MODES:
            raise ValueError(f"mode must be one of {sorted(MODES)}")
        if not (params.is_cuda and params.dtype == torch.float32 and params.is_contiguous()):
            raise ValueError("params must be a contiguous float32 CUDA tensor")
        if params.numel() != 9 * problem.n_cams:
            raise ValueError(f"params must hold {9 * problem.n_cams} values")
        save = MODES[mode]
        # one loss per scene of a batched problem; a scalar for one scene
        S = getattr(problem, "S", 1)
        loss = torch.empty(() if S == 1 else (S,), dtype=torch.float32, device=params.device)
        saved = _saved_buffer(problem, save, params.device)
        F.fm_ea_forward(problem.handle, params.data_ptr(), loss.data_ptr(), save,
                        saved.data_ptr() if saved is not None else None)
        ctx.problem = problem
        ctx.save = save
        ctx.save_for_backward(params, saved)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        params, saved = ctx.saved_tensors
        g = grad_loss.detach()
        if g.dtype != torch.float32:
            g = g.float()
        g = g.contiguous()
        grad = torch.empty_like(params)
        F.fm_ea_backward(ctx.problem.handle, params.data_ptr(), ctx.save,
                         saved.data_ptr() if saved is not None else None, g.data_ptr(), grad.data_ptr())
        return grad, None, None


def epipolar_loss(params, problem, mode="recompute"):
    """The epipolar loss of `problem` at `params` with the hand-written adjoint."""
    return EpipolarLoss.apply(params, problem, mode)


class EpipolarFocalLoss(torch.autograd.Function):
    """loss = EpipolarFocalLoss.apply(params [N, 9], phi [N], problem): the
    direct epipolar objective with the focal lengths folded into the
    matrices (Sec. 3.3, last paragraph of "Epipolar Adjustment"):
    E'_n = S_j E_n S_i with S_c = diag(e^-phi_c, e^-phi_c, 1), phi_c the log
    ratio of camera c's focal length to the one its keypoints were calibrated
    at.  Forward keeps dL/dE'_n per image pair (``fm_ea_focal_forward``);
    backward returns the poses' and the focal ratios' gradients
    (``fm_ea_focal_backward``)."""

    @staticmethod
    def forward(ctx, params, phi, problem):
        for name, t, n in (("params", params, 9 * problem.n_cams), ("phi", phi, problem.n_cams)):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
            if t.numel() != n:
                raise ValueError(f"{name} must hold {n} values")
        S = getattr(problem, "S", 1)
        loss = torch.empty(() if S == 1 else (S,), dtype=torch.float32, device=params.device)
        saved = _saved_buffer(problem, F.FM_EA_SAVE_DLDE, params.device)
        F._check(F.lib().fm_ea_focal_forward(problem.handle, params.data_ptr(), phi.data_ptr(), loss.data_ptr(),
                                             saved.data_ptr()), problem.handle)
        ctx.problem = problem
        ctx.save_for_backward(params, phi, saved)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        params, phi, saved = ctx.saved_tensors
        g = grad_loss.detach().float().contiguous()
        grad = torch.empty_like(params)
        gphi = torch.empty_like(phi)
        F._check(F.lib().fm_ea_focal_backward(ctx.problem.handle, params.data_ptr(), phi.data_ptr(),
                                              saved.data_ptr(), g.data_ptr(), grad.data_ptr(), gphi.data_ptr()),
                 ctx.problem.handle)
        return grad, gphi, None


def epipolar_focal_loss(params, phi, problem):
    """The epipolar loss of `problem` at `params` with free log focal ratios
    `phi` (hand-written adjoint for both)."""
    return EpipolarFocalLoss.apply(params, phi, problem)
