"""torch.autograd.Function around one Gauss-Newton step (project form: the
paper has no backward pass).

GNStep.apply(X_canon, q, T_wc, plan, params, idx) returns (tau [N, 7] FP64,
cost scalar FP64): tau = -H^-1 g is the gauge-fixed Gauss-Newton step at the
poses T_wc (Eq. gauss_newton) and cost the ray-error cost E_g (Eq.
backend_ray).  Its backward calls mslam_gn_backward, which recomputes the
per-pixel residuals and Jacobians (nothing per-pixel is stored) and returns
the gradients with respect to the canonical pointmaps and the match
confidences; matches, poses and the q_min mask are not differentiated.  The
gradient of a converged cost follows from the cost output alone (at a
stationary point the step term vanishes).
"""
from __future__ import annotations

import torch

from . import api


class GNStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X_canon, q, T_wc, plan, params, idx):
        H, g, cost, _ = api.gn_linearize(plan, params, T_wc, X_canon, idx, q)
        T_new = T_wc.clone()
        tau = torch.zeros(plan.N, 7, dtype=torch.float64, device=X_canon.device)
        status = torch.zeros(plan.G, dtype=torch.int32, device=X_canon.device)
        api.gn_solve(plan, params, H, g, T_new, tau, status)
        ctx.plan, ctx.params = plan, params
        ctx.save_for_backward(X_canon, q, T_wc, idx, H, g)
        ctx.mark_non_differentiable(status)
        return tau, cost.sum()

    @staticmethod
    def backward(ctx, dtau, dcost):
        X_canon, q, T_wc, idx, H, g = ctx.saved_tensors
        a = None if dtau is None else dtau.to(torch.float64).contiguous()
        c = 0.0 if dcost is None else float(dcost)
        dX, dq, _ = api.gn_backward(ctx.plan, ctx.params, T_wc, X_canon, idx, q, H, g, dL_dtau=a, dL_dcost=c)
        return dX.view_as(X_canon).to(X_canon.dtype), dq.to(q.dtype), None, None, None, None


def gn_step(X_canon, q, T_wc, plan, params, idx):
    """Functional form of GNStep: (tau, cost)."""
    return GNStep.apply(X_canon, q, T_wc, plan, params, idx)
