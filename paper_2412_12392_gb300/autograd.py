"""torch.autograd.Function around one whole Gauss-Newton step (project form:
the paper has no backward pass).

GNStep.apply(X_canon, q, T_wc, plan, params, idx) returns (T_new [N, 8]
FP64, tau [N, 7] FP64, cost scalar FP64): tau = -H^-1 g is the gauge-fixed
Gauss-Newton step at the poses T_wc (Eq. gauss_newton), T_new = Exp(tau) o
T_wc its retraction (Eq. 1) and cost the ray-error cost E_g at T_wc (Eq.
backend_ray).  Its backward calls mslam_gn_step_backward, which recomputes
the per-pixel residuals and Jacobians (nothing per pixel is stored) and
returns the gradients with respect to the canonical pointmaps, the match
confidences and the poses, so that steps chain: unrolled steps are
successive applications on the previous step's T_new.  Matches and the q_min
mask are not differentiated.  Pose gradients live in the [N, 8] embedding
(no component along the quaternion's norm).  A step whose system is not
positive definite, or whose step is not finite, raises.
"""
from __future__ import annotations

import torch

from . import _lib, api


def _check_status(status: torch.Tensor, what: str):
    bad = status[(status != 0) & (status != 1)]
    if bad.numel():
        code = int(bad[0])
        raise _lib.MslamError(code, f"{what}: a graph returned {_lib.STATUS_NAMES.get(code, code)}")


class GNStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X_canon, q, T_wc, plan, params, idx):
        H, g, cost, _ = api.gn_linearize(plan, params, T_wc, X_canon, idx, q)
        T_new = T_wc.detach().clone()
        tau = torch.zeros(plan.N, 7, dtype=torch.float64, device=X_canon.device)
        status = torch.zeros(plan.G, dtype=torch.int32, device=X_canon.device)
        api.gn_solve(plan, params, H, g, T_new, tau, status)
        _check_status(status, "GNStep forward")
        ctx.plan, ctx.params = plan, params
        ctx.save_for_backward(X_canon, q, T_wc, idx, H, g)
        return T_new, tau, cost.sum()

    @staticmethod
    def backward(ctx, dT_new, dtau, dcost):
        X_canon, q, T_wc, idx, H, g = ctx.saved_tensors
        a = None if dtau is None else dtau.to(torch.float64).contiguous()
        gT = None if dT_new is None else dT_new.to(torch.float64).contiguous()
        c = 0.0 if dcost is None else float(dcost)
        dX, dq, dT, status = api.gn_step_backward(ctx.plan, ctx.params, T_wc.detach(), X_canon.detach(), idx,
                                                  q.detach(), H, g, dL_dTnew=gT, dL_dtau=a, dL_dcost=c)
        _check_status(status, "GNStep backward")
        return dX.view_as(X_canon).to(X_canon.dtype), dq.to(q.dtype), dT, None, None, None


def gn_step(X_canon, q, T_wc, plan, params, idx):
    """Functional form of GNStep: (T_new, tau, cost)."""
    return GNStep.apply(X_canon, q, T_wc, plan, params, idx)


def gn_unrolled(X_canon, q, T_wc, plan, params, idx, steps: int):
    """`steps` chained Gauss-Newton steps from T_wc; returns (T_final, [tau
    of each step], [cost at the start of each step])."""
    taus, costs = [], []
    T = T_wc
    for _ in range(steps):
        T, tau, cost = gn_step(X_canon, q, T, plan, params, idx)
        taus.append(tau)
        costs.append(cost)
    return T, taus, costs
