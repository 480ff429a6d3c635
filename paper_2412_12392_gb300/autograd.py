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
    def forward(ctx, X_canon, q, T_wc, plan, params, idx, X_route=None, q_route=None):
        """X_route / q_route (optional, FP32 tensors holding the same values
        as X_canon / q): when given, the gradients are returned for them in
        FP32 instead of for X_canon / q in the storage dtype, so that
        gradients summed over several steps are accumulated in FP32."""
        H, g, cost, _ = api.gn_linearize(plan, params, T_wc, X_canon, idx, q)
        T_new = T_wc.detach().clone()
        tau = torch.zeros(plan.N, 7, dtype=torch.float64, device=X_canon.device)
        status = torch.zeros(plan.G, dtype=torch.int32, device=X_canon.device)
        api.gn_solve(plan, params, H, g, T_new, tau, status)
        _check_status(status, "GNStep forward")
        ctx.plan, ctx.params = plan, params
        ctx.route = (X_route is not None, q_route is not None)
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
        dX = dX.view_as(X_canon)
        rx, rq = ctx.route
        gx, gxr = (None, dX) if rx else (dX.to(X_canon.dtype), None)
        gq, gqr = (None, dq) if rq else (dq.to(q.dtype), None)
        return gx, gq, dT, None, None, None, gxr, gqr


def gn_step(X_canon, q, T_wc, plan, params, idx):
    """Functional form of GNStep: (T_new, tau, cost)."""
    return GNStep.apply(X_canon, q, T_wc, plan, params, idx)


def gn_unrolled(X_canon, q, T_wc, plan, params, idx, steps: int, storage=None):
    """`steps` chained Gauss-Newton steps from T_wc; returns (T_final, [tau
    of each step], [cost at the start of each step]).

    storage (optional dtype, e.g. torch.float16): the kernels read X_canon
    and q rounded to it, and the gradients are returned for X_canon and q in
    their own dtype.  An FP32 caller that stores FP16 keeps FP32 gradients
    this way: the point gradients of a large graph are mostly below 1e-4
    (each point moves the poses by little) and fall into FP16's subnormal
    range, where a rounded FP16 gradient keeps only a few bits.  Without
    `storage`, FP16 tensors that require gradients get the steps' gradients
    summed in FP32 (each step routes them to an FP32 copy) and rounded to
    FP16 once, not once per step."""
    if storage is None:
        storage = X_canon.dtype

    def split(t):
        # (tensor the kernels read, tensor that receives its gradient or None)
        if t.dtype != storage:
            return t.detach().to(storage), (t if t.requires_grad else None)
        if t.requires_grad and t.dtype != torch.float32:
            return t.detach(), t.float()
        return t, None

    (Xs, Xr), (qs, qr) = split(X_canon), split(q)
    taus, costs = [], []
    T = T_wc
    for _ in range(steps):
        T, tau, cost = GNStep.apply(Xs, qs, T, plan, params, idx, Xr, qr)
        taus.append(tau)
        costs.append(cost)
    return T, taus, costs
