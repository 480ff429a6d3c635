"""Comparison helpers for the GPU-vs-oracle parity tests.

Tolerances (from the stated bars of the method's hot path):
* matched indices agree on >= 99.9 % of the pixels valid on either side;
  a disagreement is a decision the kernel takes in FP32 and the oracle in
  FP64 (the rounding of p*, the window argmax, the 3D threshold): those
  that are not within FP32 reach of a tie are counted separately and capped
  (``classify_disagreements``);
* Hessian and gradient blocks: |X_gpu - X_ref|_F / |X_ref|_F <= 1e-5 per edge;
* poses: rotation error <= 1e-5 rad, translation error <= 1e-5 relative
  to max(|t_ref|, 0.1 m), scale error <= 1e-5 relative.  The floor: the
  FP32 rounding of the normal equations moves a pose by an amount set by the
  scene's metric scale (depths of 1-9 m), not by the pose's distance from
  the fixed keyframe, which is as small as 0.05 m on the largest loop graph;
  below 0.1 m the bar is an absolute 1e-6 m.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle

MATCH_AGREE = 0.999
# disagreements explained only by an LM iterate the oracle had not converged
# (last step above 1e-3 px after the 10 iterations) may make up at most this
# fraction of the pixels valid on either side -- the whole budget of the
# 99.9 % bar, never more -- and those explained by nothing at most
# UNEXPLAINED_MAX
MOVING_MAX = 1e-3
UNEXPLAINED_MAX = 1e-4
T_FLOOR = 0.1
BLOCK_RTOL = 1e-5
POSE_TOL = 1e-5


def f64(t) -> np.ndarray:
    if torch.is_tensor(t):
        return t.detach().cpu().to(torch.float64).numpy()
    return np.asarray(t, dtype=np.float64)


def pose_errors(T_gpu, T_ref):
    """(rotation rad, relative translation, relative scale) per pose."""
    Tg, Tr = f64(T_gpu).reshape(-1, 8), f64(T_ref).reshape(-1, 8)
    out = []
    for a, b in zip(Tg, Tr):
        d = oracle.sim3_mul(a, oracle.sim3_inv(b))
        rot = 2.0 * np.arcsin(min(1.0, np.linalg.norm(d[3:6])))
        tr = np.linalg.norm(a[:3] - b[:3]) / max(np.linalg.norm(b[:3]), T_FLOOR)
        sc = abs(a[7] - b[7]) / abs(b[7])
        out.append((rot, tr, sc))
    return np.array(out)


def assert_poses_close(T_gpu, T_ref, tol=POSE_TOL):
    e = pose_errors(T_gpu, T_ref)
    assert e.max() <= tol, f"pose errors (rot, trans, scale) max {e.max(axis=0)}"
    return e


def block_rel_err(A_gpu, A_ref):
    A, B = f64(A_gpu), f64(A_ref)
    A = A.reshape(A.shape[0], -1)
    B = B.reshape(B.shape[0], -1)
    return np.linalg.norm(A - B, axis=1) / np.maximum(np.linalg.norm(B, axis=1), 1e-300)


def classify_disagreements(idx_gpu, idx_ref, diag_ref, params=None):
    """Counts over the pixels valid on either side: (union, disagreements,
    near ties, LM iterates still moving, unexplained).  A near tie is a
    decision within FP32 reach of its boundary in the oracle's FP64 run:
    p* within 2e-3 px of a rounding boundary, a window argmax margin below
    1e-4, or the 3D ratio within 1e-4 of its threshold.  "Moving" counts the
    other disagreements whose oracle LM step was still above 1e-3 px after
    the last iteration; the rest are unexplained."""
    g, r = f64(idx_gpu).astype(np.int64), f64(idx_ref).astype(np.int64)
    union = (g >= 0) | (r >= 0)
    dis = union & (g != r)
    n_union, n_dis = int(union.sum()), int(dis.sum())
    if n_dis == 0:
        return dict(union=n_union, dis=0, ties=0, moving=0, unexplained=0)
    d = diag_ref[dis]
    thr = params["max_rel_dist3d"] if params else 0.1
    tie = (d[:, 5] < 2e-3) | (d[:, 3] < 1e-4) | (d[:, 4] < 1e-4) | (np.abs(d[:, 6] - thr) < 1e-4)
    moving = ~tie & (d[:, 2] > 1e-3)
    return dict(union=n_union, dis=n_dis, ties=int(tie.sum()), moving=int(moving.sum()),
                unexplained=int((~tie & ~moving).sum()))


def check_disagreements(c: dict, what: str = ""):
    """The match bars on counts from classify_disagreements (possibly summed
    over several edges): all-pixel agreement >= MATCH_AGREE, the
    moving-iterate share <= MOVING_MAX and the unexplained share <=
    UNEXPLAINED_MAX of the union."""
    u = max(c["union"], 1)
    msg = (f"{what} agree {1 - c['dis'] / u:.6f} ({c['dis']} of {c['union']}: {c['ties']} near ties, "
           f"{c['moving']} moving iterates ({c['moving'] / u:.2e}), {c['unexplained']} unexplained)")
    print(msg)
    assert 1 - c["dis"] / u >= MATCH_AGREE, msg
    assert c["moving"] / u <= MOVING_MAX, msg
    assert c["unexplained"] / u <= UNEXPLAINED_MAX, msg
    return msg


def add_counts(a: dict, b: dict) -> dict:
    return {k: a.get(k, 0) + b[k] for k in b}


def match_agreement(idx_gpu, idx_ref, diag_ref=None, params=None):
    """(agreement over the union of valid pixels, disagreements, union size,
    fraction of disagreements that are near ties)."""
    g, r = f64(idx_gpu).astype(np.int64), f64(idx_ref).astype(np.int64)
    union = (g >= 0) | (r >= 0)
    dis = union & (g != r)
    agree = 1.0 - dis.sum() / max(union.sum(), 1)
    explained = 1.0
    if diag_ref is not None and dis.any():
        c = classify_disagreements(idx_gpu, idx_ref, diag_ref, params)
        explained = c["ties"] / c["dis"]
    return agree, int(dis.sum()), int(union.sum()), explained


def solve_flags(plan, ws):
    """Per-graph flags the mixed-precision solve leaves at the end of the
    solve workspace: 1 = solved by FP32 factorisation + FP64 refinement,
    0 = left to the FP64 kernel."""
    import torch
    n = 4 * plan.G
    off = ws.numel() - ((n + 255) // 256) * 256
    return ws[off:off + n].view(torch.int32).cpu()
