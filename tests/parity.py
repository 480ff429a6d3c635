"""Comparison helpers for the GPU-vs-oracle parity tests.

Tolerances (from the stated bars of the method's hot path):
* matched indices agree on >= 99.9 % of the pixels valid on either side;
* Hessian and gradient blocks: |X_gpu - X_ref|_F / |X_ref|_F <= 1e-5 per edge;
* poses: rotation error <= 1e-5 rad, translation error <= 1e-5 relative
  (to max(|t_ref|, 0.1 m)), scale error <= 1e-5 relative.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle

MATCH_AGREE = 0.999
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
        tr = np.linalg.norm(a[:3] - b[:3]) / max(np.linalg.norm(b[:3]), 0.1)
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


def match_agreement(idx_gpu, idx_ref, diag_ref=None, params=None):
    """Fraction of agreeing indices over the union of valid pixels, and the
    fraction of disagreements explained by a near tie of a decision the
    kernel takes in FP32 (rounding of p*, window argmax, 3D threshold) or by
    an LM iterate the oracle had not converged."""
    g, r = f64(idx_gpu).astype(np.int64), f64(idx_ref).astype(np.int64)
    union = (g >= 0) | (r >= 0)
    dis = union & (g != r)
    agree = 1.0 - dis.sum() / max(union.sum(), 1)
    explained = 1.0
    if diag_ref is not None and dis.any():
        d = diag_ref[dis]
        thr = params["max_rel_dist3d"] if params else 0.1
        ok = (d[:, 5] < 2e-3) | (d[:, 3] < 1e-4) | (d[:, 4] < 1e-4) | (np.abs(d[:, 6] - thr) < 1e-4) | (d[:, 2] > 1e-3)
        explained = ok.mean()
    return agree, int(dis.sum()), int(union.sum()), explained


def match_agreement_unexplained(idx_gpu, idx_ref, diag_ref, params):
    """(agreement over all pixels valid on either side, disagreements,
    disagreements that are not a near tie of an FP32 decision or an LM
    iterate still moving, union size)."""
    agree, ndis, nunion, expl = match_agreement(idx_gpu, idx_ref, diag_ref, params)
    return agree, ndis, int(round(ndis * (1.0 - expl))), nunion


def solve_flags(plan, ws):
    """Per-graph flags the mixed-precision solve leaves at the end of the
    solve workspace: 1 = solved by FP32 factorisation + FP64 refinement,
    0 = left to the FP64 kernel."""
    import torch
    n = 4 * plan.G
    off = ws.numel() - ((n + 255) // 256) * 256
    return ws[off:off + n].view(torch.int32).cpu()
