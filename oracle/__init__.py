"""FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package; the product path never does.  It wraps the plain
C implementation in ``oracle.c`` (built with gcc, OpenMP over independent
pixels or edges) and converts every input to float64 exactly, so that the
oracle consumes the same stored values as the GPU path (dequantised).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Dict, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
# ORC_MUTANT=<NAME> selects a copy of the oracle with one planted mistake
# (oracle.c, ORC_MUTANT_<NAME>); only the mutation tests set it
_MUTANT = os.environ.get("ORC_MUTANT", "")
_SO = os.path.join(_BUILD, f"liboracle_mutant_{_MUTANT.lower()}.so" if _MUTANT else "liboracle.so")
_lib = None

DEFAULT_PARAMS: Dict = dict(
    sigma_ray=0.01, sigma_dist=0.1, huber_delta=1.345, q_min=1.5,
    lm_lambda=1e-8, lm_iters=10, win_radius=3, n_levels=2, win_dilation=(2, 1, 1, 1),
    max_rel_dist3d=0.1, conv_tol=1e-10,
    residual=0, sigma_point=0.05, sigma_pixel=1.0, sigma_depth=0.1, fx=0.0, fy=0.0, cx=0.0, cy=0.0, img_w=0,
)

RES_RAY, RES_POINT, RES_PIXEL = 0, 1, 2


class _Params(C.Structure):
    _fields_ = [
        ("sigma_ray", C.c_double), ("sigma_dist", C.c_double), ("huber_delta", C.c_double),
        ("q_min", C.c_double), ("lm_lambda", C.c_double), ("lm_iters", C.c_int),
        ("win_radius", C.c_int), ("n_levels", C.c_int), ("win_dilation", C.c_int * 4),
        ("max_rel_dist3d", C.c_double), ("conv_tol", C.c_double),
        ("residual", C.c_int), ("sigma_point", C.c_double), ("sigma_pixel", C.c_double),
        ("sigma_depth", C.c_double), ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double),
        ("cy", C.c_double), ("img_w", C.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (C11, OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, src, "-lm"] + ([f"-DORC_MUTANT_{_MUTANT}"] if _MUTANT else [])
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        lp = C.POINTER(C.c_int64)
        pp = C.POINTER(_Params)
        for name, args, res in [
            ("orc_sim3_exp", [dp, dp], None), ("orc_sim3_log", [dp, dp], None),
            ("orc_sim3_mul", [dp, dp, dp], None), ("orc_sim3_inv", [dp, dp], None),
            ("orc_sim3_act", [dp, dp, dp], None), ("orc_sim3_matrix", [dp, dp], None),
            ("orc_sim3_adjoint", [dp, dp], None), ("orc_sim3_retract", [dp, dp], None),
            ("orc_ray_image", [dp, C.c_int64, dp], None),
            ("orc_match", [pp, C.c_int, C.c_int, C.c_int, dp, dp, dp, dp, dp, dp, ip, lp, C.c_int64, ip, dp, dp],
             None),
            ("orc_residual_jacobian", [dp, dp, dp, dp, dp, dp], C.c_int),
            ("orc_residual_jacobian_p", [pp, dp, dp, dp, dp, C.c_int32, dp, dp], C.c_int),
            ("orc_linearize_edge", [pp, dp, dp, C.c_int64, dp, dp, ip, dp, dp, dp, dp, lp], None),
            ("orc_gn_solve", [C.c_int, C.c_int, ip, dp, dp, C.c_int, dp, dp], C.c_int),
            ("orc_gauss_newton", [pp, C.c_int, C.c_int, ip, lp, lp, dp, ip, dp, C.c_int, C.c_int, dp, dp,
                                  C.POINTER(C.c_int)], C.c_int),
            ("orc_cost_grad", [pp, C.c_int, C.c_int, ip, lp, lp, dp, dp, ip, dp, dp, dp, dp], None),
            ("orc_gn_step_grad", [pp, C.c_int, C.c_int, ip, lp, lp, dp, dp, ip, dp, dp, C.c_double, dp, dp, dp],
             C.c_int),
            ("orc_fuse", [dp, C.c_int64, dp, dp, dp, dp], None),
            ("orc_match_stats", [C.c_int64, C.c_int64, ip, lp, lp], None),
            ("orc_calib_backproject", [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, dp],
             None),
            ("orc_num_threads", [], C.c_int),
        ]:
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def params(**over) -> _Params:
    p = dict(DEFAULT_PARAMS)
    p.update(over)
    s = _Params()
    for k, v in p.items():
        if k == "win_dilation":
            dil = list(v) + [1] * (4 - len(v))
            s.win_dilation = (C.c_int * 4)(*dil[:4])
        else:
            setattr(s, k, v)
    return s


def _d(a) -> np.ndarray:
    """Exact float64 copy of a torch tensor or array (dequantises fp16/fp32)."""
    try:
        import torch
        if torch.is_tensor(a):
            a = a.detach().to("cpu").to(torch.float64).numpy()
    except ImportError:  # pragma: no cover
        pass
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a) -> np.ndarray:
    try:
        import torch
        if torch.is_tensor(a):
            a = a.detach().to("cpu").numpy()
    except ImportError:  # pragma: no cover
        pass
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _i64(a) -> np.ndarray:
    try:
        import torch
        if torch.is_tensor(a):
            a = a.detach().to("cpu").numpy()
    except ImportError:  # pragma: no cover
        pass
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


# ---------------------------------------------------------------- Sim(3)

def sim3_exp(tau) -> np.ndarray:
    tau = _d(tau).reshape(7)
    T = np.zeros(8)
    lib().orc_sim3_exp(_p(tau), _p(T))
    return T


def sim3_log(T) -> np.ndarray:
    T = _d(T).reshape(8)
    tau = np.zeros(7)
    lib().orc_sim3_log(_p(T), _p(tau))
    return tau


def sim3_mul(A, B) -> np.ndarray:
    A, B = _d(A).reshape(8), _d(B).reshape(8)
    out = np.zeros(8)
    lib().orc_sim3_mul(_p(A), _p(B), _p(out))
    return out


def sim3_inv(A) -> np.ndarray:
    A = _d(A).reshape(8)
    out = np.zeros(8)
    lib().orc_sim3_inv(_p(A), _p(out))
    return out


def sim3_act(T, x) -> np.ndarray:
    T, x = _d(T).reshape(8), _d(x).reshape(3)
    y = np.zeros(3)
    lib().orc_sim3_act(_p(T), _p(x), _p(y))
    return y


def sim3_matrix(T) -> np.ndarray:
    T = _d(T).reshape(8)
    M = np.zeros(16)
    lib().orc_sim3_matrix(_p(T), _p(M))
    return M.reshape(4, 4)


def sim3_adjoint(T) -> np.ndarray:
    T = _d(T).reshape(8)
    Ad = np.zeros(49)
    lib().orc_sim3_adjoint(_p(T), _p(Ad))
    return Ad.reshape(7, 7)


def sim3_retract(tau, T) -> np.ndarray:
    tau, T = _d(tau).reshape(7), _d(T).reshape(8).copy()
    lib().orc_sim3_retract(_p(tau), _p(T))
    return T


def ray_image(X) -> np.ndarray:
    X = _d(X).reshape(-1, 3)
    R = np.zeros_like(X)
    lib().orc_ray_image(_p(X), X.shape[0], _p(R))
    return R


# ---------------------------------------------------------------- matching

def match(H: int, W: int, X_ref, X_qry, D_ref, D_qry, Q_ref, Q_qry, init_idx=None, pix=None,
          diag: bool = False, **par):
    """Projective matching plus refinement for one edge.  Returns (idx int32,
    q float64[, diag [n, 9]]) for the query pixels `pix` (all if None)."""
    Xr, Xq = _d(X_ref).reshape(-1, 3), _d(X_qry).reshape(-1, 3)
    Dr, Dq = _d(D_ref), _d(D_qry)
    d = Dr.shape[-1]
    Dr, Dq = Dr.reshape(-1, d), Dq.reshape(-1, d)
    Qr, Qq = _d(Q_ref).reshape(-1), _d(Q_qry).reshape(-1)
    n = H * W if pix is None else len(pix)
    idx = np.zeros(n, dtype=np.int32)
    q = np.zeros(n)
    dg = np.zeros((n, 9)) if diag else None
    ini = _i32(init_idx) if init_idx is not None else None
    px = _i64(pix) if pix is not None else None
    lib().orc_match(C.byref(params(**par)), H, W, d, _p(Xr), _p(Xq), _p(Dr), _p(Dq), _p(Qr), _p(Qq),
                    _p(ini, C.c_int32) if ini is not None else None,
                    _p(px, C.c_int64) if px is not None else None, n,
                    _p(idx, C.c_int32), _p(q), _p(dg) if dg is not None else None)
    return (idx, q, dg) if diag else (idx, q)


def match_workload(w, e: int, pix=None, diag=False, init_idx=None, **par):
    sl = w.edge_slice(e)
    H, W = int(w.kf_hw[w.edges[e, 1], 0]), int(w.kf_hw[w.edges[e, 1], 1])
    return match(H, W, w.X_ref[sl], w.X_qry[sl], w.D_ref[sl], w.D_qry[sl], w.Q_ref[sl], w.Q_qry[sl],
                 init_idx=init_idx, pix=pix, diag=diag, **par)


# ---------------------------------------------------------------- Gauss-Newton

def residual_jacobian(Ti, Tj, Xj_n, Xi_m):
    Ti, Tj, a, b = _d(Ti).reshape(8), _d(Tj).reshape(8), _d(Xj_n).reshape(3), _d(Xi_m).reshape(3)
    r = np.zeros(4)
    J = np.zeros(56)
    ok = lib().orc_residual_jacobian(_p(Ti), _p(Tj), _p(a), _p(b), _p(r), _p(J))
    return bool(ok), r, J.reshape(4, 14)


def residual_jacobian_p(Ti, Tj, Xj_n, Xi_m, m=0, **par):
    """Any residual family (par["residual"]): (rows, r [rows], J [rows, 14]);
    rows = 0 for a degenerate match."""
    Ti, Tj, a, b = _d(Ti).reshape(8), _d(Tj).reshape(8), _d(Xj_n).reshape(3), _d(Xi_m).reshape(3)
    r = np.zeros(4)
    J = np.zeros(56)
    rows = lib().orc_residual_jacobian_p(C.byref(params(**par)), _p(Ti), _p(Tj), _p(a), _p(b), int(m), _p(r),
                                         _p(J))
    return rows, r[:rows], J.reshape(4, 14)[:rows]


def linearize_edge(Ti, Tj, X_i, X_j, idx, q, **par):
    Ti, Tj = _d(Ti).reshape(8), _d(Tj).reshape(8)
    Xi, Xj = _d(X_i).reshape(-1, 3), _d(X_j).reshape(-1, 3)
    idx = _i32(idx).reshape(-1)
    q = _d(q).reshape(-1)
    H = np.zeros(196)
    g = np.zeros(14)
    c = np.zeros(1)
    nv = np.zeros(1, dtype=np.int64)
    lib().orc_linearize_edge(C.byref(params(**par)), _p(Ti), _p(Tj), idx.shape[0], _p(Xi), _p(Xj),
                             _p(idx, C.c_int32), _p(q), _p(H), _p(g), _p(c), _p(nv, C.c_int64))
    return H.reshape(14, 14), g, float(c[0]), int(nv[0])


def gn_solve(N, edges, H14, g14, T, gauge=0):
    edges = _i32(edges).reshape(-1, 2)
    H14 = _d(H14).reshape(-1, 196)
    g14 = _d(g14).reshape(-1, 14)
    T = _d(T).reshape(N, 8).copy()
    tau = np.zeros((N, 7))
    st = lib().orc_gn_solve(N, edges.shape[0], _p(edges, C.c_int32), _p(H14), _p(g14), gauge, _p(T), _p(tau))
    return st, T, tau


def gauss_newton(N, edges, kf_off, e_off, X_canon, idx, q, T, iters, gauge=0, **par):
    edges = _i32(edges).reshape(-1, 2)
    kf_off, e_off = _i64(kf_off), _i64(e_off)
    X = _d(X_canon).reshape(-1, 3)
    idx = _i32(idx).reshape(-1)
    q = _d(q).reshape(-1)
    T = _d(T).reshape(N, 8).copy()
    hist = np.zeros(max(iters, 1))
    done = C.c_int(0)
    st = lib().orc_gauss_newton(C.byref(params(**par)), N, edges.shape[0], _p(edges, C.c_int32),
                                _p(kf_off, C.c_int64), _p(e_off, C.c_int64), _p(X), _p(idx, C.c_int32), _p(q),
                                iters, gauge, _p(T), _p(hist), C.byref(done))
    return st, T, hist[:done.value], done.value


def cost_grad(N, edges, kf_off, e_off, T, X_canon, idx, q, **par):
    edges = _i32(edges).reshape(-1, 2)
    kf_off, e_off = _i64(kf_off), _i64(e_off)
    X = _d(X_canon).reshape(-1, 3)
    idx = _i32(idx).reshape(-1)
    q = _d(q).reshape(-1)
    T = _d(T).reshape(N, 8)
    dX = np.zeros_like(X)
    dq = np.zeros_like(q)
    c = np.zeros(1)
    lib().orc_cost_grad(C.byref(params(**par)), N, edges.shape[0], _p(edges, C.c_int32), _p(kf_off, C.c_int64),
                        _p(e_off, C.c_int64), _p(T), _p(X), _p(idx, C.c_int32), _p(q), _p(dX), _p(dq), _p(c))
    return float(c[0]), dX, dq


def gn_step_grad(N, edges, kf_off, e_off, T, X_canon, idx, q, dL_dtau=None, dL_dcost=1.0, **par):
    """Gradient of dL_dcost * E + dL_dtau . tau (one GN step) w.r.t. X_canon
    and q.  Returns (status, dX [P, 3], dq [P_e], tau [N, 7])."""
    edges = _i32(edges).reshape(-1, 2)
    kf_off, e_off = _i64(kf_off), _i64(e_off)
    X = _d(X_canon).reshape(-1, 3)
    idx = _i32(idx).reshape(-1)
    q = _d(q).reshape(-1)
    T = _d(T).reshape(N, 8)
    a = None if dL_dtau is None else _d(dL_dtau).reshape(N * 7)
    dX = np.zeros_like(X)
    dq = np.zeros_like(q)
    tau = np.zeros((N, 7))
    st = lib().orc_gn_step_grad(C.byref(params(**par)), N, edges.shape[0], _p(edges, C.c_int32),
                                _p(kf_off, C.c_int64), _p(e_off, C.c_int64), _p(T), _p(X), _p(idx, C.c_int32), _p(q),
                                _p(a) if a is not None else None, float(dL_dcost), _p(dX), _p(dq), _p(tau))
    return st, dX, dq, tau


def fuse(T_kf, X_canon, C_canon, X_kf, C_kf):
    """Pointmap fusion (Sec. 3.3); returns the updated (X_canon, C_canon)."""
    T = _d(T_kf).reshape(8)
    X = _d(X_canon).reshape(-1, 3).copy()
    Cc = _d(C_canon).reshape(-1).copy()
    Xk = _d(X_kf).reshape(-1, 3)
    Ck = _d(C_kf).reshape(-1)
    lib().orc_fuse(_p(T), X.shape[0], _p(X), _p(Cc), _p(Xk), _p(Ck))
    return X, Cc


def match_stats(idx, n_ref: int):
    """(valid matches, distinct reference pixels) of one edge (Sec. 3.4)."""
    idx = _i32(idx).reshape(-1)
    v = np.zeros(1, dtype=np.int64)
    u = np.zeros(1, dtype=np.int64)
    lib().orc_match_stats(idx.shape[0], int(n_ref), _p(idx, C.c_int32), _p(v, C.c_int64), _p(u, C.c_int64))
    return int(v[0]), int(u[0])


def num_threads() -> int:
    return int(lib().orc_num_threads())


def calib_backproject(H, W, fx, fy, cx, cy, X):
    """Sec. 3.6: keep the depth, rebuild each point on its pixel's pinhole ray."""
    X = _d(X).reshape(H * W, 3).copy()
    lib().orc_calib_backproject(H, W, fx, fy, cx, cy, _p(X))
    return X
