"""Thin Python binding of include/mslam.h: argument marshalling only.

Every function here checks tensor devices, dtypes and shapes, then calls the
C entry point of the same name on the current CUDA stream; all computation
happens in the CUDA kernels of libmslam.so.  Device memory (outputs and
workspaces) is allocated with torch and handed to the library, which
allocates nothing itself.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

from . import _lib
from ._lib import Params, PlanOpts, check, lib

DTYPES = {torch.float32: _lib.MSLAM_F32, torch.float16: _lib.MSLAM_F16}


def default_params(**over) -> Params:
    """mslam_default_params with optional field overrides."""
    p = Params()
    lib().mslam_default_params(C.byref(p))
    for k, v in over.items():
        if k == "win_dilation":
            dil = list(v) + [1] * (4 - len(v))
            p.win_dilation = (C.c_int32 * 4)(*dil[:4])
        else:
            setattr(p, k, v)
    return p


def params_dict(p: Params) -> dict:
    """The parameter block as a plain dict (for the oracle)."""
    return dict(sigma_ray=p.sigma_ray, sigma_dist=p.sigma_dist, huber_delta=p.huber_delta, q_min=p.q_min,
                lm_lambda=p.lm_lambda, lm_iters=p.lm_iters, win_radius=p.win_radius, n_levels=p.n_levels,
                win_dilation=tuple(p.win_dilation), max_rel_dist3d=p.max_rel_dist3d, conv_tol=p.conv_tol,
                residual=p.residual, sigma_point=p.sigma_point, sigma_pixel=p.sigma_pixel,
                sigma_depth=p.sigma_depth, fx=p.fx, fy=p.fy, cx=p.cx, cy=p.cy)


def _stream(device=None) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else t.data_ptr()


def _need(t: torch.Tensor, name: str, dtype=None, numel=None, device=None):
    if not torch.is_tensor(t):
        raise TypeError(f"{name} must be a torch tensor")
    if t.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor (got {t.device})")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype} (got {t.dtype})")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")


def _workspace(plan: "Plan", op: int, workspace):
    """The caller's workspace for op (a contiguous uint8 CUDA tensor; the
    library checks its size) or a new one."""
    if workspace is None:
        return plan.workspace(op)
    _need(workspace, "workspace", torch.uint8)
    return workspace


class Plan:
    """mslam_plan: the static structure of one or more keyframe graphs,
    uploaded to a torch-owned device buffer."""

    def __init__(self, kf_hw, edges, graph_of_kf=None, device="cuda", opts: Optional[dict] = None):
        kf = np.ascontiguousarray(np.asarray(kf_hw, dtype=np.int32).reshape(-1, 2))
        ed = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
        gk = None if graph_of_kf is None else np.ascontiguousarray(np.asarray(graph_of_kf, dtype=np.int32))
        self.N, self.E = kf.shape[0], ed.shape[0]
        o = PlanOpts()
        lib().mslam_default_plan_opts(C.byref(o))
        for k, v in (opts or {}).items():
            setattr(o, k, int(v))
        self.opts = {k: getattr(o, k) for k in ("lin_tile", "lin_blocks_per_sm", "match_block_w", "lin_form",
                                                   "solve_form", "match_form", "match_ppt", "wait_limit")}
        self.graph_of_kf = gk
        h = C.c_void_p()
        check(lib().mslam_plan_create_ex(self.N, kf.ctypes.data, self.E, ed.ctypes.data if self.E else None,
                                         gk.ctypes.data if gk is not None else None, C.byref(o), C.byref(h)),
              "mslam_plan_create_ex")
        self._h = h
        self.kf_hw, self.edges = kf, ed
        self.kf_pixels = int(lib().mslam_plan_kf_pixels(h))
        self.edge_pixels = int(lib().mslam_plan_edge_pixels(h))
        self.G = int(lib().mslam_plan_num_graphs(h))
        self.kf_off = np.zeros(self.N + 1, dtype=np.int64)
        self.e_off = np.zeros(self.E + 1, dtype=np.int64)
        lib().mslam_plan_offsets(h, self.kf_off.ctypes.data, self.e_off.ctypes.data)
        self.order = np.zeros(self.N, dtype=np.int32)
        self.counts = np.zeros(4, dtype=np.int64)
        lib().mslam_plan_stats(h, self.order.ctypes.data, self.counts.ctypes.data)
        self.device = torch.device(device)
        self.dev = None
        if self.device.type == "cuda":
            self.upload()

    def upload(self):
        nbytes = int(lib().mslam_plan_device_bytes(self._h))
        self.dev = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        check(lib().mslam_plan_upload(self._h, self.dev.data_ptr(), nbytes, _stream(self.device)),
              "mslam_plan_upload")

    @property
    def solve_launches(self) -> int:
        """Kernel launches of one gn_solve call (mslam_gn_solve_launches)."""
        return int(lib().mslam_gn_solve_launches(self._h))

    def workspace_bytes(self, op: int) -> int:
        return int(lib().mslam_workspace_bytes(self._h, op))

    def workspace(self, op: int) -> torch.Tensor:
        return torch.empty(max(self.workspace_bytes(op), 256), dtype=torch.uint8, device=self.device)

    @property
    def handle(self):
        return self._h

    def __del__(self):
        try:
            if getattr(self, "_h", None) and _lib._lib is not None:
                lib().mslam_plan_destroy(self._h)
                self._h = None
        except Exception:  # pragma: no cover - interpreter shutdown
            pass


def chunk_descriptors(D: torch.Tensor, out: Optional[torch.Tensor] = None, p0: int = 0) -> torch.Tensor:
    """[P, d] descriptors -> the chunk-planar [d / c, P, c] layout of
    mslam_match (c = 16 bytes of elements): mslam_desc_to_chunked on CUDA
    tensors (the same permutation with torch on CPU tensors).  With `out` a
    larger chunk-planar pool [d / c, P_out, c], D fills its pixels
    [p0, p0 + P).  A layout change only."""
    c = 16 // D.element_size()
    P, d = D.shape
    if d % c:
        raise ValueError(f"descriptor dimension {d} is not a multiple of {c}")
    if not D.is_cuda:
        return D.reshape(P, d // c, c).permute(1, 0, 2).contiguous()
    if D.dtype not in DTYPES:
        raise ValueError(f"unsupported descriptor dtype {D.dtype}")
    _need(D, "D", D.dtype, P * d)
    out = torch.empty(d // c, P, c, dtype=D.dtype, device=D.device) if out is None else out
    _need(out, "out", D.dtype)
    if out.dim() != 3 or out.shape[0] != d // c or out.shape[2] != c or not 0 <= p0 <= out.shape[1] - P:
        raise ValueError(f"out must be chunk-planar [{d // c}, >= {p0 + P}, {c}] (got {tuple(out.shape)})")
    dst = out.data_ptr() + p0 * 16
    check(lib().mslam_desc_to_chunked(DTYPES[D.dtype], d, P, D.data_ptr(), dst, out.shape[1], _stream(D.device)),
          "mslam_desc_to_chunked")
    return out


def match(plan: Plan, params: Params, X_ref, X_qry, D_ref, D_qry, Q_ref, Q_qry, init_idx=None, idx_out=None,
          q_out=None, edge_range: Tuple[int, int] = (-1, -1), per_edge: bool = False, workspace=None,
          counts: Optional[Tuple[torch.Tensor, torch.Tensor]] = None):
    """mslam_match (Sec. 3.2): returns (idx int32 [P], q [P]).  D_ref and
    D_qry are chunk-planar [d / c, P, c] (see chunk_descriptors).
    workspace: the ray-image workspace (MSLAM_OP_MATCH; allocated when None),
    or False to normalise the rays at the taps instead (same result).
    counts: (n_valid, n_unique) int32 [E] tensors that receive the Sec. 3.4
    keyframe counts of the matched edges, taken in the matching epilogue."""
    dt = X_ref.dtype
    if dt not in DTYPES:
        raise ValueError(f"unsupported storage dtype {dt}")
    P = plan.edge_pixels
    c = 16 // X_ref.element_size()
    if D_ref.dim() != 3 or D_ref.shape[1] != P or D_ref.shape[2] != c or D_qry.shape != D_ref.shape:
        raise ValueError(f"descriptors must be chunk-planar [d/{c}, {P}, {c}] (got {tuple(D_ref.shape)})")
    d = D_ref.shape[0] * c
    for t, nm, ne in ((X_ref, "X_ref", 3 * P), (X_qry, "X_qry", 3 * P), (D_ref, "D_ref", d * P),
                      (D_qry, "D_qry", d * P), (Q_ref, "Q_ref", P), (Q_qry, "Q_qry", P)):
        _need(t, nm, dt, ne)
    if init_idx is not None:
        _need(init_idx, "init_idx", torch.int32, P)
    if idx_out is None:
        idx_out = torch.empty(P, dtype=torch.int32, device=X_ref.device)
    if q_out is None:
        q_out = torch.empty(P, dtype=dt, device=X_ref.device)
    _need(idx_out, "idx_out", torch.int32, P)
    _need(q_out, "q_out", dt, P)
    if workspace is not False:
        workspace = _workspace(plan, _lib.MSLAM_OP_MATCH, workspace)
    ws_ptr, ws_n = (None, 0) if workspace is False else (workspace.data_ptr(), workspace.numel())
    nv = nu = None
    if counts is not None:
        nv, nu = counts
        _need(nv, "n_valid", torch.int32, plan.E)
        _need(nu, "n_unique", torch.int32, plan.E)
    check(lib().mslam_match(C.byref(params), plan.handle, DTYPES[dt], d, X_ref.data_ptr(), X_qry.data_ptr(),
                            D_ref.data_ptr(), D_qry.data_ptr(), Q_ref.data_ptr(), Q_qry.data_ptr(),
                            _ptr(init_idx), idx_out.data_ptr(), q_out.data_ptr(), _ptr(nv), _ptr(nu),
                            int(edge_range[0]),
                            int(edge_range[1]), ws_ptr, ws_n, _lib.MSLAM_FLAG_PER_EDGE if per_edge else 0,
                            _stream(X_ref.device)), "mslam_match")
    return idx_out, q_out


def match_stats(plan: Plan, idx, workspace=None):
    """mslam_match_stats (Sec. 3.4): (n_valid [E], n_unique [E]) int32."""
    _need(idx, "idx", torch.int32, plan.edge_pixels)
    dev = idx.device
    nv = torch.empty(plan.E, dtype=torch.int32, device=dev)
    nu = torch.empty(plan.E, dtype=torch.int32, device=dev)
    ws = _workspace(plan, _lib.MSLAM_OP_STATS, workspace)
    check(lib().mslam_match_stats(plan.handle, idx.data_ptr(), nv.data_ptr(), nu.data_ptr(), ws.data_ptr(),
                                  ws.numel(), _stream(dev)), "mslam_match_stats")
    return nv, nu


OMEGA_K = 0.333  # keyframe threshold omega_k of the paper's evaluation setup (Supp. S4)


def keyframe_needed(n_valid, n_unique, n_query, omega_k: float = OMEGA_K):
    """The keyframe criterion of Sec. 3.4 from mslam_match_stats' counts
    (mslam_keyframe_criterion, host C): True where the fraction of the
    frame's query pixels with a valid match, or of distinct keyframe pixels
    they hit, falls below omega_k.  n_valid, n_unique: per-edge counts
    (tensors or arrays, any device); n_query: query pixels per edge (scalar
    or per edge).  Returns a bool tensor on the host."""
    nv = np.ascontiguousarray(torch.as_tensor(n_valid).cpu().numpy().astype(np.int32).reshape(-1))
    nu = np.ascontiguousarray(torch.as_tensor(n_unique).cpu().numpy().astype(np.int32).reshape(-1))
    nq = np.ascontiguousarray(np.broadcast_to(np.asarray(torch.as_tensor(n_query).cpu().numpy(), dtype=np.int64),
                                              nv.shape))
    out = np.zeros(nv.shape, dtype=np.int32)
    check(lib().mslam_keyframe_criterion(int(nv.size), nv.ctypes.data, nu.ctypes.data, nq.ctypes.data,
                                         float(omega_k), out.ctypes.data), "mslam_keyframe_criterion")
    return torch.from_numpy(out.astype(bool))


def ray_image(X: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """mslam_ray_image (a1, Sec. 3.1): psi(X) = X / |X| for X [..., 3] (FP32 or
    FP16, CUDA), the zero ray for a zero or non-finite point."""
    if X.shape[-1] != 3 or not X.is_contiguous() or not X.is_cuda or X.dtype not in DTYPES:
        raise ValueError("X must be a contiguous FP32 or FP16 CUDA tensor of shape [..., 3]")
    R = torch.empty_like(X) if out is None else out
    if R.shape != X.shape or R.dtype != X.dtype or not R.is_contiguous() or R.device != X.device:
        raise ValueError("out must match X in shape, dtype, layout and device")
    check(lib().mslam_ray_image(DTYPES[X.dtype], X.numel() // 3, X.data_ptr(), R.data_ptr(), _stream(X.device)),
          "mslam_ray_image")
    return R


def calib_backproject(X: torch.Tensor, fx: float, fy: float, cx: float, cy: float) -> torch.Tensor:
    """mslam_calib_backproject (Sec. 3.6), in place on X [n, H, W, 3] (FP32 or
    FP16, CUDA); returns X."""
    if X.dim() != 4 or X.shape[-1] != 3 or not X.is_contiguous() or not X.is_cuda or X.dtype not in DTYPES:
        raise ValueError("X must be a contiguous FP32 or FP16 CUDA tensor of shape [n, H, W, 3]")
    check(lib().mslam_calib_backproject(DTYPES[X.dtype], X.shape[0], X.shape[1], X.shape[2], fx, fy, cx, cy, X.data_ptr(),
                                        _stream(X.device)), "mslam_calib_backproject")
    return X


def gn_linearize(plan: Plan, params: Params, T_wc, X_canon, idx, q, H=None, g=None, cost=None, n_valid=None,
                 workspace=None, per_edge: bool = False):
    """mslam_gn_linearize (Eq. backend_ray): returns (H [E,14,14], g [E,14],
    cost [E], n_valid [E])."""
    dt = X_canon.dtype
    if dt not in DTYPES:
        raise ValueError(f"unsupported storage dtype {dt}")
    dev = X_canon.device
    _need(T_wc, "T_wc", torch.float64, 8 * plan.N)
    _need(X_canon, "X_canon", dt, 3 * plan.kf_pixels)
    _need(idx, "idx", torch.int32, plan.edge_pixels)
    _need(q, "q", dt, plan.edge_pixels)
    E = plan.E
    H = torch.empty(E, 14, 14, dtype=torch.float32, device=dev) if H is None else H
    g = torch.empty(E, 14, dtype=torch.float32, device=dev) if g is None else g
    cost = torch.empty(E, dtype=torch.float64, device=dev) if cost is None else cost
    n_valid = torch.empty(E, dtype=torch.int32, device=dev) if n_valid is None else n_valid
    _need(H, "H", torch.float32, 196 * E)
    _need(g, "g", torch.float32, 14 * E)
    _need(cost, "cost", torch.float64, E)
    _need(n_valid, "n_valid", torch.int32, E)
    ws = _workspace(plan, _lib.MSLAM_OP_LINEARIZE, workspace)
    check(lib().mslam_gn_linearize(C.byref(params), plan.handle, DTYPES[dt], T_wc.data_ptr(), X_canon.data_ptr(),
                                   idx.data_ptr(), q.data_ptr(), H.data_ptr(), g.data_ptr(), cost.data_ptr(),
                                   n_valid.data_ptr(), ws.data_ptr(), ws.numel(),
                                   _lib.MSLAM_FLAG_PER_EDGE if per_edge else 0, _stream(dev)), "mslam_gn_linearize")
    return H, g, cost, n_valid


def pack_bytes(plan: Plan, dtype) -> int:
    op = _lib.MSLAM_OP_PACK_F16 if dtype == torch.float16 else _lib.MSLAM_OP_PACK_F32
    return plan.workspace_bytes(op)


def gn_pack(plan: Plan, params: Params, X_canon, idx, q, packed=None):
    """mslam_gn_pack: gather the inputs of every used match once (the
    matches are fixed during the Gauss-Newton loop).  Returns the packed
    buffer (uint8 device tensor)."""
    dt = X_canon.dtype
    if dt not in DTYPES:
        raise ValueError(f"unsupported storage dtype {dt}")
    _need(X_canon, "X_canon", dt, 3 * plan.kf_pixels)
    _need(idx, "idx", torch.int32, plan.edge_pixels)
    _need(q, "q", dt, plan.edge_pixels)
    nb = pack_bytes(plan, dt)
    if packed is None:
        packed = torch.empty(max(nb, 256), dtype=torch.uint8, device=X_canon.device)
    _need(packed, "packed", torch.uint8)
    check(lib().mslam_gn_pack(C.byref(params), plan.handle, DTYPES[dt], X_canon.data_ptr(), idx.data_ptr(),
                              q.data_ptr(), packed.data_ptr(), packed.numel(), _stream(X_canon.device)),
          "mslam_gn_pack")
    return packed


def gn_track(plan: Plan, params: Params, dtype, T_wc, packed, n_iters: int, dev_status=None, workspace=None):
    """mslam_gn_track (Sec. 3.3): n_iters tracking Gauss-Newton iterations, one
    launch each, on plans whose every graph is one keyframe and one frame
    joined by one edge; T_wc [N, 8] FP64 updated in place.  Returns the
    per-graph status."""
    if dtype not in DTYPES:
        raise ValueError(f"unsupported storage dtype {dtype}")
    dev = packed.device
    _need(T_wc, "T_wc", torch.float64, 8 * plan.N)
    _need(packed, "packed", torch.uint8)
    st = torch.zeros(plan.G, dtype=torch.int32, device=dev) if dev_status is None else dev_status
    _need(st, "dev_status", torch.int32, plan.G)
    ws = _workspace(plan, _lib.MSLAM_OP_TRACK, workspace)
    check(lib().mslam_gn_track(C.byref(params), plan.handle, DTYPES[dtype], T_wc.data_ptr(), packed.data_ptr(),
                               packed.numel(), int(n_iters), st.data_ptr(), ws.data_ptr(), ws.numel(), _stream(dev)),
          "mslam_gn_track")
    return st


def gn_linearize_packed(plan: Plan, params: Params, dtype, T_wc, packed, H=None, g=None, cost=None, n_valid=None,
                        workspace=None, per_edge: bool = False, dev_status=None):
    """mslam_gn_linearize_packed: the linearisation of gn_linearize from the
    records of gn_pack.  dev_status (int32 [G] or None) receives
    MSLAM_ERR_TIMEOUT for the graphs of a streamed launch whose bounded wait
    gave up."""
    if dtype not in DTYPES:
        raise ValueError(f"unsupported storage dtype {dtype}")
    dev = packed.device
    _need(T_wc, "T_wc", torch.float64, 8 * plan.N)
    _need(packed, "packed", torch.uint8)
    E = plan.E
    H = torch.empty(E, 14, 14, dtype=torch.float32, device=dev) if H is None else H
    g = torch.empty(E, 14, dtype=torch.float32, device=dev) if g is None else g
    cost = torch.empty(E, dtype=torch.float64, device=dev) if cost is None else cost
    n_valid = torch.empty(E, dtype=torch.int32, device=dev) if n_valid is None else n_valid
    _need(H, "H", torch.float32, 196 * E)
    _need(g, "g", torch.float32, 14 * E)
    _need(cost, "cost", torch.float64, E)
    _need(n_valid, "n_valid", torch.int32, E)
    if dev_status is not None:
        _need(dev_status, "dev_status", torch.int32, plan.G)
    ws = _workspace(plan, _lib.MSLAM_OP_LINEARIZE, workspace)
    check(lib().mslam_gn_linearize_packed(C.byref(params), plan.handle, DTYPES[dtype], T_wc.data_ptr(),
                                          packed.data_ptr(), packed.numel(), H.data_ptr(), g.data_ptr(),
                                          cost.data_ptr(), n_valid.data_ptr(), _ptr(dev_status), ws.data_ptr(),
                                          ws.numel(), _lib.MSLAM_FLAG_PER_EDGE if per_edge else 0, _stream(dev)),
          "mslam_gn_linearize_packed")
    return H, g, cost, n_valid


def gn_solve(plan: Plan, params: Params, H, g, T_wc, tau=None, dev_status=None, workspace=None):
    """mslam_gn_solve (Sec. 3.5): updates T_wc in place; returns (tau, dev_status)."""
    dev = T_wc.device
    _need(H, "H", torch.float32, 196 * plan.E)
    _need(g, "g", torch.float32, 14 * plan.E)
    _need(T_wc, "T_wc", torch.float64, 8 * plan.N)
    if dev_status is None:
        dev_status = torch.zeros(plan.G, dtype=torch.int32, device=dev)
    _need(dev_status, "dev_status", torch.int32, plan.G)
    if tau is not None:
        _need(tau, "tau", torch.float64, 7 * plan.N)
    ws = _workspace(plan, _lib.MSLAM_OP_SOLVE, workspace)
    check(lib().mslam_gn_solve(C.byref(params), plan.handle, H.data_ptr(), g.data_ptr(), T_wc.data_ptr(),
                               _ptr(tau), dev_status.data_ptr(), ws.data_ptr(), ws.numel(), _stream(dev)),
          "mslam_gn_solve")
    return tau, dev_status


def gn_backward(plan: Plan, params: Params, T_wc, X_canon, idx, q, H=None, g=None, dL_dtau=None,
                dL_dcost: float = 1.0, dL_dX=None, dL_dq=None, dev_status=None, workspace=None):
    """mslam_gn_backward: gradient of dL_dcost * E_g + dL_dtau . tau with
    respect to X_canon and q.  Returns (dL_dX float32 [Pk,3], dL_dq float32 [P], dev_status)."""
    dt = X_canon.dtype
    dev = X_canon.device
    _need(T_wc, "T_wc", torch.float64, 8 * plan.N)
    _need(X_canon, "X_canon", dt, 3 * plan.kf_pixels)
    _need(idx, "idx", torch.int32, plan.edge_pixels)
    _need(q, "q", dt, plan.edge_pixels)
    if dL_dtau is not None:
        _need(dL_dtau, "dL_dtau", torch.float64, 7 * plan.N)
        _need(H, "H", torch.float32, 196 * plan.E)
        _need(g, "g", torch.float32, 14 * plan.E)
    dL_dX = torch.empty(plan.kf_pixels, 3, dtype=torch.float32, device=dev) if dL_dX is None else dL_dX
    dL_dq = torch.empty(plan.edge_pixels, dtype=torch.float32, device=dev) if dL_dq is None else dL_dq
    if dev_status is None:
        dev_status = torch.zeros(plan.G, dtype=torch.int32, device=dev)
    _need(dL_dX, "dL_dX", torch.float32, 3 * plan.kf_pixels)
    _need(dL_dq, "dL_dq", torch.float32, plan.edge_pixels)
    _need(dev_status, "dev_status", torch.int32, plan.G)
    ws = _workspace(plan, _lib.MSLAM_OP_BACKWARD, workspace)
    check(lib().mslam_gn_backward(C.byref(params), plan.handle, DTYPES[dt], T_wc.data_ptr(), X_canon.data_ptr(),
                                  idx.data_ptr(), q.data_ptr(), _ptr(H), _ptr(g), _ptr(dL_dtau), float(dL_dcost),
                                  dL_dX.data_ptr(), dL_dq.data_ptr(), dev_status.data_ptr(), ws.data_ptr(),
                                  ws.numel(), _stream(dev)), "mslam_gn_backward")
    return dL_dX, dL_dq, dev_status


def gn_step_backward(plan: Plan, params: Params, T_wc, X_canon, idx, q, H, g, dL_dTnew=None, dL_dtau=None,
                     dL_dcost: float = 0.0, dL_dX=None, dL_dq=None, dL_dT=None, dev_status=None, workspace=None):
    """mslam_gn_step_backward: gradient of dL_dcost * E_g(T) + dL_dtau . tau
    + <dL_dTnew, T'> over one Gauss-Newton step T' = Exp(tau) o T with
    respect to X_canon, q and T_wc (pose gradients in the [N, 8] embedding).
    Returns (dL_dX float32 [Pk, 3], dL_dq float32 [P], dL_dT float64 [N, 8],
    dev_status)."""
    dt = X_canon.dtype
    dev = X_canon.device
    _need(T_wc, "T_wc", torch.float64, 8 * plan.N)
    _need(X_canon, "X_canon", dt, 3 * plan.kf_pixels)
    _need(idx, "idx", torch.int32, plan.edge_pixels)
    _need(q, "q", dt, plan.edge_pixels)
    _need(H, "H", torch.float32, 196 * plan.E)
    _need(g, "g", torch.float32, 14 * plan.E)
    if dL_dTnew is not None:
        _need(dL_dTnew, "dL_dTnew", torch.float64, 8 * plan.N)
    if dL_dtau is not None:
        _need(dL_dtau, "dL_dtau", torch.float64, 7 * plan.N)
    dL_dX = torch.empty(plan.kf_pixels, 3, dtype=torch.float32, device=dev) if dL_dX is None else dL_dX
    dL_dq = torch.empty(plan.edge_pixels, dtype=torch.float32, device=dev) if dL_dq is None else dL_dq
    dL_dT = torch.empty(plan.N, 8, dtype=torch.float64, device=dev) if dL_dT is None else dL_dT
    _need(dL_dT, "dL_dT", torch.float64, 8 * plan.N)
    if dev_status is None:
        dev_status = torch.zeros(plan.G, dtype=torch.int32, device=dev)
    _need(dL_dX, "dL_dX", torch.float32, 3 * plan.kf_pixels)
    _need(dL_dq, "dL_dq", torch.float32, plan.edge_pixels)
    _need(dev_status, "dev_status", torch.int32, plan.G)
    ws = _workspace(plan, _lib.MSLAM_OP_BACKWARD, workspace)
    check(lib().mslam_gn_step_backward(C.byref(params), plan.handle, DTYPES[dt], T_wc.data_ptr(),
                                       X_canon.data_ptr(), idx.data_ptr(), q.data_ptr(), H.data_ptr(), g.data_ptr(),
                                       _ptr(dL_dTnew), _ptr(dL_dtau), float(dL_dcost), dL_dX.data_ptr(),
                                       dL_dq.data_ptr(), dL_dT.data_ptr(), dev_status.data_ptr(), ws.data_ptr(),
                                       ws.numel(), _stream(dev)), "mslam_gn_step_backward")
    return dL_dX, dL_dq, dL_dT, dev_status


def fuse(T_wc, k: int, f: int, X_canon_k, C_canon_k, X_kf, C_kf):
    """mslam_fuse (Sec. 3.3): update keyframe k's canonical pointmap and
    confidence in place with the prediction made together with frame f."""
    dt = X_canon_k.dtype
    if dt not in DTYPES:
        raise ValueError(f"unsupported storage dtype {dt}")
    n = C_canon_k.numel()
    for t, nm, ne in ((X_canon_k, "X_canon_k", 3 * n), (C_canon_k, "C_canon_k", n), (X_kf, "X_kf", 3 * n),
                      (C_kf, "C_kf", n)):
        _need(t, nm, dt, ne)
    _need(T_wc, "T_wc", torch.float64)
    if max(k, f) >= T_wc.numel() // 8:
        raise ValueError("pose index out of range")
    check(lib().mslam_fuse(DTYPES[dt], T_wc.data_ptr(), int(k), int(f), n, X_canon_k.data_ptr(),
                           C_canon_k.data_ptr(), X_kf.data_ptr(), C_kf.data_ptr(), _stream(X_canon_k.device)),
          "mslam_fuse")
    return X_canon_k, C_canon_k


class GaussNewton:
    """Device-resident Gauss-Newton loop over a plan (Sec. 3.5): buffers are
    allocated once, so the loop can be captured into a CUDA graph.  With
    packed=True the used matches are gathered once per run (mslam_gn_pack)
    and every iteration streams them (mslam_gn_linearize_packed)."""

    def __init__(self, plan: Plan, params: Params, X_canon, idx, q, per_edge: bool = False, packed: bool = False):
        self.plan, self.params, self.per_edge, self.packed = plan, params, per_edge, packed
        self.X, self.idx, self.q = X_canon, idx, q
        dev = X_canon.device
        E, N = plan.E, plan.N
        self.H = torch.empty(E, 14, 14, dtype=torch.float32, device=dev)
        self.g = torch.empty(E, 14, dtype=torch.float32, device=dev)
        self.cost = torch.empty(E, dtype=torch.float64, device=dev)
        self.n_valid = torch.empty(E, dtype=torch.int32, device=dev)
        self.tau = torch.zeros(N, 7, dtype=torch.float64, device=dev)
        self.status = torch.zeros(plan.G, dtype=torch.int32, device=dev)
        self.ws_lin = plan.workspace(_lib.MSLAM_OP_LINEARIZE)
        self.ws_solve = plan.workspace(_lib.MSLAM_OP_SOLVE)
        self.pack_buf = (torch.empty(max(pack_bytes(plan, X_canon.dtype), 256), dtype=torch.uint8, device=dev)
                         if packed else None)
        self.T = torch.empty(N, 8, dtype=torch.float64, device=dev)
        self.graph = None

    def pack(self):
        if self.packed:
            gn_pack(self.plan, self.params, self.X, self.idx, self.q, self.pack_buf)

    def linearize(self):
        if self.packed:
            gn_linearize_packed(self.plan, self.params, self.X.dtype, self.T, self.pack_buf, self.H, self.g,
                                self.cost, self.n_valid, self.ws_lin, self.per_edge, self.status)
        else:
            gn_linearize(self.plan, self.params, self.T, self.X, self.idx, self.q, self.H, self.g, self.cost,
                         self.n_valid, self.ws_lin, self.per_edge)

    def solve(self):
        gn_solve(self.plan, self.params, self.H, self.g, self.T, self.tau, self.status, self.ws_solve)

    def step(self):
        self.linearize()
        self.solve()

    def run(self, T_init, iters: int):
        """Pack (if packed) and run `iters` iterations from T_init."""
        self.T.copy_(T_init)
        self.status.zero_()
        self.pack()
        for _ in range(iters):
            self.step()
        return self.T

    def run_tracking(self, T_init, iters: int):
        """Pack and run `iters` iterations with mslam_gn_track (one launch per
        iteration; plans of one keyframe and one frame per graph, packed form)."""
        if not self.packed:
            raise ValueError("run_tracking needs the packed form")
        if not hasattr(self, "ws_track"):
            self.ws_track = self.plan.workspace(_lib.MSLAM_OP_TRACK)
        self.T.copy_(T_init)
        self.status.zero_()
        self.pack()
        gn_track(self.plan, self.params, self.X.dtype, self.T, self.pack_buf, iters, self.status, self.ws_track)
        return self.T

    def capture(self, iters: int):
        """Capture pack + `iters` steps (on the current buffers) into a CUDA graph."""
        s = torch.cuda.Stream(self.X.device)
        s.wait_stream(torch.cuda.current_stream(self.X.device))
        with torch.cuda.stream(s):
            self.pack()
            self.step()  # warm-up outside capture (lazy module loading)
        torch.cuda.current_stream(self.X.device).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.pack()
            for _ in range(iters):
                self.step()
        self.graph = g
        return g

    def replay(self, T_init):
        self.T.copy_(T_init)
        self.status.zero_()
        self.graph.replay()
        return self.T
