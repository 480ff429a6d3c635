"""Seeded synthetic two-view pointmap workloads.

The paper (MASt3R-SLAM, arXiv 2412.12392) feeds its matching and Gauss-Newton
stages with the outputs of a two-view prior network (Sec. 3.1): per image pair
(i, j) the pointmaps X^i_i, X^j_i (H x W x 3), per-pixel confidences, d-dim
descriptors D and descriptor confidences Q, at 512 x 384 (Sec. 4 setup).  No
network weights or datasets are used here; this module synthesises inputs with
the same shapes and structure:

* scene: a box room with eight axis-aligned boxes, ray-cast by a generic
  central camera (pinhole plus optional radial term k1), so every pointmap is a
  consistent view of one world and cross-view correspondences exist;
* pointmaps: ground truth plus Gaussian depth noise (standard deviation 1 % of
  depth, along each pixel's ray), drawn independently for every prediction;
* descriptors: smooth value noise over 5 cm world voxels (unit vectors hashed
  at voxel corners, trilinearly blended, normalised) plus per-prediction noise;
* confidences: uniform U(1, 10) or log-normal exp(N(1, 0.5^2));
* trajectories: a random walk (2 deg, 0.2 m) or a 1 m loop facing the far wall;
* edges: bidirectional sequential and skip-one pairs plus seeded loop closures,
  each with a contiguous invalid column band that sets its overlap.

Every random number comes from a counter-based hash of (seed, stream, frame,
pixel, channel) evaluated with torch integer ops, so the same call gives the
same workload on the CPU and on a GPU (up to the rounding of transcendental
functions).  This module holds scene synthesis only: it contains none of the
method's arithmetic (no ray normalisation of the method, no Lie-group maps, no
matching, no Gauss-Newton).  Both the oracle tests and the GPU path consume it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import torch

M32 = 0xFFFFFFFF

# hash streams
S_NOISE_X = 1
S_NOISE_Y = 2
S_DESC_CORNER = 3
S_DESC_NOISE = 4
S_CONF = 5
S_TRAJ = 6
S_BOX = 7
S_EDGE = 8
S_OCC = 9
S_CANON = 10
S_INIT = 11


def _mul32(x: torch.Tensor, k: int) -> torch.Tensor:
    """(x * k) mod 2^32 for 0 <= x < 2^32, without int64 overflow."""
    lo = x & 0xFFFF
    hi = x >> 16
    return (lo * k + (((hi * k) & 0xFFFF) << 16)) & M32


def _fmix32(x: torch.Tensor) -> torch.Tensor:
    """MurmurHash3's 32-bit finaliser (public domain avalanche mix)."""
    x = x ^ (x >> 16)
    x = _mul32(x, 0x85EBCA6B)
    x = x ^ (x >> 13)
    x = _mul32(x, 0xC2B2AE35)
    x = x ^ (x >> 16)
    return x


def hash_u32(seed: int, stream: int, *keys, device="cpu") -> torch.Tensor:
    """Counter-based hash of (seed, stream, keys...) -> uint32 values in int64."""
    h = _fmix32(torch.tensor((seed * 0x9E3779B1) & M32, dtype=torch.int64, device=device))
    h = _fmix32(h ^ (stream & M32))
    for k in keys:
        if not torch.is_tensor(k):
            k = torch.tensor(int(k) & M32, dtype=torch.int64, device=device)
        h = _fmix32(h ^ (k.to(torch.int64) & M32))
    return h


def uniform(seed, stream, *keys, device="cpu") -> torch.Tensor:
    """U(0, 1) float64, open interval, 24-bit resolution."""
    h = hash_u32(seed, stream, *keys, device=device)
    return ((h >> 8).to(torch.float64) + 0.5) * (1.0 / 16777216.0)


def normal(seed, stream, *keys, device="cpu") -> torch.Tensor:
    """N(0, 1) float64 by the Box-Muller transform of two hashed uniforms."""
    u1 = uniform(seed, stream, *keys, 0, device=device)
    u2 = uniform(seed, stream, *keys, 1, device=device)
    return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------
# rigid-body helpers for scene synthesis (rotation matrices, float64)
# ----------------------------------------------------------------------------

def _rodrigues(axis: torch.Tensor, angle: float) -> torch.Tensor:
    a = axis / torch.linalg.norm(axis)
    K = torch.tensor([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]], dtype=torch.float64)
    return torch.eye(3, dtype=torch.float64) + math.sin(angle) * K + (1.0 - math.cos(angle)) * (K @ K)


def _rot_to_quat(R: torch.Tensor) -> torch.Tensor:
    """Rotation matrix -> unit quaternion (x, y, z, w), w >= 0 (Shepperd's method)."""
    m = R
    tr = float(m[0, 0] + m[1, 1] + m[2, 2])
    if tr > 0:
        s = math.sqrt(tr + 1.0) * 2
        w = 0.25 * s
        x = float(m[2, 1] - m[1, 2]) / s
        y = float(m[0, 2] - m[2, 0]) / s
        z = float(m[1, 0] - m[0, 1]) / s
    elif m[0, 0] > m[1, 1] and m[0, 0] > m[2, 2]:
        s = math.sqrt(1.0 + float(m[0, 0] - m[1, 1] - m[2, 2])) * 2
        w = float(m[2, 1] - m[1, 2]) / s
        x = 0.25 * s
        y = float(m[0, 1] + m[1, 0]) / s
        z = float(m[0, 2] + m[2, 0]) / s
    elif m[1, 1] > m[2, 2]:
        s = math.sqrt(1.0 + float(m[1, 1] - m[0, 0] - m[2, 2])) * 2
        w = float(m[0, 2] - m[2, 0]) / s
        x = float(m[0, 1] + m[1, 0]) / s
        y = 0.25 * s
        z = float(m[1, 2] + m[2, 1]) / s
    else:
        s = math.sqrt(1.0 + float(m[2, 2] - m[0, 0] - m[1, 1])) * 2
        w = float(m[1, 0] - m[0, 1]) / s
        x = float(m[0, 2] + m[2, 0]) / s
        y = float(m[1, 2] + m[2, 1]) / s
        z = 0.25 * s
    q = torch.tensor([x, y, z, w], dtype=torch.float64)
    q = q / torch.linalg.norm(q)
    if q[3] < 0:
        q = -q
    return q


def quat_to_rot(q: torch.Tensor) -> torch.Tensor:
    x, y, z, w = [float(v) for v in q]
    return torch.tensor([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ], dtype=torch.float64)


def pose_pack(R: torch.Tensor, t: torch.Tensor, s: float) -> torch.Tensor:
    """Pose as 8 float64: translation (3), quaternion x y z w (4), scale (1)."""
    return torch.cat([t.to(torch.float64), _rot_to_quat(R), torch.tensor([s], dtype=torch.float64)])


def pose_unpack(T: torch.Tensor) -> Tuple[torch.Tensor, torch.Tensor, float]:
    return quat_to_rot(T[3:7]), T[0:3].clone(), float(T[7])


# ----------------------------------------------------------------------------
# scene and camera
# ----------------------------------------------------------------------------

ROOM_LO = (-4.0, -3.0, -2.5)
ROOM_HI = (4.0, 3.0, 7.0)
VOXEL = 0.05


def scene_boxes(seed: int) -> torch.Tensor:
    """Eight seeded axis-aligned boxes [8, 2, 3] (lo, hi), in front of the cameras."""
    out = []
    for b in range(8):
        u = [float(uniform(seed, S_BOX, b, c)) for c in range(6)]
        cx = -2.5 + 5.0 * u[0]
        cy = -2.0 + 4.0 * u[1]
        cz = 2.2 + 3.3 * u[2]
        hx, hy, hz = 0.2 + 0.4 * u[3], 0.2 + 0.4 * u[4], 0.2 + 0.4 * u[5]
        out.append([[cx - hx, cy - hy, cz - hz], [cx + hx, cy + hy, cz + hz]])
    return torch.tensor(out, dtype=torch.float64)


def camera_dirs(H: int, W: int, k1: float, device) -> torch.Tensor:
    """Camera-frame ray directions (z = 1) of a generic central camera: pinhole
    with focal 0.8 W, principal point at the image centre and radial factor
    (1 + k1 r^2) on the normalised coordinates.  Returns [H*W, 3] float64."""
    f = 0.8 * W
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    v, u = torch.meshgrid(torch.arange(H, dtype=torch.float64, device=device),
                          torch.arange(W, dtype=torch.float64, device=device), indexing="ij")
    xn = (u - cx) / f
    yn = (v - cy) / f
    rad = 1.0 + k1 * (xn * xn + yn * yn)
    d = torch.stack([xn * rad, yn * rad, torch.ones_like(xn)], dim=-1)
    return d.reshape(-1, 3)


def raycast(T_wc: torch.Tensor, dirs_c: torch.Tensor, boxes: torch.Tensor) -> torch.Tensor:
    """Ray-cast the room from camera pose T_wc (scale 1).  Returns camera-frame
    points [P, 3] float64 (the depth parameter along the z = 1 direction)."""
    device = dirs_c.device
    R, t, _ = pose_unpack(T_wc.cpu())
    R = R.to(device)
    t = t.to(device)
    w = dirs_c @ R.T  # world directions
    o = t.view(1, 3)
    big = torch.full_like(w[:, 0], float("inf"))
    lo = torch.tensor(ROOM_LO, dtype=torch.float64, device=device)
    hi = torch.tensor(ROOM_HI, dtype=torch.float64, device=device)
    t_room = big.clone()
    for a in range(3):
        wa = w[:, a]
        ta = torch.where(wa > 0, (hi[a] - o[0, a]) / wa, torch.where(wa < 0, (lo[a] - o[0, a]) / wa, big))
        t_room = torch.minimum(t_room, ta)
    t_hit = t_room
    for b in range(boxes.shape[0]):
        blo = boxes[b, 0].to(device)
        bhi = boxes[b, 1].to(device)
        tn = torch.full_like(big, -float("inf"))
        tf = big.clone()
        for a in range(3):
            wa = w[:, a]
            safe = torch.where(wa == 0, torch.full_like(wa, 1e-300), wa)
            t1 = (blo[a] - o[0, a]) / safe
            t2 = (bhi[a] - o[0, a]) / safe
            tn = torch.maximum(tn, torch.minimum(t1, t2))
            tf = torch.minimum(tf, torch.maximum(t1, t2))
        hit = (tn <= tf) & (tn > 1e-6)
        t_hit = torch.where(hit & (tn < t_hit), tn, t_hit)
    return dirs_c * t_hit.unsqueeze(-1)


def transform(T: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
    """Apply a scene pose (s R X + t) to points [P, 3] float64."""
    R, t, s = pose_unpack(T.cpu())
    return s * (X @ R.to(X.device).T) + t.to(X.device)


def pose_inv(T: torch.Tensor) -> torch.Tensor:
    R, t, s = pose_unpack(T)
    Ri = R.T
    return pose_pack(Ri, -(Ri @ t) / s, 1.0 / s)


def pose_mul(A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    Ra, ta, sa = pose_unpack(A)
    Rb, tb, sb = pose_unpack(B)
    return pose_pack(Ra @ Rb, sa * (Ra @ tb) + ta, sa * sb)


# ----------------------------------------------------------------------------
# descriptors and confidences
# ----------------------------------------------------------------------------

def desc_gt(seed: int, P_world: torch.Tensor, d: int, chunk: int = 1 << 16) -> torch.Tensor:
    """Smooth world-anchored descriptors: unit vectors hashed at the corners of
    5 cm voxels, trilinearly blended, normalised.  P_world [P, 3] -> [P, d] f32."""
    device = P_world.device
    out = torch.empty(P_world.shape[0], d, dtype=torch.float32, device=device)
    ch = torch.arange(d, dtype=torch.int64, device=device).view(1, 1, d)
    for s0 in range(0, P_world.shape[0], chunk):
        P = P_world[s0:s0 + chunk]
        g = P / VOXEL
        base = torch.floor(g)
        fr = g - base
        bi = base.to(torch.int64) + 512
        corners = []
        weights = []
        for cz in (0, 1):
            for cy in (0, 1):
                for cx in (0, 1):
                    key = ((bi[:, 0] + cx) & 1023) | (((bi[:, 1] + cy) & 1023) << 10) | (((bi[:, 2] + cz) & 1023) << 20)
                    corners.append(key)
                    wx = fr[:, 0] if cx else 1 - fr[:, 0]
                    wy = fr[:, 1] if cy else 1 - fr[:, 1]
                    wz = fr[:, 2] if cz else 1 - fr[:, 2]
                    weights.append(wx * wy * wz)
        key = torch.stack(corners, dim=1).unsqueeze(-1)  # [p, 8, 1]
        vec = normal(seed, S_DESC_CORNER, key, ch, device=device)  # [p, 8, d]
        vec = vec / torch.linalg.norm(vec, dim=-1, keepdim=True)
        wgt = torch.stack(weights, dim=1).unsqueeze(-1)
        D = (vec * wgt).sum(dim=1)
        D = D / torch.linalg.norm(D, dim=-1, keepdim=True).clamp_min(1e-12)
        out[s0:s0 + chunk] = D.to(torch.float32)
    return out


def desc_noisy(seed: int, Dgt: torch.Tensor, stream_key: int, sigma: float = 0.05) -> torch.Tensor:
    device = Dgt.device
    P, d = Dgt.shape
    pix = torch.arange(P, dtype=torch.int64, device=device).view(P, 1)
    ch = torch.arange(d, dtype=torch.int64, device=device).view(1, d)
    n = normal(seed, S_DESC_NOISE, stream_key, pix, ch, device=device)
    D = Dgt.to(torch.float64) + sigma * n
    D = D / torch.linalg.norm(D, dim=-1, keepdim=True).clamp_min(1e-12)
    return D.to(torch.float32)


def confidence(seed: int, P: int, stream_key: int, kind: str, device) -> torch.Tensor:
    pix = torch.arange(P, dtype=torch.int64, device=device)
    if kind == "uniform":
        return (1.0 + 9.0 * uniform(seed, S_CONF, stream_key, pix, device=device)).to(torch.float32)
    z = normal(seed, S_CONF, stream_key, pix, device=device)
    return torch.exp(1.0 + 0.5 * z).to(torch.float32)


def noisy_points(seed: int, X: torch.Tensor, stream_key: int, rel: float = 0.01) -> torch.Tensor:
    """Depth noise along each pixel's ray: X (1 + rel n), n ~ N(0, 1) per pixel,
    i.e. a standard deviation of 1 % of depth.  The ray directions (the
    predicted camera model) stay smooth."""
    device = X.device
    P = X.shape[0]
    pix = torch.arange(P, dtype=torch.int64, device=device)
    n = normal(seed, S_NOISE_X, stream_key, pix, device=device)
    return X * (1.0 + rel * n).unsqueeze(-1)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    """A keyframe graph with per-edge two-view predictions, stored in pools.

    Keyframe pools (canonical pointmaps X_canon [sum_k H_k W_k, 3] and
    confidences C_canon) are indexed by kf_off; per-edge pools (reference and
    query pointmaps, descriptors and descriptor confidences of the pair
    prediction) are indexed by e_off.  Edge e = (i, j) has reference keyframe
    i and query keyframe j; its pools hold H_j W_j pixels (H_i = H_j)."""
    name: str
    N: int
    E: int
    d: int
    kf_hw: torch.Tensor          # int32 [N, 2]
    edges: torch.Tensor          # int32 [E, 2]  (i = reference, j = query)
    graph_of_kf: torch.Tensor    # int32 [N]
    kf_off: torch.Tensor         # int64 [N + 1]
    e_off: torch.Tensor          # int64 [E + 1]
    T_gt: torch.Tensor           # float64 [N, 8]
    T_init: torch.Tensor         # float64 [N, 8]
    X_canon: torch.Tensor        # [sum HW, 3]
    C_canon: torch.Tensor        # [sum HW]
    X_ref: torch.Tensor          # [sum_e HW, 3]  X^i_i of the pair prediction
    X_qry: torch.Tensor          # [sum_e HW, 3]  X^j_i of the pair prediction
    D_ref: torch.Tensor          # [sum_e HW, d]
    D_qry: torch.Tensor          # [sum_e HW, d]
    Q_ref: torch.Tensor          # [sum_e HW]
    Q_qry: torch.Tensor          # [sum_e HW]
    gt_match: torch.Tensor       # int32 [sum_e HW]: nearest-pixel GT correspondence or -1
    n_match_iters: int = 10
    n_gn_iters: int = 10
    k1: float = 0.0
    meta: Dict = field(default_factory=dict)

    @property
    def device(self):
        return self.X_canon.device

    def to_storage(self, dtype: torch.dtype) -> "Workload":
        """Cast the floating-point pools to a storage dtype (float32 or float16)."""
        kw = dict(self.__dict__)
        for k in ("X_canon", "C_canon", "X_ref", "X_qry", "D_ref", "D_qry", "Q_ref", "Q_qry"):
            kw[k] = getattr(self, k).to(dtype).contiguous()
        kw["meta"] = dict(self.meta, storage=str(dtype))
        return Workload(**kw)

    def to(self, device) -> "Workload":
        kw = dict(self.__dict__)
        for k, v in self.__dict__.items():
            if torch.is_tensor(v) and k not in ("kf_hw", "edges", "graph_of_kf", "kf_off", "e_off", "T_gt", "T_init"):
                kw[k] = v.to(device)
        return Workload(**kw)

    def edge_slice(self, e: int) -> slice:
        return slice(int(self.e_off[e]), int(self.e_off[e + 1]))

    def kf_slice(self, k: int) -> slice:
        return slice(int(self.kf_off[k]), int(self.kf_off[k + 1]))


def _random_unit(seed, stream, *keys) -> torch.Tensor:
    v = torch.stack([normal(seed, stream, *keys, c) for c in range(3)]).to(torch.float64).view(3)
    return v / torch.linalg.norm(v)


def traj_random_walk(seed: int, n: int) -> List[torch.Tensor]:
    Ts = [pose_pack(torch.eye(3, dtype=torch.float64), torch.zeros(3, dtype=torch.float64), 1.0)]
    R = torch.eye(3, dtype=torch.float64)
    t = torch.zeros(3, dtype=torch.float64)
    for k in range(1, n):
        R = _rodrigues(_random_unit(seed, S_TRAJ, k, 0), math.radians(2.0)) @ R
        step = _random_unit(seed, S_TRAJ, k, 1)
        t = t + 0.2 * step
        Ts.append(pose_pack(R, t, 1.0))
    return Ts


def traj_loop(seed: int, n: int) -> List[torch.Tensor]:
    ph = 2 * math.pi * float(uniform(seed, S_TRAJ, 0, 7))
    Ts = []
    for k in range(n):
        a = 2 * math.pi * k / n
        c = torch.tensor([math.sin(a), 0.1 * math.sin(2 * a), -0.5 - math.cos(a)], dtype=torch.float64)
        yaw = math.radians(15.0) * math.sin(3 * a + ph)
        pitch = math.radians(4.0) * math.sin(2 * a + 1.0)
        R = _rodrigues(torch.tensor([0.0, 1.0, 0.0], dtype=torch.float64), yaw) @ \
            _rodrigues(torch.tensor([1.0, 0.0, 0.0], dtype=torch.float64), pitch)
        Ts.append(pose_pack(R, c, 1.0))
    return Ts


def perturb_init(seed: int, Ts: List[torch.Tensor]) -> List[torch.Tensor]:
    """Initial poses: 2 deg about a random axis, translation off by 5 % of the
    baseline to pose 0, scale x1.05; pose 0 exact."""
    out = [Ts[0].clone()]
    t0 = Ts[0][0:3]
    for k in range(1, len(Ts)):
        R, t, s = pose_unpack(Ts[k])
        R2 = _rodrigues(_random_unit(seed, S_INIT, k, 0), math.radians(2.0)) @ R
        base = float(torch.linalg.norm(t - t0))
        t2 = t + 0.05 * max(base, 1e-3) * _random_unit(seed, S_INIT, k, 1)
        out.append(pose_pack(R2, t2, s * 1.05))
    return out


def graph_pairs(seed: int, N: int, n_pairs: int, min_gap: int = 8) -> List[Tuple[int, int]]:
    """Undirected keyframe pairs: (k, k+1), then (k, k+2), then seeded loop
    closures with |i - j| >= min_gap."""
    pairs = [(k, k + 1) for k in range(N - 1)]
    rem = n_pairs - len(pairs)
    n_skip = max(0, min(rem, N - 2, (rem + 1) // 2))
    pairs += [(k, k + 2) for k in range(n_skip)]
    min_gap = min(min_gap, max(3, N // 2))
    have = set(pairs)
    c = 0
    while len(pairs) < n_pairs:
        i = int(uniform(seed, S_EDGE, c, 0) * N)
        j = int(uniform(seed, S_EDGE, c, 1) * N)
        c += 1
        a, b = min(i, j), max(i, j)
        if b - a >= min_gap and (a, b) not in have:
            have.add((a, b))
            pairs.append((a, b))
        if c > 100000:
            raise RuntimeError("cannot place loop closures")
    return pairs


def _make_graph(name: str, seed: int, N: int, edges: List[Tuple[int, int]], H: int, W: int, d: int,
                traj: List[torch.Tensor], k1: float, conf_kind: str, device, overlap: Optional[Tuple[float, float]],
                occlusion: float, n_match_iters: int, n_gn_iters: int) -> Workload:
    boxes = scene_boxes(seed)
    dirs = camera_dirs(H, W, k1, device)
    P = H * W
    gt_pts = []  # camera-frame GT points per keyframe
    world = []
    for k in range(N):
        Xc = raycast(traj[k], dirs, boxes)
        gt_pts.append(Xc)
        world.append(transform(traj[k], Xc))
    Dgt = [desc_gt(seed, world[k], d) for k in range(N)]

    X_canon = torch.empty(N * P, 3, dtype=torch.float32, device=device)
    C_canon = torch.empty(N * P, dtype=torch.float32, device=device)
    for k in range(N):
        X_canon[k * P:(k + 1) * P] = noisy_points(seed, gt_pts[k], 100000 + k).to(torch.float32)
        C_canon[k * P:(k + 1) * P] = confidence(seed, P, 200000 + k, conf_kind, device)

    E = len(edges)
    X_ref = torch.empty(E * P, 3, dtype=torch.float32, device=device)
    X_qry = torch.empty_like(X_ref)
    D_ref = torch.empty(E * P, d, dtype=torch.float32, device=device)
    D_qry = torch.empty_like(D_ref)
    Q_ref = torch.empty(E * P, dtype=torch.float32, device=device)
    Q_qry = torch.empty_like(Q_ref)
    gt_match = torch.empty(E * P, dtype=torch.int32, device=device)
    occluded = torch.zeros(E * P, dtype=torch.bool, device=device)
    f = 0.8 * W
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    overlaps = []
    for e, (i, j) in enumerate(edges):
        sl = slice(e * P, (e + 1) * P)
        Tij = pose_mul(pose_inv(traj[i]), traj[j])
        Xj_in_i = transform(Tij, gt_pts[j])
        X_ref[sl] = noisy_points(seed, gt_pts[i], 300000 + 2 * e).to(torch.float32)
        # query prediction: depth noise in the query camera, expressed in frame i
        xq = transform(Tij, noisy_points(seed, gt_pts[j], 300000 + 2 * e + 1))
        valid = torch.ones(P, dtype=torch.bool, device=device)
        if overlap is not None:
            ov = overlap[0] + (overlap[1] - overlap[0]) * float(uniform(seed, S_EDGE, 1000 + e, 0))
            band = int(round((1.0 - ov) * W))
            start = int(float(uniform(seed, S_EDGE, 1000 + e, 1)) * (W - band + 1)) if band > 0 else 0
            cols = torch.arange(P, device=device) % W
            valid &= ~((cols >= start) & (cols < start + band))
            overlaps.append(ov)
        if occlusion > 0:
            occ = torch.zeros(P, dtype=torch.bool, device=device)
            scale = torch.ones(P, dtype=torch.float64, device=device)
            rr = torch.arange(P, device=device) // W
            cc = torch.arange(P, device=device) % W
            r = 0
            while float(occ.float().mean()) < occlusion and r < 64:
                u = [float(uniform(seed, S_OCC, e, r, c)) for c in range(5)]
                rw, rh = int(W * (0.08 + 0.12 * u[0])), int(H * (0.08 + 0.12 * u[1]))
                x0, y0 = int(u[2] * (W - rw)), int(u[3] * (H - rh))
                m = (cc >= x0) & (cc < x0 + rw) & (rr >= y0) & (rr < y0 + rh)
                scale = torch.where(m & ~occ, torch.full_like(scale, 0.3 + 0.4 * u[4]), scale)
                occ |= m
                r += 1
            xq = xq * scale.unsqueeze(-1)
            occluded[sl] = occ & valid
        xq = torch.where(valid.unsqueeze(-1), xq, torch.zeros_like(xq))
        X_qry[sl] = xq.to(torch.float32)
        D_ref[sl] = desc_noisy(seed, Dgt[i], 400000 + 2 * e)
        D_qry[sl] = desc_noisy(seed, Dgt[j], 400000 + 2 * e + 1)
        Q_ref[sl] = confidence(seed, P, 500000 + 2 * e, conf_kind, device)
        Q_qry[sl] = confidence(seed, P, 500000 + 2 * e + 1, conf_kind, device)
        # ground-truth correspondence: the pinhole-with-radial projection of the
        # noise-free point, found by inverting the radial factor with Newton steps
        xn = Xj_in_i[:, 0] / Xj_in_i[:, 2]
        yn = Xj_in_i[:, 1] / Xj_in_i[:, 2]
        rd = torch.sqrt(xn * xn + yn * yn)
        ru = rd.clone()
        for _ in range(20):
            fval = ru * (1 + k1 * ru * ru) - rd
            ru = ru - fval / (1 + 3 * k1 * ru * ru)
        sc = torch.where(rd > 0, ru / rd.clamp_min(1e-300), torch.ones_like(rd))
        pu = xn * sc * f + cx
        pv = yn * sc * f + cy
        ui = torch.floor(pu + 0.5).to(torch.int64)
        vi = torch.floor(pv + 0.5).to(torch.int64)
        inside = (ui >= 0) & (ui < W) & (vi >= 0) & (vi < H) & (Xj_in_i[:, 2] > 0) & valid
        gm = torch.where(inside, vi * W + ui, torch.full_like(ui, -1))
        gt_match[sl] = gm.to(torch.int32)

    # poses are reported relative to keyframe 0 (identity, the gauge); the
    # camera-frame pointmaps do not depend on the choice of world frame
    T0i = pose_inv(traj[0])
    rel = [pose_mul(T0i, T) for T in traj]
    T_gt = torch.stack(rel)
    T_init = torch.stack(perturb_init(seed, rel))
    kf_hw = torch.tensor([[H, W]] * N, dtype=torch.int32)
    kf_off = torch.arange(N + 1, dtype=torch.int64) * P
    e_off = torch.arange(E + 1, dtype=torch.int64) * P
    return Workload(name=name, N=N, E=E, d=d, kf_hw=kf_hw, edges=torch.tensor(edges, dtype=torch.int32).view(-1, 2),
                    graph_of_kf=torch.zeros(N, dtype=torch.int32), kf_off=kf_off, e_off=e_off,
                    T_gt=T_gt, T_init=T_init, X_canon=X_canon, C_canon=C_canon, X_ref=X_ref, X_qry=X_qry,
                    D_ref=D_ref, D_qry=D_qry, Q_ref=Q_ref, Q_qry=Q_qry, gt_match=gt_match,
                    n_match_iters=n_match_iters, n_gn_iters=n_gn_iters, k1=k1,
                    meta=dict(seed=seed, H=H, W=W, overlaps=overlaps, occluded=occluded))


def tiny(device="cpu", seed: int = 0, H: int = 96, W: int = 128) -> Workload:
    """4 keyframes in a chain (3 forward edges), 128 x 96, d = 16, pinhole,
    random walk, U(1, 10) confidences, 10 match and 10 GN iterations."""
    traj = traj_random_walk(seed, 4)
    edges = [(0, 1), (1, 2), (2, 3)]
    return _make_graph("tiny", seed, 4, edges, H, W, 16, traj, 0.0, "uniform", device, None, 0.0, 10, 10)


def tracking(device="cpu", seed: int = 1, H: int = 384, W: int = 512) -> Workload:
    """One frame against one keyframe at 512 x 384 with a radial camera
    (k1 ~ U[-0.2, 0.2]), d = 24, 10 % occluded query pixels, 20 GN iterations.
    Pose 0 is the keyframe (gauge), pose 1 the frame; edge (0, 1)."""
    traj = traj_random_walk(seed, 2)
    k1 = -0.2 + 0.4 * float(uniform(seed, S_TRAJ, 99, 0))
    return _make_graph("tracking", seed, 2, [(0, 1)], H, W, 24, traj, k1, "uniform", device, None, 0.10, 10, 20)


def global_graph(device="cpu", seed: int = 2, N: int = 64, n_pairs: int = 128, H: int = 384, W: int = 512,
                 d: int = 24, name: str = "global") -> Workload:
    """A loop trajectory of N keyframes with 2 * n_pairs directed edges
    (sequential, skip-one and seeded loop-closure pairs, both directions),
    overlap U(20 %, 90 %) per edge, log-normal confidences, 10 GN iterations."""
    traj = traj_loop(seed, N)
    pairs = graph_pairs(seed, N, n_pairs)
    edges = []
    for a, b in pairs:
        edges.append((a, b))
        edges.append((b, a))
    return _make_graph(name, seed, N, edges, H, W, d, traj, 0.0, "lognormal", device, (0.2, 0.9), 0.0, 10, 10)


BATCHED_KF = [16, 24, 32, 48, 64, 80, 96, 128]
BATCHED_EDGES = [40, 64, 96, 150, 256, 320, 400, 600]
BATCHED_LOWRES = (1, 3, 6)


def batched_graph(g: int, device="cpu", scale: int = 1, seed_offset: int = 0) -> Workload:
    """Graph g (0..7) of the batched workload: seed 100 + g (+ seed_offset),
    BATCHED_KF[g] keyframes, BATCHED_EDGES[g] directed edges, 256 x 192 for
    the graphs in BATCHED_LOWRES and 512 x 384 otherwise (divided by scale)."""
    H, W = (192, 256) if g in BATCHED_LOWRES else (384, 512)
    return global_graph(device, 100 + g + seed_offset, BATCHED_KF[g], BATCHED_EDGES[g] // 2, H // scale, W // scale,
                        name=f"batched{g}")


def batched_storage(device="cpu", dtype: torch.dtype = torch.float16, scale: int = 1,
                    seed_offset: int = 0) -> Workload:
    """The eight batched graphs merged into one set of pools, each graph cast
    to the storage dtype as soon as it is made (the FP32 pools of all eight
    full-size graphs together are about 65 GB)."""
    gs = []
    for g in range(8):
        gs.append(batched_graph(g, device, scale, seed_offset).to_storage(dtype))
        if torch.cuda.is_available() and torch.device(device).type == "cuda":
            torch.cuda.empty_cache()
    return merge(gs, name="batched")


def batched(device="cpu", scale: int = 1) -> List[Workload]:
    """Eight independent keyframe graphs (seeds 100 + g) with 16..128
    keyframes and 40..600 directed edges; graphs 1, 3, 6 at 256 x 192 and the
    rest at 512 x 384 (both divided by `scale`)."""
    return [batched_graph(g, device, scale) for g in range(8)]


def differentiation(device="cpu", seed: int = 3, H: int = 384, W: int = 512) -> Workload:
    """32 keyframes, 96 directed edges at 512 x 384, log-normal confidences."""
    return global_graph(device, seed, 32, 48, H, W, name="diff")


def merge(workloads: List[Workload], name: str = "merged") -> Workload:
    """Concatenate independent graphs into one set of pools: keyframes and
    edges are renumbered, graph_of_kf records each keyframe's graph, and the
    pools are concatenated in order (pool layout only; no arithmetic)."""
    kf_hw, edges, gof, T_gt, T_init = [], [], [], [], []
    pools = {k: [] for k in ("X_canon", "C_canon", "X_ref", "X_qry", "D_ref", "D_qry", "Q_ref", "Q_qry", "gt_match")}
    kf_base = 0
    for g, w in enumerate(workloads):
        kf_hw.append(w.kf_hw)
        edges.append(w.edges + kf_base)
        gof.append(torch.full((w.N,), g, dtype=torch.int32))
        T_gt.append(w.T_gt)
        T_init.append(w.T_init)
        for k in pools:
            pools[k].append(getattr(w, k))
        kf_base += w.N
    kf_hw = torch.cat(kf_hw)
    edges = torch.cat(edges)
    N, E = kf_hw.shape[0], edges.shape[0]
    sizes = (kf_hw[:, 0].to(torch.int64) * kf_hw[:, 1].to(torch.int64))
    kf_off = torch.zeros(N + 1, dtype=torch.int64)
    kf_off[1:] = torch.cumsum(sizes, 0)
    esz = sizes[edges[:, 1].to(torch.int64)]
    e_off = torch.zeros(E + 1, dtype=torch.int64)
    e_off[1:] = torch.cumsum(esz, 0)
    d = workloads[0].d
    return Workload(name=name, N=N, E=E, d=d, kf_hw=kf_hw, edges=edges, graph_of_kf=torch.cat(gof), kf_off=kf_off,
                    e_off=e_off, T_gt=torch.cat(T_gt), T_init=torch.cat(T_init),
                    **{k: torch.cat(v) for k, v in pools.items()},
                    n_match_iters=workloads[0].n_match_iters, n_gn_iters=workloads[0].n_gn_iters,
                    meta=dict(graphs=[w.name for w in workloads], graph_kf=[w.N for w in workloads],
                              graph_edges=[w.E for w in workloads]))
