"""Pins of the oracle's projective matching and refinement (Sec. 3.2, Eq. 2):

* noise-free pointmaps from a known camera: the LM result equals the analytic
  projection (pinhole closed form; radial camera by Newton inversion);
* the LM optimum's ray error is no worse than the best integer pixel (brute
  force over the whole image);
* convergence within 10 iterations for almost all valid pixels;
* the refinement with one level covering the whole image is the global
  descriptor argmax (exhaustive);
* a pointmap matched against itself maps every pixel to itself;
* occluded query points (depth scaled by 0.3-0.7) are rejected by the 3D
  distance test unless refinement moved them onto a surface within it.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import gen

PAR = dict(oracle.DEFAULT_PARAMS)


def noise_free_pair(H, W, k1, seed=0, rot_deg=1.5, step=0.15):
    boxes = gen.scene_boxes(seed)
    dirs = gen.camera_dirs(H, W, k1, "cpu")
    Ti = gen.pose_pack(torch.eye(3, dtype=torch.float64), torch.zeros(3, dtype=torch.float64), 1.0)
    R = gen._rodrigues(torch.tensor([0.3, 1.0, 0.2], dtype=torch.float64), np.radians(rot_deg))
    Tj = gen.pose_pack(R, torch.tensor([step, -0.05, 0.1], dtype=torch.float64), 1.0)
    Xi = gen.raycast(Ti, dirs, boxes)
    Xj = gen.raycast(Tj, dirs, boxes)
    Tij = gen.pose_mul(gen.pose_inv(Ti), Tj)
    Xq = gen.transform(Tij, Xj)
    return Xi.numpy(), Xq.numpy()


def project(X, H, W, k1):
    f = 0.8 * W
    cx, cy = (W - 1) / 2, (H - 1) / 2
    xn, yn = X[:, 0] / X[:, 2], X[:, 1] / X[:, 2]
    rd = np.hypot(xn, yn)
    ru = rd.copy()
    for _ in range(30):  # invert r (1 + k1 r^2) = rd by Newton's method
        ru = ru - (ru * (1 + k1 * ru * ru) - rd) / (1 + 3 * k1 * ru * ru)
    sc = np.where(rd > 0, ru / np.maximum(rd, 1e-300), 1.0)
    return xn * sc * f + cx, yn * sc * f + cy


@pytest.mark.parametrize("k1", [0.0, 0.15, -0.2])
def test_lm_recovers_analytic_projection(k1):
    H, W = 48, 64
    Xi, Xq = noise_free_pair(H, W, k1)
    D = np.zeros((H * W, 4))
    D[:, 0] = 1.0
    Q = np.full(H * W, 3.0)
    idx, q, dg = oracle.match(H, W, Xi, Xq, D, D, Q, Q, diag=True, **{**PAR, "lm_iters": 10})
    pu, pv = project(Xq, H, W, k1)
    inside = (pu > 0.5) & (pu < W - 1.5) & (pv > 0.5) & (pv < H - 1.5) & (Xq[:, 2] > 0)
    assert inside.mean() > 0.8
    err = np.hypot(dg[inside, 0] - pu[inside], dg[inside, 1] - pv[inside])
    assert np.quantile(err, 0.999) <= 1e-2, np.sort(err)[-10:]


def bilinear_np(R, H, W, u, v):
    u0 = min(max(int(np.floor(u)), 0), W - 2)
    v0 = min(max(int(np.floor(v)), 0), H - 2)
    a, b = u - u0, v - v0
    Rg = R.reshape(H, W, 3)
    return ((1 - a) * (1 - b) * Rg[v0, u0] + a * (1 - b) * Rg[v0, u0 + 1] + (1 - a) * b * Rg[v0 + 1, u0]
            + a * b * Rg[v0 + 1, u0 + 1])


def test_lm_no_worse_than_integer_brute_force():
    H, W = 24, 32
    Xi, Xq = noise_free_pair(H, W, 0.1, rot_deg=2.0)
    rng = np.random.default_rng(0)
    Xq = Xq + rng.normal(size=Xq.shape) * 0.01 * Xq[:, 2:3]  # off the ray surface
    D = np.zeros((H * W, 2))
    D[:, 0] = 1
    Q = np.full(H * W, 3.0)
    idx, q, dg = oracle.match(H, W, Xi, Xq, D, D, Q, Q, diag=True, **PAR)
    R = oracle.ray_image(Xi)
    pu, pv = project(Xq, H, W, 0.1)
    inside = (pu > 1) & (pu < W - 2) & (pv > 1) & (pv < H - 2)
    checked = 0
    for n in np.nonzero(inside)[0]:
        t = Xq[n] / np.linalg.norm(Xq[n])
        e_lm = np.sum((bilinear_np(R, H, W, dg[n, 0], dg[n, 1]) - t) ** 2)
        e_int = np.min(np.sum((R - t) ** 2, axis=1))
        assert e_lm <= e_int + 1e-15, (n, e_lm, e_int)
        checked += 1
    assert checked > 300


def test_convergence_within_ten_iterations(tiny_wl):
    w = tiny_wl
    valid_total, conv_total = 0, 0
    for e in range(w.E):
        idx, q, dg = oracle.match_workload(w, e, diag=True, **PAR)
        gm = w.gt_match[w.edge_slice(e)].numpy()
        sel = gm >= 0  # query pixels whose true projection lies in the image
        valid_total += sel.sum()
        conv_total += (dg[sel, 2] < 1e-3).sum()
    assert conv_total / valid_total >= 0.99, conv_total / valid_total


def _gt_agreement(w, e, **par):
    W = int(w.kf_hw[0, 1])
    idx, q = oracle.match_workload(w, e, **{**PAR, **par})
    gm = w.gt_match[w.edge_slice(e)].numpy()
    both = (idx >= 0) & (gm >= 0)
    du = np.abs(idx[both] % W - gm[both] % W)
    dv = np.abs(idx[both] // W - gm[both] // W)
    return both.mean(), np.mean((du == 0) & (dv == 0)), np.mean((du <= 2) & (dv <= 2))


def test_projection_alone_finds_ground_truth(tiny_wl):
    """Without refinement the rounded LM projection is the ground-truth pixel
    (the ray image is the exact camera model; depth noise moves the query
    point off its ray only through parallax)."""
    valid, exact, near = _gt_agreement(tiny_wl, 0, n_levels=0)
    assert valid > 0.9 and exact > 0.95 and near == 1.0


def test_refined_matches_near_ground_truth():
    import synth
    w = synth.tiny(H=192, W=256)
    valid, exact, near = _gt_agreement(w, 0)
    assert valid > 0.9 and near > 0.95


def test_single_level_full_window_is_global_argmax():
    rng = np.random.default_rng(1)
    H, W, d = 12, 16, 8
    X = np.c_[rng.uniform(-1, 1, H * W), rng.uniform(-1, 1, H * W), rng.uniform(2, 4, H * W)]
    Dr = rng.normal(size=(H * W, d))
    Dr /= np.linalg.norm(Dr, axis=1, keepdims=True)
    Dq = rng.normal(size=(H * W, d))
    Dq /= np.linalg.norm(Dq, axis=1, keepdims=True)
    Q = np.full(H * W, 2.0)
    par = {**PAR, "n_levels": 1, "win_radius": max(H, W), "win_dilation": (1, 1, 1, 1), "max_rel_dist3d": 1e9}
    idx, q = oracle.match(H, W, X, X, Dr, Dq, Q, Q, **par)
    ref = np.argmax(Dq @ Dr.T, axis=1)
    assert np.array_equal(idx, ref.astype(np.int32))


def test_self_match_is_identity(tiny_wl):
    w = tiny_wl
    H, W = int(w.kf_hw[0, 0]), int(w.kf_hw[0, 1])
    sl = w.edge_slice(0)
    X, D, Q = w.X_ref[sl], w.D_ref[sl], w.Q_ref[sl]
    Q2 = w.Q_qry[sl]
    idx, q = oracle.match(H, W, X, X, D, D, Q, Q2, **PAR)
    assert np.array_equal(idx, np.arange(H * W, dtype=np.int32))
    assert np.allclose(q, np.sqrt(Q.double().numpy() * Q2.double().numpy()), rtol=1e-15)


def test_invalid_query_points_rejected():
    H, W = 12, 16
    rng = np.random.default_rng(2)
    X = np.c_[rng.uniform(-1, 1, H * W), rng.uniform(-1, 1, H * W), rng.uniform(2, 4, H * W)]
    Xq = X.copy()
    Xq[::7] = 0.0
    Xq[3::11] = np.nan
    D = np.zeros((H * W, 2))
    D[:, 0] = 1
    Q = np.full(H * W, 2.0)
    idx, q = oracle.match(H, W, X, Xq, D, D, Q, Q, **PAR)
    bad = np.zeros(H * W, bool)
    bad[::7] = True
    bad[3::11] = True
    assert np.all(idx[bad] == -1) and np.all(q[bad] == 0)


def test_occluded_points_rejected():
    w = gen_small_tracking()
    occ = w.meta["occluded"].numpy()
    idx, q, dg = oracle.match_workload(w, 0, diag=True, **PAR)
    assert occ.sum() > 0.08 * occ.size
    # an occluded point survives only where refinement moved its match onto a
    # surface that really lies within the 3D threshold
    assert (idx[occ] == -1).mean() >= 0.99
    kept = occ & (idx >= 0)
    assert np.all(dg[kept, 6] <= PAR["max_rel_dist3d"])
    assert (idx[~occ] >= 0).mean() > 0.8


_TRACK = {}


def gen_small_tracking():
    if "w" not in _TRACK:
        import synth
        _TRACK["w"] = synth.tracking(H=96, W=128)
    return _TRACK["w"]


def test_init_from_previous_matches(tiny_wl):
    """Initialising from the converged matches gives the same result as the
    identity initialisation (the ray image is smooth, Sec. 3.2)."""
    w = tiny_wl
    idx0, q0 = oracle.match_workload(w, 1, **PAR)
    gm = w.gt_match[w.edge_slice(1)].numpy()
    init = np.where(gm >= 0, gm, -1).astype(np.int32)
    idx1, q1 = oracle.match_workload(w, 1, init_idx=init, **PAR)
    agree = np.mean(idx0 == idx1)
    assert agree > 0.99, agree


def test_fusion_weighted_average():
    """Sec. 3.3 fusion: with equal confidences and the same prediction twice
    the canonical pointmap becomes the mean of the three; a prediction moved
    by T_kf lands where the transform puts it; invalid predictions change
    nothing; the confidence accumulates."""
    rng = np.random.default_rng(0)
    n = 500
    X0 = np.c_[rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(2, 5, n)]
    C0 = np.full(n, 2.0)
    Xf = X0 + rng.normal(size=X0.shape) * 0.05
    Cf = np.full(n, 2.0)
    I8 = np.array([0, 0, 0, 0, 0, 0, 1.0, 1.0])
    X1, C1 = oracle.fuse(I8, X0, C0, Xf, Cf)
    X2, C2 = oracle.fuse(I8, X1, C1, Xf, Cf)
    assert np.allclose(X2, (X0 + 2 * Xf) / 3, atol=1e-14) and np.allclose(C2, 6.0)
    # a transformed prediction: fusing T X (with T the inverse of a known
    # motion) of the keyframe's own points reproduces them
    T = oracle.sim3_exp(np.array([0.1, -0.2, 0.05, 0.02, 0.03, -0.01, 0.01]))
    Ti = oracle.sim3_inv(T)
    Xp = np.array([oracle.sim3_act(Ti, x) for x in X0])
    X3, C3 = oracle.fuse(T, X0, C0, Xp, np.full(n, 5.0))
    assert np.allclose(X3, X0, atol=1e-12) and np.allclose(C3, 7.0)
    Xbad = Xf.copy()
    Xbad[::3] = 0.0
    Cbad = Cf.copy()
    Cbad[1::3] = -1.0
    X4, C4 = oracle.fuse(I8, X0, C0, Xbad, Cbad)
    untouched = np.zeros(n, bool)
    untouched[::3] = True
    untouched[1::3] = True
    assert np.array_equal(X4[untouched], X0[untouched]) and np.array_equal(C4[untouched], C0[untouched])


def test_match_stats_counts():
    """Sec. 3.4 counts against numpy's unique (brute force)."""
    rng = np.random.default_rng(2)
    idx = rng.integers(-1, 300, 5000).astype(np.int32)
    v, u = oracle.match_stats(idx, 300)
    assert v == int((idx >= 0).sum()) and u == len(np.unique(idx[idx >= 0]))
    assert oracle.match_stats(np.full(10, -1, np.int32), 5) == (0, 0)
