"""Gradients through whole Gauss-Newton steps, poses included
(mslam_gn_step_backward and the chained GNStep autograd function), against
central differences of the FP64 oracle's own Gauss-Newton steps (dense FP64
Cholesky, literal 14 x 14 blocks, Sim(3) retraction) on the same stored
values.  The loss mixes every output of the steps:
  L = sum W * T_final + sum_k a_k . tau_k + c sum_k E_g(T_k),
so that the gradient runs through the retraction, the step and the cost.
Matches and the q_min mask are held fixed; perturbed confidences stay away
from q_min.  Pose directions are tangent: T -> Exp(h e_j) T."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available()
    from paper_2412_12392_gb300 import build
    build.build()
    import paper_2412_12392_gb300 as M
    return M


def oracle_loss(w, X, q, T0, steps, Wt, a, c, par):
    """L of `steps` oracle Gauss-Newton steps from T0 (numpy FP64)."""
    T = np.array(T0, dtype=np.float64)
    edges = w.edges.numpy()
    L = 0.0
    for k in range(steps):
        Hs, gs, cost = [], [], 0.0
        for e in range(w.E):
            i, j = int(edges[e, 0]), int(edges[e, 1])
            sl = slice(int(w.e_off[e]), int(w.e_off[e + 1]))
            Hb, gb, ce, _ = oracle.linearize_edge(T[i], T[j], X[int(w.kf_off[i]):int(w.kf_off[i + 1])],
                                                  X[int(w.kf_off[j]):int(w.kf_off[j + 1])], w._idx[sl], q[sl], **par)
            Hs.append(Hb)
            gs.append(gb)
            cost += ce
        st, T, tau = oracle.gn_solve(w.N, edges, np.array(Hs), np.array(gs), T)
        assert st == 0
        L += float((a[k] * tau).sum()) + c * cost
    return L + float((Wt * T).sum())


def gpu_grad(M, w, plan, P, X, q, T0, steps, Wt, a, c):
    from paper_2412_12392_gb300.autograd import gn_unrolled
    Xg = X.clone().requires_grad_(True)
    qg = q.clone().requires_grad_(True)
    Tg = T0.clone().requires_grad_(True)
    T, taus, costs = gn_unrolled(Xg, qg, Tg, plan, P, w._idx_dev, steps)
    L = (T * torch.from_numpy(Wt).cuda()).sum() + c * sum(costs)
    for k in range(steps):
        L = L + (taus[k] * torch.from_numpy(a[k]).cuda()).sum()
    L.backward()
    return float(L.detach()), Xg.grad.double().cpu().numpy(), qg.grad.double().cpu().numpy(), Tg.grad.cpu().numpy()


def setup(w, dtype, seed):
    ws = w.to_storage(dtype)
    ws._idx = ws.gt_match.numpy()
    rng = np.random.default_rng(seed)
    Wt = rng.normal(size=(w.N, 8)) * 0.1
    a = rng.normal(size=(3, w.N, 7)) * 1e-2
    a[:, 0] = 0.0
    return ws, rng, Wt, a


def check_against_fd(M, w, dtype, steps, n_x=12, n_q=8, poses=(1, 2), seed=0, tol=2e-4, tol_pose=2e-4):
    ws, rng, Wt, a = setup(w, dtype, seed)
    P = M.default_params()
    par = M.params_dict(P)
    c = 0.3
    plan = M.Plan(ws.kf_hw.numpy(), ws.edges.numpy())
    Xd, qd = ws.X_canon.cuda(), ws.Q_qry.cuda()
    ws._idx_dev = ws.gt_match.cuda()
    T0 = ws.T_init.cuda()
    L_gpu, dX, dq, dT = gpu_grad(M, ws, plan, P, Xd, qd, T0, steps, Wt, a, c)
    X64 = ws.X_canon.double().numpy().copy()
    q64 = ws.Q_qry.double().numpy().copy()
    T64 = ws.T_init.numpy().copy()
    L_ref = oracle_loss(ws, X64, q64, T64, steps, Wt, a, c, par)
    assert abs(L_gpu - L_ref) <= 1e-4 * max(1.0, abs(L_ref)), (L_gpu, L_ref)
    # sampled point coordinates of matched pixels (query side and reference side)
    used = np.nonzero((ws._idx >= 0) & (q64 > P.q_min + 0.05))[0]
    fd_x, gp_x = [], []
    for n in rng.choice(used, n_x, replace=False):
        e = int(np.searchsorted(ws.e_off.numpy(), n, side="right") - 1)
        j = int(ws.edges[e, 1])
        pix = int(ws.kf_off[j]) + (n - int(ws.e_off[e]))
        k = int(rng.integers(3))
        h = 1e-4
        Xp, Xm = X64.copy(), X64.copy()
        Xp[pix, k] += h
        Xm[pix, k] -= h
        fd_x.append((oracle_loss(ws, Xp, q64, T64, steps, Wt, a, c, par) -
                     oracle_loss(ws, Xm, q64, T64, steps, Wt, a, c, par)) / (2 * h))
        gp_x.append(dX[pix, k])
    fd_q, gp_q = [], []
    for n in rng.choice(used, n_q, replace=False):
        h = 1e-4 * q64[n]
        qp, qm = q64.copy(), q64.copy()
        qp[n] += h
        qm[n] -= h
        fd_q.append((oracle_loss(ws, X64, qp, T64, steps, Wt, a, c, par) -
                     oracle_loss(ws, X64, qm, T64, steps, Wt, a, c, par)) / (2 * h))
        gp_q.append(dq[n])
    fd_t, gp_t = [], []
    for kf in poses:
        for jdir in range(7):
            h = 1e-6
            e = np.zeros(7)
            e[jdir] = h
            Tp, Tm = T64.copy(), T64.copy()
            Tp[kf] = oracle.sim3_mul(oracle.sim3_exp(e), T64[kf])
            Tm[kf] = oracle.sim3_mul(oracle.sim3_exp(-e), T64[kf])
            fd_t.append((oracle_loss(ws, X64, q64, Tp, steps, Wt, a, c, par) -
                         oracle_loss(ws, X64, q64, Tm, steps, Wt, a, c, par)) / (2 * h))
            # the GPU's embedding gradient along the same tangent direction
            gp_t.append(float(dT[kf] @ ((Tp[kf] - Tm[kf]) / (2 * h))))
        # no component along the quaternion's norm direction
        assert abs(float(dT[kf, 3:7] @ T64[kf, 3:7])) <= 1e-9 * max(1.0, np.abs(dT[kf]).max())
    for name, g, f in (("X", gp_x, fd_x), ("q", gp_q, fd_q), ("T", gp_t, fd_t)):
        g, f = np.array(g), np.array(f)
        err = np.abs(g - f).max() / max(np.abs(f).max(), 1e-300)
        print(f"{w.name} {dtype} steps={steps} d{name}: max |gpu - fd| / max |fd| = {err:.2e} over {len(f)}")
        assert err <= (tol_pose if name == "T" else tol), (name, g, f)


def test_one_step_with_poses(M):
    w = synth.global_graph(N=5, n_pairs=7, H=24, W=32, seed=5)
    check_against_fd(M, w, torch.float32, 1, poses=(0, 1, 3))


def test_three_unrolled_steps_differentiation_graph(M):
    """The differentiation workload's graph (32 keyframes, 96 edges) at
    reduced resolution, FP32 storage, three chained steps."""
    w = synth.differentiation(H=24, W=32)
    check_against_fd(M, w, torch.float32, 3, n_x=10, n_q=6, poses=(1, 17))


def test_three_unrolled_steps_fp16(M):
    """FP16-stored pointmaps and confidences (FP32 math): gradients with
    respect to the stored values against the oracle on the dequantised ones.
    autograd returns a tensor's gradient in the tensor's dtype; gn_unrolled
    sums the steps' point and confidence gradients in FP32 and the result is
    rounded to FP16 once (at most 2^-12 of an entry): the bar for them is
    5e-4 of the largest entry."""
    w = synth.differentiation(H=24, W=32)
    check_against_fd(M, w, torch.float16, 3, n_x=8, n_q=4, poses=(5,), seed=1, tol=5e-4, tol_pose=2e-4)


def near_kink_points(w, X64, idx, q, Ts, par, band=1e-3):
    """Canonical points that take part in a match whose whitened ray or
    distance residual lies within `band` (relative) of the Huber threshold
    at any of the pose sets Ts (FP64).  There the step's derivative jumps
    (the weight's derivative is 0 below the threshold and -h / (2 e^2)
    above), so the adjoint takes the side its FP32 evaluation lands on and
    a central difference straddles the kink."""
    edges, kf_off, e_off = w.edges.numpy(), w.kf_off.numpy(), w.e_off.numpy()
    idx, q = np.asarray(idx), np.asarray(q, dtype=np.float64)
    d2 = par["huber_delta"] ** 2
    mark = np.zeros(X64.shape[0], dtype=bool)
    for T in Ts:
        for e in range(w.E):
            i, j = int(edges[e, 0]), int(edges[e, 1])
            sl = slice(int(e_off[e]), int(e_off[e + 1]))
            m, qe = idx[sl], q[sl]
            n = np.nonzero((m >= 0) & (qe > par["q_min"]))[0]
            Mx = oracle.sim3_matrix(oracle.sim3_mul(oracle.sim3_inv(T[i]), T[j]))
            x = X64[kf_off[j] + n] @ Mx[:3, :3].T + Mx[:3, 3]
            y = X64[kf_off[i] + m[n]]
            dx, dy = np.linalg.norm(x, axis=1), np.linalg.norm(y, axis=1)
            rr = x / dx[:, None] - y / dy[:, None]
            er2 = qe[n] / par["sigma_ray"] ** 2 * (rr * rr).sum(1)
            ed2 = qe[n] / par["sigma_dist"] ** 2 * (dx - dy) ** 2
            bad = (np.abs(er2 / d2 - 1) < band) | (np.abs(ed2 / d2 - 1) < band)
            mark[kf_off[j] + n[bad]] = True
            mark[kf_off[i] + m[n[bad]]] = True
    return mark


def test_three_unrolled_steps_full_size_directional(M):
    """The differentiation workload at full size (32 keyframes, 96 edges,
    512 x 384, FP16 storage): the gradient of L = sum W * T_3 + c sum_k E_g(T_k)
    through three chained steps, with respect to every canonical point and
    every pose, along a random direction v, against the central difference
    of the oracle's own three Gauss-Newton steps (FP64, dense Cholesky) on
    the dequantised values: <grad, v> = (L(x + h v) - L(x - h v)) / 2h.
    Pose directions are tangent (T_k -> Exp(h v_k) T_k).  The point
    direction leaves out the points of matches within 1e-3 of the Huber
    threshold at any of the three linearisation poses (about 16,000 of
    6.3 M): there the step is not differentiable, and h = 1e-6 keeps every
    other match on its side of the threshold.  The points are an FP32 leaf
    stored as FP16 for the kernels (gn_unrolled's `storage`), so the point
    gradients stay in FP32: most of them lie below 1e-4, in FP16's subnormal
    range.  The bar, 1e-3, is the central difference's own spread: across
    h = 1e-7 .. 1e-5 it moves by up to 2e-4 of its value (matches that cross
    the threshold outside the excluded band)."""
    from paper_2412_12392_gb300.autograd import gn_unrolled
    w = synth.differentiation(device="cuda").to_storage(torch.float16)
    P = M.default_params()
    par = M.params_dict(P)
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), opts={"lin_form": 1})
    rng = np.random.default_rng(11)
    Wt = rng.normal(size=(w.N, 8)) * 0.1
    c = 0.3
    X = w.X_canon.float().requires_grad_(True)
    T0 = w.T_init.cuda().clone().requires_grad_(True)
    idx = w.gt_match
    q = w.Q_qry
    T, taus, costs = gn_unrolled(X, q, T0, plan, P, idx, 3, storage=torch.float16)
    L = (T * torch.from_numpy(Wt).cuda()).sum() + c * sum(costs)
    L.backward()
    assert X.grad.dtype == torch.float32
    gX = X.grad.double().cpu().numpy()
    gT = T0.grad.cpu().numpy()
    # the oracle's L: three steps of its Gauss-Newton (costs at the start of each)
    X64 = w.X_canon.double().cpu().numpy()
    T64 = w.T_init.numpy().copy()
    idx_c, q_c = idx.cpu(), q.cpu()
    args = (w.N, w.edges.numpy(), w.kf_off.numpy(), w.e_off.numpy())

    def L_ref(Xv, Tv, steps=3):
        st, T3, hist, done = oracle.gauss_newton(*args, Xv, idx_c, q_c, Tv, steps, **par)
        assert st == 0 and done == steps
        return float((Wt * T3).sum()) + c * float(hist.sum()), T3

    L0, _ = L_ref(X64, T64)
    assert abs(float(L) - L0) <= 1e-4 * abs(L0), (float(L), L0)
    Ts = [T64, L_ref(X64, T64, 1)[1], L_ref(X64, T64, 2)[1]]
    kink = near_kink_points(w, X64, idx_c.numpy(), q_c.double().numpy(), Ts, par)
    print(f"full size: {int(kink.sum())} of {len(kink)} points touch a match near the Huber threshold")
    assert kink.sum() < 1e-2 * len(kink)
    # direction over the points
    vX = rng.normal(size=X64.shape)
    vX[kink] = 0.0
    h = 1e-6
    fd = (L_ref(X64 + h * vX, T64)[0] - L_ref(X64 - h * vX, T64)[0]) / (2 * h)
    an = float((gX * vX).sum())
    print(f"full size, points: <grad, v> {an:.6e}, central difference {fd:.6e}, rel {abs(an - fd) / abs(fd):.2e}")
    assert abs(an - fd) <= 1e-3 * abs(fd)
    # direction over the poses (tangent), the fixed first pose included
    vT = rng.normal(size=(w.N, 7)) * np.r_[0.01, 0.01, 0.01, 0.002, 0.002, 0.002, 0.002]
    ht = 1e-5
    Tp, Tm, dT = T64.copy(), T64.copy(), np.zeros_like(T64)
    for k in range(w.N):
        Tp[k] = oracle.sim3_mul(oracle.sim3_exp(ht * vT[k]), T64[k])
        Tm[k] = oracle.sim3_mul(oracle.sim3_exp(-ht * vT[k]), T64[k])
        dT[k] = (Tp[k] - Tm[k]) / (2 * ht)
    fdT = (L_ref(X64, Tp)[0] - L_ref(X64, Tm)[0]) / (2 * ht)
    anT = float((gT * dT).sum())
    print(f"full size, poses: <grad, v> {anT:.6e}, central difference {fdT:.6e}, rel {abs(anT - fdT) / abs(fdT):.2e}")
    assert abs(anT - fdT) <= 1e-3 * abs(fdT)
