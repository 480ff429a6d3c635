"""Pins of the oracle's linearisation and Gauss-Newton solve (Eq. backend_ray,
Eq. gauss_newton, Sec. 3.5) against properties fixed by the mathematics:

* g = dE/dtau: the gradient it accumulates is the derivative of the Huber cost
  it reports (central differences under expm-based left perturbations);
* at zero residual the Gauss-Newton matrix is the cost Hessian;
* noise-free pixel-exact correspondences: GN recovers the poses to 1e-10;
* the GN optimum equals scipy's least_squares optimum (an independent solver
  and parametrisation) when no Huber weight is active;
* the Cholesky solve equals a dense numpy solve; the first pose stays fixed;
  a graph component not tied to the fixed pose is reported as not PD.
"""
import numpy as np
import pytest
import torch
from scipy.linalg import expm
from scipy.optimize import least_squares
from scipy.spatial.transform import Rotation

import oracle
from synth import gen
from test_oracle_sim3 import hat

PAR = dict(oracle.DEFAULT_PARAMS)


def mat(T):
    return oracle.sim3_matrix(T)


def pose_from_matrix(M):
    s = np.cbrt(np.linalg.det(M[:3, :3]))
    q = Rotation.from_matrix(M[:3, :3] / s).as_quat()  # x y z w
    return np.r_[M[:3, 3], q, s]


def perturbed(T, k, h):
    e = np.zeros(7)
    e[k] = h
    return pose_from_matrix(expm(hat(e)) @ mat(T))


def exact_edge(rng, H=24, W=32):
    """Keyframe i's canonical points and keyframe j's points that map onto them
    exactly under the true T_ij (pixel-exact correspondences, idx = identity)."""
    P = H * W
    Xi = np.c_[rng.uniform(-2, 2, P), rng.uniform(-1.5, 1.5, P), rng.uniform(2, 8, P)]
    Ti = oracle.sim3_exp(rng.normal(size=7) * 0.2)
    Tj = oracle.sim3_exp(rng.normal(size=7) * 0.2)
    Tji = oracle.sim3_mul(oracle.sim3_inv(Tj), Ti)
    Xj = np.array([oracle.sim3_act(Tji, x) for x in Xi])
    idx = np.arange(P, dtype=np.int32)
    q = rng.uniform(2, 10, P)
    return Ti, Tj, Xi, Xj, idx, q


def edge_cost(Ti, Tj, Xi, Xj, idx, q, **par):
    return oracle.linearize_edge(Ti, Tj, Xi, Xj, idx, q, **{**PAR, **par})[2]


@pytest.mark.parametrize("delta", [1.345, 1e9])
def test_gradient_is_derivative_of_cost(tiny_wl, delta):
    w = tiny_wl
    e = 0
    i, j = int(w.edges[e, 0]), int(w.edges[e, 1])
    idx = w.gt_match[w.edge_slice(e)].numpy()
    q = w.Q_qry[w.edge_slice(e)].double().numpy() * 0.5 + 1.0
    Xi, Xj = w.X_canon[w.kf_slice(i)], w.X_canon[w.kf_slice(j)]
    Ti, Tj = w.T_init[i].numpy(), w.T_init[j].numpy()
    H, g, c, nv = oracle.linearize_edge(Ti, Tj, Xi, Xj, idx, q, **{**PAR, "huber_delta": delta})
    assert nv > 1000
    h = 1e-6
    fd = np.zeros(14)
    for k in range(14):
        if k < 7:
            cp = edge_cost(perturbed(Ti, k, h), Tj, Xi, Xj, idx, q, huber_delta=delta)
            cm = edge_cost(perturbed(Ti, k, -h), Tj, Xi, Xj, idx, q, huber_delta=delta)
        else:
            cp = edge_cost(Ti, perturbed(Tj, k - 7, h), Xi, Xj, idx, q, huber_delta=delta)
            cm = edge_cost(Ti, perturbed(Tj, k - 7, -h), Xi, Xj, idx, q, huber_delta=delta)
        fd[k] = (cp - cm) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-5 * np.abs(g).max(), (g, fd)
    # gauge symmetry: moving both poses by the same left perturbation leaves
    # T_ij and so the cost unchanged, hence g_i = -g_j and H_ii = H_jj = -H_ij
    assert np.abs(g[:7] + g[7:]).max() <= 1e-12 * np.abs(g).max()
    assert np.abs(H[:7, :7] + H[:7, 7:]).max() <= 1e-12 * np.abs(H).max()
    assert np.all(np.isfinite(H)) and np.allclose(H, H.T, rtol=1e-12, atol=1e-9 * np.abs(H).max())


def test_gn_matrix_is_cost_hessian_at_zero_residual():
    rng = np.random.default_rng(0)
    Ti, Tj, Xi, Xj, idx, q = exact_edge(rng)
    H, g, c, nv = oracle.linearize_edge(Ti, Tj, Xi, Xj, idx, q, **PAR)
    assert c < 1e-20 and np.abs(g).max() < 1e-6
    h = 1e-5
    Hfd = np.zeros((14, 14))
    for k in range(14):
        def grad(sgn):
            if k < 7:
                return oracle.linearize_edge(perturbed(Ti, k, sgn * h), Tj, Xi, Xj, idx, q, **PAR)[1]
            return oracle.linearize_edge(Ti, perturbed(Tj, k - 7, sgn * h), Xi, Xj, idx, q, **PAR)[1]
        Hfd[:, k] = (grad(1) - grad(-1)) / (2 * h)
    assert np.abs(H - Hfd).max() <= 1e-5 * np.abs(H).max()


def exact_graph(rng, N=4, H=24, W=32):
    """Noise-free graph: every keyframe sees the same random point set through
    its own pose; idx = identity on every edge."""
    P = H * W
    Xw = np.c_[rng.uniform(-2, 2, P), rng.uniform(-1.5, 1.5, P), rng.uniform(3, 8, P)]
    T = [np.array([0, 0, 0, 0, 0, 0, 1.0, 1.0])]
    for k in range(1, N):
        T.append(oracle.sim3_exp(np.r_[rng.normal(size=3) * 0.2, rng.normal(size=3) * 0.05, 0.0]))
    X = [np.array([oracle.sim3_act(oracle.sim3_inv(T[k]), x) for x in Xw]) for k in range(N)]
    edges = [(k, k + 1) for k in range(N - 1)] + [(k + 1, k) for k in range(N - 1)] + [(0, N - 1)]
    E = len(edges)
    kf_off = np.arange(N + 1) * P
    e_off = np.arange(E + 1) * P
    idx = np.tile(np.arange(P, dtype=np.int32), E)
    q = rng.uniform(2, 10, E * P)
    return np.array(T), np.concatenate(X), np.array(edges, dtype=np.int32), kf_off, e_off, idx, q


def test_exact_pose_recovery():
    rng = np.random.default_rng(1)
    T_gt, X, edges, kf_off, e_off, idx, q = exact_graph(rng)
    N = T_gt.shape[0]
    T0 = T_gt.copy()
    for k in range(1, N):
        T0[k] = oracle.sim3_mul(oracle.sim3_exp(np.r_[rng.normal(size=3) * 0.05, rng.normal(size=3) * 0.03, 0.05]),
                                T_gt[k])
    st, T, hist, done = oracle.gauss_newton(N, edges, kf_off, e_off, X, idx, q, T0, 30, **PAR)
    assert st == 0
    assert np.array_equal(T[0], T0[0])  # the fixed pose is untouched
    for k in range(N):
        err = oracle.sim3_log(oracle.sim3_mul(T[k], oracle.sim3_inv(T_gt[k])))
        assert np.abs(err).max() <= 1e-10, (k, err)
    assert hist[0] > hist[-1]


def test_gn_optimum_equals_scipy_least_squares(tiny_wl):
    """Weighted least squares without active Huber weights: the GN fixed point
    equals scipy's trust-region least-squares optimum over poses T_k =
    expm(hat(tau_k)) T_k^0 with pose 0 fixed."""
    w = tiny_wl
    N = w.N
    e_sel = range(w.E)
    rng = np.random.default_rng(2)
    sub = []
    for e in e_sel:
        gm = w.gt_match[w.edge_slice(e)].numpy()
        ok = np.nonzero(gm >= 0)[0]
        sub.append(rng.choice(ok, 300, replace=False))
    # a compact problem: per edge 300 pixels with their ground-truth matches
    X = w.X_canon.double().numpy()
    edges = w.edges.numpy()
    q_all = []
    rows = []
    for e, pix in zip(e_sel, sub):
        i, j = edges[e]
        gm = w.gt_match[w.edge_slice(e)].numpy()
        qv = rng.uniform(2, 10, len(pix))
        for n, qq in zip(pix, qv):
            rows.append((e, i, j, X[w.kf_off[j] + n], X[w.kf_off[i] + gm[n]], qq))
        q_all.append(qv)
    sr, sd = PAR["sigma_ray"], PAR["sigma_dist"]
    M0 = [mat(w.T_init[k].numpy()) for k in range(N)]

    def poses(z):
        return [M0[0]] + [expm(hat(z[7 * (k - 1):7 * k])) @ M0[k] for k in range(1, N)]

    def resid(z):
        Ms = poses(z)
        out = []
        for e, i, j, xj, xi, qq in rows:
            x = (np.linalg.inv(Ms[i]) @ Ms[j] @ np.r_[xj, 1.0])[:3]
            r = x / np.linalg.norm(x) - xi / np.linalg.norm(xi)
            rd = np.linalg.norm(x) - np.linalg.norm(xi)
            out.append(np.r_[np.sqrt(qq) / sr * r, np.sqrt(qq) / sd * rd])
        return np.concatenate(out)

    sol = least_squares(resid, np.zeros(7 * (N - 1)), method="trf", jac="3-point", xtol=1e-15, ftol=1e-15, gtol=1e-15)
    M_ls = poses(sol.x)
    # the same problem through the oracle: pools of 300 pixels per edge
    P = 300
    E = len(rows) // P
    Xj_pool = np.zeros((E * P, 3))
    Xi_pool = np.zeros((E * P, 3))
    for r_, (e, i, j, xj, xi, qq) in enumerate(rows):
        Xj_pool[r_], Xi_pool[r_] = xj, xi
    # the oracle on the same residuals: per-edge linearisation of the gathered
    # pixel lists (idx = identity into them), then its solve
    T = np.array([w.T_init[k].numpy() for k in range(N)])
    qv = np.array([r_[5] for r_ in rows])
    for it in range(30):
        H14, g14 = [], []
        for e in range(E):
            i, j = edges[e]
            sl = slice(e * P, (e + 1) * P)
            Hb, gb, _, _ = oracle.linearize_edge(T[i], T[j], Xi_pool[sl], Xj_pool[sl], np.arange(P, dtype=np.int32),
                                                 qv[sl], **{**PAR, "huber_delta": 1e9, "q_min": 0.0})
            H14.append(Hb)
            g14.append(gb)
        st, T, tau = oracle.gn_solve(N, edges[:E], np.array(H14), np.array(g14), T)
        assert st == 0
    for k in range(N):
        err = np.abs(mat(T[k]) - M_ls[k]).max()
        assert err <= 1e-8, (k, err)


def random_blocks(rng, N, edges):
    H14, g14 = [], []
    for _ in edges:
        J = rng.normal(size=(40, 14))
        H14.append(J.T @ J)
        g14.append(rng.normal(size=14))
    return np.array(H14), np.array(g14)


def test_solve_matches_dense_numpy():
    rng = np.random.default_rng(3)
    N = 6
    edges = np.array([(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0), (1, 4), (4, 1)], dtype=np.int32)
    H14, g14 = random_blocks(rng, N, edges)
    A = np.zeros((7 * N, 7 * N))
    g = np.zeros(7 * N)
    for e, (i, j) in enumerate(edges):
        ids = np.r_[np.arange(7 * i, 7 * i + 7), np.arange(7 * j, 7 * j + 7)]
        A[np.ix_(ids, ids)] += H14[e]
        g[ids] += g14[e]
    keep = np.arange(7, 7 * N)
    tau_np = np.linalg.solve(A[np.ix_(keep, keep)], -g[keep])
    T0 = np.array([oracle.sim3_exp(rng.normal(size=7) * 0.3) for _ in range(N)])
    st, T, tau = oracle.gn_solve(N, edges, H14, g14, T0)
    assert st == 0
    assert np.abs(tau[1:].reshape(-1) - tau_np).max() <= 1e-10 * max(1.0, np.abs(tau_np).max())
    assert np.all(tau[0] == 0) and np.array_equal(T[0], T0[0])
    for k in range(1, N):
        assert np.abs(mat(T[k]) - expm(hat(tau[k])) @ mat(T0[k])).max() <= 1e-12 * np.abs(mat(T[k])).max()
    # the residual of the solved system
    assert np.linalg.norm(A[np.ix_(keep, keep)] @ tau[1:].reshape(-1) + g[keep]) <= 1e-10 * np.linalg.norm(g)


def test_disconnected_graph_is_not_pd():
    rng = np.random.default_rng(4)
    N = 4
    edges = np.array([(0, 1), (2, 3)], dtype=np.int32)
    T0 = np.array([oracle.sim3_exp(rng.normal(size=7) * 0.3) for _ in range(N)])
    Ti, Tj, Xi, Xj, idx, q = exact_edge(rng)
    H14, g14 = [], []
    for (i, j) in edges:
        Hb, gb, _, _ = oracle.linearize_edge(T0[i], T0[j], Xi, Xj, idx, q, **PAR)
        H14.append(Hb)
        g14.append(gb)
    st, T, tau = oracle.gn_solve(N, edges, np.array(H14), np.array(g14), T0)
    assert st == 3
    assert np.array_equal(T, T0)


def test_cost_gradient_wrt_points_and_confidence(tiny_wl):
    """dE/dX_canon and dE/dq of the oracle's adjoint equal central differences
    of its cost (fixed poses and matches)."""
    w = tiny_wl
    rng = np.random.default_rng(5)
    X = w.X_canon.double().numpy().copy()
    idx = w.gt_match.numpy()
    q = w.Q_qry.double().numpy() * 0.3 + 1.0
    T = w.T_init.numpy()
    edges = w.edges.numpy()
    args = (w.N, edges, w.kf_off.numpy(), w.e_off.numpy())
    c0, dX, dq = oracle.cost_grad(*args, T, X, idx, q, **PAR)
    for _ in range(12):
        p = int(rng.integers(0, X.shape[0]))
        k = int(rng.integers(0, 3))
        if np.abs(dX[p, k]) == 0:
            continue
        h = 1e-6 * max(1.0, abs(X[p, k]))
        Xp, Xm = X.copy(), X.copy()
        Xp[p, k] += h
        Xm[p, k] -= h
        fd = (oracle.cost_grad(*args, T, Xp, idx, q, **PAR)[0] - oracle.cost_grad(*args, T, Xm, idx, q, **PAR)[0]) / (2 * h)
        assert abs(fd - dX[p, k]) <= 1e-5 * max(1.0, abs(dX[p, k])), (p, k, fd, dX[p, k])
    nz = np.nonzero(dq)[0]
    for p in rng.choice(nz, 8, replace=False):
        h = 1e-6 * q[p]
        qp, qm = q.copy(), q.copy()
        qp[p] += h
        qm[p] -= h
        fd = (oracle.cost_grad(*args, T, X, idx, qp, **PAR)[0] - oracle.cost_grad(*args, T, X, idx, qm, **PAR)[0]) / (2 * h)
        assert abs(fd - dq[p]) <= 1e-5 * max(1.0, abs(dq[p])), (p, fd, dq[p])
    # the cost equals the sum of the per-edge linearisation costs
    tot = 0.0
    for e in range(w.E):
        i, j = edges[e]
        tot += oracle.linearize_edge(T[i], T[j], X[w.kf_slice(i)], X[w.kf_slice(j)], idx[w.edge_slice(e)],
                                     q[w.edge_slice(e)], **PAR)[2]
    assert abs(tot - c0) <= 1e-12 * abs(c0)


def test_step_gradient_against_finite_differences():
    """The oracle's adjoint of one Gauss-Newton step (complex step on the
    per-match terms, dL = -b^T (dH tau + dg)) equals central differences of
    L(X, q) = c E(X, q) + a . tau(X, q), tau the oracle's own step."""
    rng = np.random.default_rng(6)
    import synth
    w = synth.global_graph(N=4, n_pairs=5, H=12, W=16, seed=5)
    N = w.N
    edges = w.edges.numpy()
    kf_off, e_off = w.kf_off.numpy(), w.e_off.numpy()
    X = w.X_canon.double().numpy().copy()
    idx = w.gt_match.numpy()
    q = w.Q_qry.double().numpy() * 0.5 + 1.0
    T = w.T_init.numpy()
    a = rng.normal(size=(N, 7))
    a[0] = 0.0
    c = 0.7
    st, dX, dq, tau = oracle.gn_step_grad(N, edges, kf_off, e_off, T, X, idx, q, dL_dtau=a, dL_dcost=c, **PAR)
    assert st == 0

    def L(Xv, qv):
        s2, _, _, t2 = oracle.gn_step_grad(N, edges, kf_off, e_off, T, Xv, idx, qv, dL_dtau=a, dL_dcost=1.0, **PAR)
        cost = oracle.cost_grad(N, edges, kf_off, e_off, T, Xv, idx, qv, **PAR)[0]
        return c * cost + float((a * t2).sum())

    used = np.nonzero((idx >= 0) & (q > PAR["q_min"]))[0]
    checked = 0
    for p in rng.choice(X.shape[0], 40, replace=False):
        k = int(rng.integers(0, 3))
        if dX[p, k] == 0.0:
            continue
        h = 1e-5 * max(1.0, abs(X[p, k]))
        Xp, Xm = X.copy(), X.copy()
        Xp[p, k] += h
        Xm[p, k] -= h
        fd = (L(Xp, q) - L(Xm, q)) / (2 * h)
        assert abs(fd - dX[p, k]) <= 2e-5 * max(1.0, abs(dX[p, k])), (p, k, fd, dX[p, k])
        checked += 1
    for p in rng.choice(used, 10, replace=False):
        h = 1e-6 * q[p]
        qp, qm = q.copy(), q.copy()
        qp[p] += h
        qm[p] -= h
        fd = (L(X, qp) - L(X, qm)) / (2 * h)
        assert abs(fd - dq[p]) <= 2e-5 * max(1.0, abs(dq[p])), (p, fd, dq[p])
    assert checked >= 10
