"""Pins of the oracle's residuals and analytic Jacobians (Supp. S1.1-S1.4):
central finite differences of the residual under left perturbations
Exp(h e_k) o T computed with scipy's expm on 4x4 matrices (independent of the
oracle's Lie maps), plus the structural facts the supplement derives."""
import numpy as np
from scipy.linalg import expm

import oracle
from test_oracle_sim3 import hat


def mat(T):
    return oracle.sim3_matrix(T)


def residual_np(Mi, Mj, Xj, Xi):
    """r = psi(T_ij X_j) - psi(X_i), r_d = |T_ij X_j| - |X_i| with matrices."""
    x = (np.linalg.inv(Mi) @ Mj @ np.r_[Xj, 1.0])[:3]
    return np.r_[x / np.linalg.norm(x) - Xi / np.linalg.norm(Xi), np.linalg.norm(x) - np.linalg.norm(Xi)]


def fd_jacobian(Ti, Tj, Xj, Xi, h=1e-6):
    Mi, Mj = mat(Ti), mat(Tj)
    J = np.zeros((4, 14))
    for k in range(14):
        e = np.zeros(7)
        e[k % 7] = h
        P, Mn = expm(hat(e)), expm(hat(-e))
        if k < 7:
            rp, rm = residual_np(P @ Mi, Mj, Xj, Xi), residual_np(Mn @ Mi, Mj, Xj, Xi)
        else:
            rp, rm = residual_np(Mi, P @ Mj, Xj, Xi), residual_np(Mi, Mn @ Mj, Xj, Xi)
        J[:, k] = (rp - rm) / (2 * h)
    return J


def test_residual_and_jacobian_vs_fd():
    rng = np.random.default_rng(0)
    for _ in range(30):
        Ti = oracle.sim3_exp(rng.normal(size=7) * 0.3)
        Tj = oracle.sim3_exp(rng.normal(size=7) * 0.3)
        Xj = rng.normal(size=3) + np.array([0, 0, 4.0])
        Xi = rng.normal(size=3) + np.array([0, 0, 4.0])
        ok, r, J = oracle.residual_jacobian(Ti, Tj, Xj, Xi)
        assert ok
        assert np.allclose(r, residual_np(mat(Ti), mat(Tj), Xj, Xi), atol=1e-13)
        Jfd = fd_jacobian(Ti, Tj, Xj, Xi)
        assert np.abs(J - Jfd).max() <= 1e-7 * max(1.0, np.abs(J).max()), np.abs(J - Jfd).max()


def test_relative_jacobian_structure():
    """With T_i = I the j-block is the relative Jacobian: ray rows are
    [(I - u u^T)/d, -[x]x/d, 0] (scale column zero, Supp. S1.2) and the
    distance row is [u^T, 0, d] (Eq. dist_jac)."""
    rng = np.random.default_rng(1)
    I8 = np.array([0, 0, 0, 0, 0, 0, 1.0, 1.0])
    for _ in range(10):
        Tj = oracle.sim3_exp(rng.normal(size=7) * 0.3)
        Xj = rng.normal(size=3) + np.array([0, 0, 3.0])
        Xi = rng.normal(size=3) + np.array([0, 0, 3.0])
        ok, r, J = oracle.residual_jacobian(I8, Tj, Xj, Xi)
        Jr = J[:, 7:]
        assert np.allclose(J[:, :7], -Jr, atol=0)
        x = oracle.sim3_act(Tj, Xj)
        d = np.linalg.norm(x)
        u = x / d
        S = np.array([[0, -x[2], x[1]], [x[2], 0, -x[0]], [-x[1], x[0], 0]])
        assert np.abs(Jr[:3, 6]).max() <= 1e-15
        assert np.allclose(Jr[:3, 0:3], (np.eye(3) - np.outer(u, u)) / d, atol=1e-15)
        assert np.allclose(Jr[:3, 3:6], -S / d, atol=1e-14)
        assert np.allclose(Jr[3], np.r_[u, 0, 0, 0, d], atol=1e-14)
        # J_psi^T J_psi = [[P/d^2, -[x]x/d^2], [[x]x/d^2, P]]
        JtJ = Jr[:3, :6].T @ Jr[:3, :6]
        P = np.eye(3) - np.outer(u, u)
        ref = np.block([[P / d ** 2, -S / d ** 2], [S / d ** 2, P]])
        assert np.allclose(JtJ, ref, atol=1e-13)


def test_adjoint_mapping_of_global_jacobian():
    """dr/dT_i = -(dr/dT_ij) Ad_{T_i^-1}, dr/dT_j = (dr/dT_ij) Ad_{T_i^-1}
    (Supp. S1.4): the two blocks are negatives of each other."""
    rng = np.random.default_rng(2)
    Ti = oracle.sim3_exp(rng.normal(size=7) * 0.5)
    Tj = oracle.sim3_exp(rng.normal(size=7) * 0.5)
    ok, r, J = oracle.residual_jacobian(Ti, Tj, np.array([0.3, -0.2, 3.0]), np.array([0.1, 0.1, 2.5]))
    assert np.allclose(J[:, :7], -J[:, 7:], atol=0)


def test_ray_error_identity():
    """|psi_1 - psi_2|^2 = 2 (1 - cos theta), cos theta = psi_1^T psi_2 (Eq. ray_error)."""
    rng = np.random.default_rng(4)
    X = rng.normal(size=(1000, 3)) * rng.uniform(0.1, 10, size=(1000, 1))
    R = oracle.ray_image(X)
    a, b = R[:500], R[500:]
    lhs = ((a - b) ** 2).sum(1)
    rhs = 2 * (1 - (a * b).sum(1))
    assert np.abs(lhs - rhs).max() <= 1e-15 * 8
    assert np.allclose(np.linalg.norm(R, axis=1), 1.0, atol=1e-15)


def test_ray_image_invalid_points_are_zero():
    X = np.array([[0.0, 0.0, 0.0], [np.nan, 1.0, 1.0], [1.0, np.inf, 0.0], [0.0, 3.0, 4.0]])
    R = oracle.ray_image(X)
    assert np.all(R[:3] == 0)
    assert np.allclose(R[3], [0, 0.6, 0.8])
