"""Pins of the oracle's Sim(3) maps (Eq. 1, Supp. S1 and S1.4) against the
matrix exponential (scipy's expm, a library routine independent of the
oracle's closed forms) and against group identities."""
import numpy as np
import pytest
from scipy.linalg import expm, logm

import oracle


def hat(tau):
    A = np.zeros((4, 4))
    p = tau[3:6]
    A[:3, :3] = np.array([[0, -p[2], p[1]], [p[2], 0, -p[0]], [-p[1], p[0], 0]]) + tau[6] * np.eye(3)
    A[:3, 3] = tau[:3]
    return A


TAUS = [
    np.array([0.1, -0.2, 0.3, 0.4, -0.5, 0.6, 0.2]),
    np.array([0.1, 0.2, 0.3, 0.0, 0.0, 0.0, 0.0]),            # theta = 0, sigma = 0
    np.array([0.3, 0.2, -0.1, 1e-7, -2e-7, 3e-8, 0.0]),       # tiny rotation
    np.array([0.3, 0.2, -0.1, 0.5, 0.2, -0.1, 1e-9]),         # tiny scale
    np.array([0.3, 0.2, -0.1, 2e-5, 1e-5, -1e-5, 3e-6]),      # both tiny
    np.array([-1.0, 2.0, 0.5, 2.0, -1.0, 0.5, -1.5]),         # large
    np.array([0.0, 0.0, 0.0, 3.0, 0.0, 0.0, 0.0]),            # near pi
    np.array([0.5, 0.5, 0.5, 1e-4, 0, 0, 2.0]),               # branch edge
]


@pytest.mark.parametrize("k", range(len(TAUS)))
def test_exp_is_matrix_exponential(k):
    tau = TAUS[k]
    M = oracle.sim3_matrix(oracle.sim3_exp(tau))
    E = expm(hat(tau))
    assert np.abs(M - E).max() <= 1e-13 * max(1.0, np.abs(E).max())


def test_exp_random_against_expm():
    rng = np.random.default_rng(7)
    for _ in range(200):
        tau = rng.normal(size=7) * rng.choice([1e-6, 1e-3, 0.1, 1.0])
        M = oracle.sim3_matrix(oracle.sim3_exp(tau))
        E = expm(hat(tau))
        assert np.abs(M - E).max() <= 1e-13 * max(1.0, np.abs(E).max())


@pytest.mark.parametrize("k", range(len(TAUS) - 1))
def test_log_exp_round_trip(k):
    tau = TAUS[k]
    back = oracle.sim3_log(oracle.sim3_exp(tau))
    assert np.abs(back - tau).max() <= 1e-12


def test_log_matches_matrix_logarithm():
    rng = np.random.default_rng(3)
    for _ in range(20):
        tau = rng.normal(size=7) * 0.4
        T = oracle.sim3_exp(tau)
        L = np.real(logm(oracle.sim3_matrix(T)))
        assert np.abs(hat(oracle.sim3_log(T)) - L).max() <= 1e-10


def random_pose(rng, scale=1.0):
    return oracle.sim3_exp(rng.normal(size=7) * scale)


def test_mul_inv_act_match_matrices():
    rng = np.random.default_rng(11)
    for _ in range(50):
        A, B = random_pose(rng), random_pose(rng)
        MA, MB = oracle.sim3_matrix(A), oracle.sim3_matrix(B)
        assert np.abs(oracle.sim3_matrix(oracle.sim3_mul(A, B)) - MA @ MB).max() <= 1e-12 * np.abs(MA @ MB).max()
        assert np.abs(oracle.sim3_matrix(oracle.sim3_inv(A)) - np.linalg.inv(MA)).max() <= 1e-11
        x = rng.normal(size=3)
        assert np.allclose(oracle.sim3_act(A, x), (MA @ np.r_[x, 1.0])[:3], rtol=1e-13, atol=1e-13)


def test_adjoint_identity():
    """T Exp(tau) T^-1 = Exp(Ad_T tau) (derived from Eq. 1's hat map)."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        T = random_pose(rng)
        tau = rng.normal(size=7) * 0.3
        M = oracle.sim3_matrix(T)
        lhs = M @ expm(hat(tau)) @ np.linalg.inv(M)
        rhs = expm(hat(oracle.sim3_adjoint(T) @ tau))
        assert np.abs(lhs - rhs).max() <= 1e-10 * max(1.0, np.abs(lhs).max())


def test_adjoint_structure():
    rng = np.random.default_rng(8)
    T = random_pose(rng)
    Ad = oracle.sim3_adjoint(T)
    M = oracle.sim3_matrix(T)
    s = np.cbrt(np.linalg.det(M[:3, :3]))
    R = M[:3, :3] / s
    assert np.allclose(Ad[3:6, 3:6], R)
    assert np.allclose(Ad[0:3, 0:3], s * R)
    assert np.allclose(Ad[6], [0, 0, 0, 0, 0, 0, 1])
    assert np.allclose(Ad[3:6, [0, 1, 2, 6]], 0)


def test_retract_is_left_plus():
    """T <- tau (+) T = Exp(tau) o T (Eq. 1)."""
    rng = np.random.default_rng(9)
    for _ in range(20):
        T = random_pose(rng)
        tau = rng.normal(size=7) * 0.1
        out = oracle.sim3_matrix(oracle.sim3_retract(tau, T))
        assert np.abs(out - expm(hat(tau)) @ oracle.sim3_matrix(T)).max() <= 1e-12 * np.abs(out).max()
