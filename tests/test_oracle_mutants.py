"""The oracle's pins catch plausible mistakes: each case builds a copy of the
oracle with one planted mistake (oracle.c, ORC_MUTANT_<NAME>) on the CPU and
runs the pin that must fail on it; the unmutated oracle passes the same pins
in the rest of the suite."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    # a flipped sign in the rotation block of dx/dtau = [I, -[x]x, x]
    "JAC_ROT_SIGN": "tests/test_oracle_jacobians.py::test_residual_and_jacobian_vs_fd",
    # a transposed operand: the Jacobian mapped with Ad^T instead of Ad
    "ADJ_T": "tests/test_oracle_jacobians.py::test_residual_and_jacobian_vs_fd",
    # a wrong branch of the Huber IRLS weight (delta / e^2 instead of delta / e)
    "HUBER_SQ": "tests/test_oracle_gn.py::test_gradient_is_derivative_of_cost",
    # a dropped term: the distance residual left out of the gradient
    "DROP_DIST_GRAD": "tests/test_oracle_gn.py::test_gradient_is_derivative_of_cost",
    # a dropped factor: the Sim(3) exponential's translation without V
    "EXP_NO_V": "tests/test_oracle_sim3.py::test_exp_random_against_expm",
    # a flipped sign of the LM step
    "LM_SIGN": "tests/test_oracle_match.py::test_lm_recovers_analytic_projection",
    # rounding p* down instead of to the nearest pixel
    "ROUND_FLOOR": "tests/test_oracle_match.py::test_projection_alone_finds_ground_truth",
    # the wrong pose held fixed (the last instead of the first)
    "GAUGE": "tests/test_oracle_gn.py::test_exact_pose_recovery",
}


@pytest.mark.parametrize("mutant", sorted(CASES))
def test_pin_catches_planted_mistake(mutant):
    env = dict(os.environ, ORC_MUTANT=mutant)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", CASES[mutant]],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    out = r.stdout + r.stderr
    assert r.returncode == 1 and " failed" in out, f"{mutant}: the pin did not fail\n{out[-2000:]}"
