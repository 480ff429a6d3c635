"""Failure paths of the Gauss-Newton loop, made on the host (no GPU fault):

* a bounded device wait that runs out: the streamed linearisation forms wait
  for their asynchronous record copies with a bounded number of polls (plan
  option wait_limit); a negative limit gives up at once without issuing a
  copy, so nothing is in flight.  The graph's status must read
  MSLAM_ERR_TIMEOUT, and the solve must then leave its poses unchanged;
* non-finite canonical pointmaps: such points are not valid matches (as in
  the oracle), so a keyframe whose whole pointmap is NaN loses its edge and
  the reduced system is singular (MSLAM_ERR_NOT_PD, poses unchanged), and a
  partly NaN pointmap gives the oracle's poses on the remaining pixels;
* a non-finite gradient handed to the solve: MSLAM_ERR_NONFINITE, poses
  unchanged, in both solve forms.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import assert_poses_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available()
    from paper_2412_12392_gb300 import build
    build.build()
    import paper_2412_12392_gb300 as M
    return M


def _matched(M, w, plan, P):
    wd = w.to("cuda")
    idx, q = M.match(plan, P, wd.X_ref, wd.X_qry, M.chunk_descriptors(wd.D_ref), M.chunk_descriptors(wd.D_qry),
                     wd.Q_ref, wd.Q_qry)
    return wd, idx, q


@pytest.mark.parametrize("lin_form", [0, 2])
def test_bounded_wait_timeout_status(M, lin_form):
    from paper_2412_12392_gb300 import _lib
    w = synth.tiny().to_storage(torch.float16)
    P = M.default_params()
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), opts={"lin_form": lin_form, "lin_tile": 4096, "wait_limit": -1})
    wd, idx, q = _matched(M, w, plan, P)
    gn = M.GaussNewton(plan, P, wd.X_canon, idx, q, packed=True)
    T0 = w.T_init.cuda()
    T = gn.run(T0, 3)
    torch.cuda.synchronize()
    assert int(gn.status[0]) == _lib.MSLAM_ERR_TIMEOUT
    assert torch.equal(T, T0)  # the solve skipped the graph
    assert torch.isnan(gn.H).all(dim=(1, 2)).any()
    # the same plan with the default limit runs normally
    plan_ok = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), opts={"lin_form": lin_form, "lin_tile": 4096})
    gn_ok = M.GaussNewton(plan_ok, P, wd.X_canon, idx, q, packed=True)
    T_ok = gn_ok.run(T0, 3)
    torch.cuda.synchronize()
    assert int(gn_ok.status[0]) in (0, 1) and not torch.equal(T_ok, T0)


@pytest.mark.parametrize("packed", [False, True])
def test_nan_pointmaps(M, packed):
    from paper_2412_12392_gb300 import _lib
    w = synth.tiny()
    P = M.default_params()
    par = M.params_dict(P)
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy())
    wd, idx, q = _matched(M, w, plan, P)
    T0 = w.T_init.cuda()
    # the last keyframe of the chain entirely NaN: its only edge contributes nothing
    X = wd.X_canon.clone()
    X[int(w.kf_off[3]):int(w.kf_off[4])] = float("nan")
    gn = M.GaussNewton(plan, P, X, idx, q, packed=packed)
    T = gn.run(T0, 2)
    torch.cuda.synchronize()
    assert int(gn.status[0]) == _lib.MSLAM_ERR_NOT_PD
    assert torch.equal(T, T0)
    st, _, _, _ = oracle.gauss_newton(w.N, w.edges.numpy(), w.kf_off.numpy(), w.e_off.numpy(), X.cpu(), idx.cpu(),
                                      q.cpu(), w.T_init.numpy(), 2, **par)
    assert st == _lib.MSLAM_ERR_NOT_PD
    # every other row of keyframe 1 NaN: those pixels drop out on both sides
    X = wd.X_canon.clone()
    H, W = int(w.kf_hw[1, 0]), int(w.kf_hw[1, 1])
    k1 = X[int(w.kf_off[1]):int(w.kf_off[2])].view(H, W, 3)
    k1[::2] = float("nan")
    gn = M.GaussNewton(plan, P, X, idx, q, packed=packed)
    T = gn.run(T0, w.n_gn_iters).cpu()
    torch.cuda.synchronize()
    assert int(gn.status[0]) in (0, 1)
    st, T_r, _, _ = oracle.gauss_newton(w.N, w.edges.numpy(), w.kf_off.numpy(), w.e_off.numpy(), X.cpu(), idx.cpu(),
                                        q.cpu(), w.T_init.numpy(), w.n_gn_iters, **par)
    assert st == 0
    assert_poses_close(T, T_r)


@pytest.mark.parametrize("solve_form", [0, 1])
def test_nonfinite_step_status(M, solve_form):
    from paper_2412_12392_gb300 import _lib
    w = synth.tiny()
    P = M.default_params()
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), opts={"solve_form": solve_form})
    wd, idx, q = _matched(M, w, plan, P)
    T0 = w.T_init.cuda()
    H, g, _, _ = M.gn_linearize(plan, P, T0, wd.X_canon, idx, q)
    g = g.clone()
    g[1, 9] = float("nan")
    T = T0.clone()
    _, st = M.gn_solve(plan, P, H, g, T)
    torch.cuda.synchronize()
    assert int(st[0]) == _lib.MSLAM_ERR_NONFINITE
    assert torch.equal(T, T0)
