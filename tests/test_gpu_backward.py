"""GPU adjoint (mslam_gn_backward and the GNStep autograd function) against
the FP64 oracle's gradient of L = c E_g + a . tau (one Gauss-Newton step),
which is itself pinned by central differences in the CPU tests."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

# FP32 per-pixel recomputation against FP64: normwise relative error, and
# every entry within ELEM of the largest entry of the oracle's gradient
REL = 1e-5
ELEM = 2e-5


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available()
    from paper_2412_12392_gb300 import build
    build.build()
    import paper_2412_12392_gb300 as M
    return M


def setup(dtype, seed=5):
    w = synth.global_graph(N=5, n_pairs=7, H=24, W=32, seed=seed)
    ws = w.to_storage(dtype)
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(w.N, 7))
    a[0] = 0.0
    q = (ws.Q_qry.float() * 0.5 + 1.0).to(dtype)
    return ws, q, a


def rel_err(x, ref):
    x, ref = np.asarray(x, np.float64), np.asarray(ref, np.float64)
    return np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300)


def elem_err(x, ref):
    """max_k |x_k - ref_k| / max_k |ref_k|"""
    x, ref = np.asarray(x, np.float64).ravel(), np.asarray(ref, np.float64).ravel()
    return np.abs(x - ref).max() / max(np.abs(ref).max(), 1e-300)


def assert_grad_close(x, ref, what):
    n, e = rel_err(x, ref), elem_err(x, ref)
    print(f"{what}: normwise {n:.2e}, entrywise {e:.2e}")
    assert n <= REL and e <= ELEM, what


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("with_step,c", [(False, 0.7), (True, 0.7), (True, 0.0)])
def test_backward_matches_oracle(M, dtype, with_step, c):
    ws, q, a = setup(dtype)
    P = M.default_params()
    par = M.params_dict(P)
    plan = M.Plan(ws.kf_hw.numpy(), ws.edges.numpy())
    X = ws.X_canon.cuda()
    idx = ws.gt_match.cuda()
    qd = q.cuda()
    T = ws.T_init.cuda()
    H, g, cost, nv = M.gn_linearize(plan, P, T, X, idx, qd)
    dL_dtau = torch.from_numpy(a).cuda() if with_step else None
    dX, dq, st = M.gn_backward(plan, P, T, X, idx, qd, H, g, dL_dtau=dL_dtau, dL_dcost=c)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    s, dXr, dqr, tau = oracle.gn_step_grad(ws.N, ws.edges.numpy(), ws.kf_off.numpy(), ws.e_off.numpy(),
                                           ws.T_init.numpy(), ws.X_canon, ws.gt_match, q,
                                           dL_dtau=a if with_step else None, dL_dcost=c, **par)
    assert s == 0
    assert_grad_close(dX.cpu().numpy(), dXr, f"backward {dtype} step={with_step} c={c}: dX")
    assert_grad_close(dq.cpu().numpy(), dqr, f"backward {dtype} step={with_step} c={c}: dq")


def test_autograd_function(M):
    from paper_2412_12392_gb300.autograd import gn_step
    ws, q, a = setup(torch.float32, seed=9)
    P = M.default_params()
    par = M.params_dict(P)
    plan = M.Plan(ws.kf_hw.numpy(), ws.edges.numpy())
    X = ws.X_canon.cuda().requires_grad_(True)
    qd = q.cuda().requires_grad_(True)
    idx = ws.gt_match.cuda()
    T = ws.T_init.cuda()
    T_new, tau, cost = gn_step(X, qd, T, plan, P, idx)
    at = torch.from_numpy(a).cuda()
    loss = (tau * at).sum() + 0.7 * cost
    loss.backward()
    s, dXr, dqr, tau_r = oracle.gn_step_grad(ws.N, ws.edges.numpy(), ws.kf_off.numpy(), ws.e_off.numpy(),
                                             ws.T_init.numpy(), ws.X_canon, ws.gt_match, q, dL_dtau=a,
                                             dL_dcost=0.7, **par)
    assert np.abs(tau.detach().cpu().numpy() - tau_r).max() <= 1e-4 * max(1.0, np.abs(tau_r).max())
    assert_grad_close(X.grad.cpu().numpy(), dXr, "autograd dX")
    assert_grad_close(qd.grad.cpu().numpy(), dqr, "autograd dq")
