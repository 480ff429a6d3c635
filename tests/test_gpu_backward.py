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


@pytest.mark.parametrize("N,n_pairs,seed", [(12, 20, 7), (128, 300, 107)])
def test_step_backward_mixed_solves_agree_with_fp64(M, N, n_pairs, seed):
    """The adjoint's two solves (tau = -H^-1 g and b = H^-1 a) run by the
    FP32 factor with FP64 refinement (the default; the 128-keyframe graph
    factors in the workspace) against the FP64 factorisation (plan option
    solve_form 1): the point, confidence and pose gradients of one step agree
    to 1e-6 of their norm (the refinement stops when its predicted next
    correction is below 1e-9 of |x|; the FP32 atomics of the gathered side
    add their own summation-order rounding, about 1e-7)."""
    from paper_2412_12392_gb300 import api
    w = synth.global_graph(N=N, n_pairs=n_pairs, H=12, W=16, seed=seed)
    P = M.default_params()
    wd = w.to("cuda")
    idx = w.gt_match.cuda()
    q = (w.Q_qry.float() * 0.5 + 1.0).cuda()
    T = w.T_init.clone().cuda()
    rng = np.random.default_rng(seed)
    a = torch.from_numpy(rng.normal(size=(w.N, 7)) * 1e-2).cuda()
    G = torch.from_numpy(rng.normal(size=(w.N, 8)) * 0.1).cuda()
    out = {}
    for form in (0, 1):
        plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), opts={"solve_form": form})
        if N == 128:
            assert plan.counts[0] * 49 * 8 > 227 * 1024  # the FP32 factor goes to the workspace
        H, g, _, _ = M.gn_linearize(plan, P, T, wd.X_canon, idx, q)
        dX, dq, dT, st = api.gn_step_backward(plan, P, T, wd.X_canon, idx, q, H, g, dL_dTnew=G, dL_dtau=a,
                                            dL_dcost=0.3)
        torch.cuda.synchronize()
        assert int(st.max()) <= 1, st
        out[form] = [t.double().cpu().numpy() for t in (dX, dq, dT)]
    for name, x, ref in zip(("dX", "dq", "dT"), out[0], out[1]):
        e = rel_err(x, ref)
        print(f"{N} keyframes, {name}: mixed against FP64 solves {e:.2e}")
        assert e <= 1e-6, (name, e)
