"""Parity at the benchmark's full sizes and in its launch configuration.

* tracking (one frame against one keyframe, 512 x 384, radial camera, FP16
  storage, 10 % occluded query pixels): every pixel's match and the poses
  after 20 Gauss-Newton iterations against the oracle;
* global graph (64 keyframes, 256 directed edges, 512 x 384, FP16 storage):
  the batched matching launch on sampled query pixels of sampled edges, and
  the packed linearisation of sampled edges (fed the oracle's own matches),
  against the oracle computed one edge at a time; and the whole step of the
  benchmark -- the batched matching launch, then 10 packed Gauss-Newton
  iterations in its launch configuration -- against the oracle's
  Gauss-Newton run on the same matches, every pose;
* the 64-keyframe graph's solve (same plan structure as the benchmark) on
  oracle blocks.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import (BLOCK_RTOL, add_counts, assert_poses_close, block_rel_err, check_disagreements,
                    classify_disagreements, f64, pose_errors, solve_flags)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available()
    from paper_2412_12392_gb300 import build
    build.build()
    import paper_2412_12392_gb300 as M
    return M


def test_tracking_full_size(M):
    w = synth.tracking().to_storage(torch.float16)
    wd = w.to("cuda")
    P = M.default_params()
    par = M.params_dict(P)
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy())
    idx_g, q_g = M.match(plan, P, wd.X_ref, wd.X_qry, M.chunk_descriptors(wd.D_ref), M.chunk_descriptors(wd.D_qry),
                         wd.Q_ref, wd.Q_qry)
    gn = M.GaussNewton(plan, P, wd.X_canon, idx_g, q_g, packed=True)
    T_g = gn.run(w.T_init.cuda(), w.n_gn_iters).cpu()
    idx_r, q_r, dg = oracle.match_workload(w, 0, diag=True, **par)
    check_disagreements(classify_disagreements(idx_g, idx_r, dg, par), "tracking match:")
    occ = w.meta["occluded"].numpy()
    assert (idx_g.cpu().numpy()[occ] == -1).mean() >= 0.99
    q16 = torch.from_numpy(q_r).to(torch.float16)
    st, T_r, hist, done = oracle.gauss_newton(w.N, w.edges.numpy(), w.kf_off.numpy(), w.e_off.numpy(), w.X_canon,
                                              idx_r, q16, w.T_init.numpy(), w.n_gn_iters, **par)
    assert st == 0
    e = assert_poses_close(T_g, T_r)
    print(f"tracking poses vs oracle (rot, trans, scale): {e.max(axis=0)}")
    # the fused tracking loop (mslam_gn_track: one launch per iteration) on the
    # same matches
    gn_f = M.GaussNewton(plan, P, wd.X_canon, idx_g, q_g, packed=True)
    T_f = gn_f.run_tracking(w.T_init.cuda(), w.n_gn_iters).cpu()
    assert int(gn_f.status[0]) in (0, 1)
    e_f = assert_poses_close(T_f, T_r)
    print(f"fused tracking poses vs oracle (rot, trans, scale): {e_f.max(axis=0)}")


@pytest.fixture(scope="module")
def global_wl():
    return synth.global_graph(device="cuda").to_storage(torch.float16)


@pytest.mark.parametrize("match_form", [0, 1])
def test_global_full_size_sampled(M, global_wl, match_form):
    w = global_wl
    P = M.default_params()
    par = M.params_dict(P)
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), opts={"match_form": match_form, "match_block_w": 16})
    Dr, Dq = M.chunk_descriptors(w.D_ref), M.chunk_descriptors(w.D_qry)
    idx_g, q_g = M.match(plan, P, w.X_ref, w.X_qry, Dr, Dq, w.Q_ref, w.Q_qry)  # batched launch
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    match_edges = rng.choice(w.E, 12, replace=False)
    edges = match_edges[:4]
    H, W = int(w.kf_hw[0, 0]), int(w.kf_hw[0, 1])
    idx_sub, q_sub = idx_g.clone(), q_g.clone()
    tot = {}
    for e in match_edges:
        sl = w.edge_slice(int(e))
        cpu = {k: getattr(w, k)[sl].cpu() for k in ("X_ref", "X_qry", "D_ref", "D_qry", "Q_ref", "Q_qry")}
        pix = np.sort(rng.choice(H * W, 16384, replace=False))
        idx_r, q_r, dg = oracle.match(H, W, cpu["X_ref"], cpu["X_qry"], cpu["D_ref"], cpu["D_qry"], cpu["Q_ref"],
                                      cpu["Q_qry"], pix=pix, diag=True, **par)
        c = classify_disagreements(idx_g[sl].cpu().numpy()[pix], idx_r, dg, par)
        print(f"edge {e}: {c}")
        tot = add_counts(tot, c)
        if e in edges:
            # the oracle's matches of the whole edge feed both linearisations
            idx_full, q_full = oracle.match(H, W, cpu["X_ref"], cpu["X_qry"], cpu["D_ref"], cpu["D_qry"],
                                            cpu["Q_ref"], cpu["Q_qry"], **par)
            idx_sub[sl] = torch.from_numpy(idx_full).cuda()
            q_sub[sl] = torch.from_numpy(q_full).to(torch.float16).cuda()
    # the bars are on all sampled valid pixels together
    check_disagreements(tot, "sampled total:")
    packed = M.gn_pack(plan, P, w.X_canon, idx_sub, q_sub)
    T0 = w.T_init.cuda()
    Hb, gb, cb, nv = M.gn_linearize_packed(plan, P, torch.float16, T0, packed)
    torch.cuda.synchronize()
    Xc = w.X_canon.cpu()
    for e in edges:
        i, j = int(w.edges[e, 0]), int(w.edges[e, 1])
        sl = w.edge_slice(int(e))
        Hr, gr, cr, nvr = oracle.linearize_edge(w.T_init[i], w.T_init[j], Xc[w.kf_slice(i)], Xc[w.kf_slice(j)],
                                                idx_sub[sl].cpu(), q_sub[sl].cpu(), **par)
        eh = block_rel_err(Hb[e:e + 1], Hr[None])[0]
        eg = block_rel_err(gb[e:e + 1], gr[None])[0]
        print(f"edge {e}: H rel {eh:.2e}, g rel {eg:.2e}, matches {int(nv[e])}")
        assert eh <= BLOCK_RTOL and eg <= BLOCK_RTOL and int(nv[e]) == nvr


def test_global_full_size_gauss_newton(M, global_wl):
    """The benchmark's step on the benchmark's graph: the batched matching
    launch, then mslam_gn_pack and 10 iterations of the packed linearisation
    and the mixed-precision solve in the launch configuration the benchmark
    keeps (8 x 32 match blocks with two query pixels per thread, the
    prefetching register-pipeline linearisation with 16384-pixel tiles),
    against the oracle's Gauss-Newton (literal 14 x 14 blocks, dense FP64
    Cholesky) on the same matches and confidences: every one of the 64 poses
    within 1e-5.  The plain register pipeline (lin_form 1) on the same
    records gives the same poses bit for bit.  About two minutes of oracle
    time on 16 host threads."""
    w = global_wl
    P = M.default_params()
    par = M.params_dict(P)
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy(),
                  opts={"match_block_w": 8, "match_ppt": 2, "lin_tile": 16384, "lin_blocks_per_sm": 2,
                        "lin_form": 3})
    Dr, Dq = M.chunk_descriptors(w.D_ref), M.chunk_descriptors(w.D_qry)
    idx_g, q_g = M.match(plan, P, w.X_ref, w.X_qry, Dr, Dq, w.Q_ref, w.Q_qry)
    del Dr, Dq
    gn = M.GaussNewton(plan, P, w.X_canon, idx_g, q_g, packed=True)
    T_g = gn.run(w.T_init.cuda(), w.n_gn_iters).cpu()
    status = gn.status.cpu()
    assert int(status[0]) in (0, 1)
    plan1 = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), opts=dict(plan.opts, lin_form=1))
    gn1 = M.GaussNewton(plan1, P, w.X_canon, idx_g, q_g, packed=True)
    assert torch.equal(gn1.run(w.T_init.cuda(), w.n_gn_iters).cpu(), T_g)
    del gn1, plan1
    st, T_r, hist, done = oracle.gauss_newton(w.N, w.edges.numpy(), w.kf_off.numpy(), w.e_off.numpy(),
                                              w.X_canon.cpu(), idx_g.cpu(), q_g.cpu(), w.T_init.numpy(),
                                              w.n_gn_iters, **par)
    assert st == 0
    e = assert_poses_close(T_g, T_r)
    assert torch.equal(T_g[0], w.T_init[0])
    e_gt = pose_errors(T_g, w.T_gt)[1:].max(axis=0)
    print(f"global graph, 64 keyframes: GPU poses vs oracle (rot, trans, scale) max {e.max(axis=0)}; "
          f"vs ground truth {e_gt}")


def test_global_graph_solve_structure(M):
    """The 64-keyframe / 256-edge plan of the benchmark (small images, same
    graph structure and hence the same symbolic factorisation): the solve on
    oracle blocks against the oracle's dense solve."""
    w = synth.global_graph(H=24, W=32)
    P = M.default_params()
    par = M.params_dict(P)
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy())
    Hr, gr = [], []
    idx = w.gt_match.numpy()
    q = w.Q_qry.double().numpy()
    T0 = w.T_init.numpy()
    for e in range(w.E):
        i, j = int(w.edges[e, 0]), int(w.edges[e, 1])
        sl = w.edge_slice(e)
        Hb, gb, _, _ = oracle.linearize_edge(T0[i], T0[j], w.X_canon[w.kf_slice(i)], w.X_canon[w.kf_slice(j)], idx[sl],
                                             q[sl], **par)
        Hr.append(Hb)
        gr.append(gb)
    H32, g32 = torch.from_numpy(np.array(Hr)).float(), torch.from_numpy(np.array(gr)).float()
    T = w.T_init.clone().cuda()
    tau = torch.zeros(w.N, 7, dtype=torch.float64, device="cuda")
    ws = plan.workspace(M._lib.MSLAM_OP_SOLVE)
    tau, st = M.gn_solve(plan, P, H32.cuda(), g32.cuda(), T, tau=tau, workspace=ws)
    torch.cuda.synchronize()
    s, T_r, tau_r = oracle.gn_solve(w.N, w.edges.numpy(), H32.double(), g32.double(), T0)
    assert s == 0 and int(st[0]) in (0, 1)
    err = np.abs(f64(tau) - tau_r).max() / max(1.0, np.abs(tau_r).max())
    print(f"64-keyframe solve: tau rel err {err:.2e}, mixed-precision flags {solve_flags(plan, ws).tolist()}")
    assert err <= 1e-8
    assert_poses_close(T, T_r, 1e-8)
    # this graph is solved by the FP32 factorisation with FP64 refinement
    assert solve_flags(plan, ws).tolist() == [1]
    # the FP64-only form (plan option solve_form = 1) agrees with both
    plan64 = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), opts={"solve_form": 1})
    assert plan64.solve_launches == 1 and plan.solve_launches == 3
    T64 = w.T_init.clone().cuda()
    tau64, st64 = M.gn_solve(plan64, P, H32.cuda(), g32.cuda(), T64, tau=torch.zeros_like(tau))
    torch.cuda.synchronize()
    err64 = np.abs(f64(tau64) - tau_r).max() / max(1.0, np.abs(tau_r).max())
    print(f"FP64-only solve: tau rel err {err64:.2e}")
    assert int(st64[0]) in (0, 1) and err64 <= 1e-8



def test_largest_batched_graph_solve_structure(M):
    """The largest graph of the batched workload (128 keyframes, 600 directed
    edges; small images, same graph structure): its FP32 factor (1,123
    blocks) is too large for one SM's shared memory, so the mixed-precision
    solve factors it in place in the workspace; the solve on oracle blocks
    against the oracle's dense solve, and the FP64-only form beside it."""
    w = synth.batched_graph(7, scale=16)
    P = M.default_params()
    par = M.params_dict(P)
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy())
    assert plan.solve_launches == 3
    idx = w.gt_match.numpy()
    q = w.Q_qry.double().numpy()
    T0 = w.T_init.numpy()
    Hr, gr = [], []
    for e in range(w.E):
        i, j = int(w.edges[e, 0]), int(w.edges[e, 1])
        sl = w.edge_slice(e)
        Hb, gb, _, _ = oracle.linearize_edge(T0[i], T0[j], w.X_canon[w.kf_slice(i)], w.X_canon[w.kf_slice(j)], idx[sl],
                                             q[sl], **par)
        Hr.append(Hb)
        gr.append(gb)
    H32, g32 = torch.from_numpy(np.array(Hr)).float(), torch.from_numpy(np.array(gr)).float()
    s, T_r, tau_r = oracle.gn_solve(w.N, w.edges.numpy(), H32.double(), g32.double(), T0)
    assert s == 0
    for form in (0, 1):
        pl = plan if form == 0 else M.Plan(w.kf_hw.numpy(), w.edges.numpy(), opts={"solve_form": 1})
        T = w.T_init.clone().cuda()
        ws = pl.workspace(M._lib.MSLAM_OP_SOLVE)
        tau, st = M.gn_solve(pl, P, H32.cuda(), g32.cuda(), T, tau=torch.zeros(w.N, 7, dtype=torch.float64,
                                                                                device="cuda"), workspace=ws)
        torch.cuda.synchronize()
        assert int(st[0]) in (0, 1)
        err = np.abs(f64(tau) - tau_r).max() / max(1.0, np.abs(tau_r).max())
        flags = solve_flags(pl, ws).tolist() if form == 0 else None
        print(f"128-keyframe solve, form {form}: tau rel err {err:.2e}, mixed-precision flags {flags}")
        assert err <= 1e-8
        assert_poses_close(T, T_r, 1e-8)
        if form == 0:
            assert flags == [1]  # solved by the FP32 factorisation (in the workspace) with FP64 refinement
