"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs (the oracle consumes the stored values, dequantised).

Covers matching (Sec. 3.2), linearisation (Eq. backend_ray, Supp. S1), the
gauge-fixed solve and retraction (Sec. 3.5), the full Gauss-Newton loop, both
storage dtypes, the plain per-edge and the batched launch forms, CUDA-graph
capture, and the degenerate cases (invalid pixels, disconnected graphs,
single keyframe, empty edge list)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import (BLOCK_RTOL, MATCH_AGREE, assert_poses_close, block_rel_err, f64, match_agreement,
                    pose_errors, solve_flags)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2412_12392_gb300 import build
    build.build()
    import paper_2412_12392_gb300 as M
    return M


def to_dev(w, dtype=torch.float32):
    return w.to_storage(dtype).to("cuda")


def gpu_match(M, plan, P, wd, **kw):
    return M.match(plan, P, wd.X_ref, wd.X_qry, M.chunk_descriptors(wd.D_ref), M.chunk_descriptors(wd.D_qry),
                   wd.Q_ref, wd.Q_qry, **kw)


def oracle_match_all(w, par, diag=True):
    idx, q, dg = [], [], []
    for e in range(w.E):
        out = oracle.match_workload(w, e, diag=diag, **par)
        idx.append(out[0])
        q.append(out[1])
        if diag:
            dg.append(out[2])
    return np.concatenate(idx), np.concatenate(q), (np.concatenate(dg) if diag else None)


@pytest.mark.parametrize("dtype,match_form", [(torch.float32, 0), (torch.float16, 0), (torch.float16, 1),
                                              (torch.float16, 2)])
def test_match_parity_tiny(M, tiny_wl, dtype, match_form):
    """match_form 1: the refinement windows scored on the tensor cores;
    match_form 2: the windows scored from a block's staged box."""
    P = M.default_params()
    par = M.params_dict(P)
    ws = tiny_wl.to_storage(dtype)  # the oracle reads the stored (dequantised) values
    wd = ws.to("cuda")
    plan = M.Plan(ws.kf_hw.numpy(), ws.edges.numpy(), opts={"match_form": match_form})
    idx_g, q_g = gpu_match(M, plan, P, wd)
    torch.cuda.synchronize()
    idx_r, q_r, dg = oracle_match_all(ws, par)
    agree, ndis, nunion, expl = match_agreement(idx_g, idx_r, dg, par)
    print(f"match parity {dtype} form {match_form}: agree {agree:.6f} ({ndis} of {nunion}), explained {expl:.3f}")
    assert agree >= MATCH_AGREE
    both = (f64(idx_g) == idx_r) & (idx_r >= 0)
    qg = f64(q_g)[both]
    qr = q_r[both].astype(np.float32 if dtype == torch.float32 else np.float16).astype(np.float64)
    rtol = 2e-6 if dtype == torch.float32 else 1e-3
    assert np.abs(qg - qr).max() <= rtol * np.abs(qr).max()
    # launch shapes change no result: block width and query pixels per thread
    # (for the tensor-core form also the warp groups a query falls in)
    for opts in ({"match_block_w": 8}, {"match_ppt": 2}, {"match_block_w": 64, "match_ppt": 2}):
        plan_b = M.Plan(ws.kf_hw.numpy(), ws.edges.numpy(), opts=dict(opts, match_form=match_form))
        idx_b, q_b = gpu_match(M, plan_b, P, wd)
        assert torch.equal(idx_b, idx_g) and torch.equal(q_b, q_g), opts


def test_match_forms_and_init_agree(M, tiny_wl):
    P = M.default_params()
    wd = to_dev(tiny_wl)
    plan = M.Plan(tiny_wl.kf_hw.numpy(), tiny_wl.edges.numpy())
    a_idx, a_q = gpu_match(M, plan, P, wd)
    b_idx, b_q = gpu_match(M, plan, P, wd, per_edge=True)
    assert torch.equal(a_idx, b_idx) and torch.equal(a_q, b_q)
    # edge sub-range touches only that edge's slice
    c_idx = torch.full_like(a_idx, -7)
    c_q = torch.zeros_like(a_q)
    gpu_match(M, plan, P, wd, idx_out=c_idx, q_out=c_q, edge_range=(1, 2))
    sl = tiny_wl.edge_slice(1)
    assert torch.equal(c_idx[sl], a_idx[sl])
    assert bool((c_idx[:sl.start] == -7).all()) and bool((c_idx[sl.stop:] == -7).all())
    # initialisation from previous matches (tracking) against the oracle
    par = M.params_dict(P)
    init = tiny_wl.gt_match.to("cuda")
    i_idx, _ = gpu_match(M, plan, P, wd, init_idx=init)
    r_idx = np.concatenate([oracle.match_workload(tiny_wl, e, init_idx=tiny_wl.gt_match[tiny_wl.edge_slice(e)],
                                                  **par)[0] for e in range(tiny_wl.E)])
    agree, *_ = match_agreement(i_idx, r_idx)
    assert agree >= MATCH_AGREE


@pytest.mark.parametrize("dtype,match_form", [(torch.float32, 0), (torch.float16, 1), (torch.float16, 2)])
def test_match_invalid_and_edge_pixels(M, dtype, match_form):
    """Zero / NaN query points are rejected; queries projecting outside the
    reference image clamp to the border; out-of-range init indices fall back
    to the identity; an image whose width (36) is not a multiple of the block
    width leaves partial blocks (ragged tail)."""
    rng = np.random.default_rng(3)
    H, W, d = 20, 36, 16
    X = np.c_[rng.uniform(-1, 1, H * W), rng.uniform(-1, 1, H * W), rng.uniform(2, 4, H * W)].astype(np.float32)
    Xq = X.copy() * 1.01
    Xq[::5] = 0
    Xq[2::17] = np.nan
    Xq[3::13, 0] += 5.0  # far outside the field of view
    D = rng.normal(size=(H * W, d)).astype(np.float32)
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    Q = rng.uniform(1, 10, H * W).astype(np.float32)
    init = np.arange(H * W, dtype=np.int32)
    init[1::9] = 10 ** 8
    init[4::11] = -3
    plan = M.Plan([[H, W], [H, W]], [[0, 1]], opts={"match_form": match_form})
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()
    P = M.default_params()
    Dc = M.chunk_descriptors(t(D))
    idx_g, q_g = M.match(plan, P, t(X), t(Xq), Dc, Dc, t(Q), t(Q), init_idx=t(init).int())
    par = M.params_dict(P)
    st = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dtype)  # the stored values
    idx_r, q_r, dg = oracle.match(H, W, st(X), st(Xq), st(D), st(D), st(Q), st(Q),
                                  init_idx=np.where((init >= 0) & (init < H * W), init, -1), diag=True, **par)
    assert bool((idx_g.cpu().numpy()[::5] == -1).all()) and bool((idx_g.cpu().numpy()[2::17] == -1).all())
    agree, *_ = match_agreement(idx_g, idx_r)
    assert agree >= 0.99


def oracle_blocks(w, T, idx, q, par):
    H, g, c, nv = [], [], [], []
    for e in range(w.E):
        i, j = int(w.edges[e, 0]), int(w.edges[e, 1])
        sl = w.edge_slice(e)
        Hb, gb, cb, nb = oracle.linearize_edge(T[i], T[j], w.X_canon[w.kf_slice(i)], w.X_canon[w.kf_slice(j)],
                                               idx[sl], q[sl], **par)
        H.append(Hb)
        g.append(gb)
        c.append(cb)
        nv.append(nb)
    return np.array(H), np.array(g), np.array(c), np.array(nv)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_linearize_parity_tiny(M, tiny_wl, dtype):
    P = M.default_params()
    par = M.params_dict(P)
    ws = tiny_wl.to_storage(dtype)
    # matches from the oracle, q stored in the storage dtype for both sides
    idx_r, q_r, _ = oracle_match_all(ws, par, diag=False)
    q_s = torch.from_numpy(q_r).to(dtype)
    wd = ws.to("cuda")
    plan = M.Plan(ws.kf_hw.numpy(), ws.edges.numpy())
    T = ws.T_init.clone()
    H, g, c, nv = M.gn_linearize(plan, P, T.cuda(), wd.X_canon, torch.from_numpy(idx_r).cuda(), q_s.cuda())
    torch.cuda.synchronize()
    Hr, gr, cr, nvr = oracle_blocks(ws, T.numpy(), idx_r, q_s, par)
    eh, eg = block_rel_err(H, Hr), block_rel_err(g, gr)
    print(f"linearize {dtype}: max H rel {eh.max():.2e}, g rel {eg.max():.2e}")
    assert eh.max() <= BLOCK_RTOL and eg.max() <= BLOCK_RTOL
    assert np.allclose(f64(c), cr, rtol=1e-5)
    assert np.array_equal(nv.cpu().numpy(), nvr)
    # the plain per-edge form gives bitwise the same blocks
    H2, g2, c2, nv2 = M.gn_linearize(plan, P, T.cuda(), wd.X_canon, torch.from_numpy(idx_r).cuda(), q_s.cuda(),
                                     per_edge=True)
    assert torch.equal(H, H2) and torch.equal(g, g2) and torch.equal(c, c2)


def test_solve_parity_on_oracle_blocks(M, tiny_wl):
    """The solve alone: both sides consume the oracle's blocks (rounded to
    FP32 for the GPU input, read back exactly by the oracle)."""
    P = M.default_params()
    par = M.params_dict(P)
    w = tiny_wl
    idx_r, q_r, _ = oracle_match_all(w, par, diag=False)
    Hr, gr, _, _ = oracle_blocks(w, w.T_init.numpy(), idx_r, q_r, par)
    H32 = torch.from_numpy(Hr).float()
    g32 = torch.from_numpy(gr).float()
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy())
    T = w.T_init.clone().cuda()
    tau, st = M.gn_solve(plan, P, H32.cuda(), g32.cuda(), T, tau=torch.zeros(w.N, 7, dtype=torch.float64,
                                                                              device="cuda"))
    torch.cuda.synchronize()
    s, T_r, tau_r = oracle.gn_solve(w.N, w.edges.numpy(), H32.double(), g32.double(), w.T_init.numpy())
    assert s == 0 and int(st[0]) in (0, 1)
    assert np.abs(f64(tau) - tau_r).max() <= 1e-9 * max(1.0, np.abs(tau_r).max())
    assert torch.equal(T[0].cpu(), w.T_init[0])  # gauge untouched, bitwise
    assert_poses_close(T, T_r, 1e-9)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_gauss_newton_parity_tiny(M, tiny_wl, dtype):
    P = M.default_params()
    par = M.params_dict(P)
    ws = tiny_wl.to_storage(dtype)
    idx_r, q_r, _ = oracle_match_all(ws, par, diag=False)
    q_s = torch.from_numpy(q_r).to(dtype)
    wd = ws.to("cuda")
    plan = M.Plan(ws.kf_hw.numpy(), ws.edges.numpy())
    gn = M.GaussNewton(plan, P, wd.X_canon, torch.from_numpy(idx_r).cuda(), q_s.cuda())
    T_g = gn.run(ws.T_init.cuda(), ws.n_gn_iters).cpu()
    st, T_r, hist, done = oracle.gauss_newton(ws.N, ws.edges.numpy(), ws.kf_off.numpy(), ws.e_off.numpy(),
                                              ws.X_canon, idx_r, q_s, ws.T_init.numpy(), ws.n_gn_iters, **par)
    assert st == 0
    e = assert_poses_close(T_g, T_r)
    print(f"GN parity {dtype}: max (rot, trans, scale) {e.max(axis=0)}")
    assert torch.equal(T_g[0], ws.T_init[0])
    # and the optimisation really moved the poses toward the ground truth
    e0 = pose_errors(ws.T_init, ws.T_gt)[1:, 0].max()
    e1 = pose_errors(T_g, ws.T_gt)[1:, 0].max()
    assert e1 < 0.25 * e0


def test_full_pipeline_tiny(M, tiny_wl):
    """GPU matching feeding GPU Gauss-Newton against the oracle doing both."""
    P = M.default_params()
    par = M.params_dict(P)
    w = tiny_wl
    wd = to_dev(w)
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy())
    idx_g, q_g = gpu_match(M, plan, P, wd)
    gn = M.GaussNewton(plan, P, wd.X_canon, idx_g, q_g)
    T_g = gn.run(w.T_init.cuda(), w.n_gn_iters).cpu()
    idx_r, q_r, _ = oracle_match_all(w, par, diag=False)
    st, T_r, _, _ = oracle.gauss_newton(w.N, w.edges.numpy(), w.kf_off.numpy(), w.e_off.numpy(), w.X_canon, idx_r,
                                        q_r, w.T_init.numpy(), w.n_gn_iters, **par)
    assert_poses_close(T_g, T_r)


def test_cuda_graph_replay_matches_eager(M, tiny_wl):
    P = M.default_params()
    w = tiny_wl
    wd = to_dev(w)
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy())
    idx_g, q_g = gpu_match(M, plan, P, wd)
    gn = M.GaussNewton(plan, P, wd.X_canon, idx_g, q_g)
    T_e = gn.run(w.T_init.cuda(), 5).clone()
    gn.capture(5)
    T_c = gn.replay(w.T_init.cuda()).clone()
    torch.cuda.synchronize()
    assert torch.equal(T_e, T_c)


def test_exact_recovery_gpu(M):
    from test_oracle_gn import exact_graph
    rng = np.random.default_rng(1)
    T_gt, X, edges, kf_off, e_off, idx, q = exact_graph(rng, N=5, H=32, W=48)
    N = T_gt.shape[0]
    T0 = T_gt.copy()
    for k in range(1, N):
        T0[k] = oracle.sim3_mul(oracle.sim3_exp(np.r_[rng.normal(size=3) * 0.05, rng.normal(size=3) * 0.03, 0.05]),
                                T_gt[k])
    plan = M.Plan([[32, 48]] * N, edges)
    P = M.default_params()
    gn = M.GaussNewton(plan, P, torch.from_numpy(X).float().cuda(), torch.from_numpy(idx).cuda(),
                       torch.from_numpy(q).float().cuda())
    T = gn.run(torch.from_numpy(T0).cuda(), 15).cpu()
    # float storage of the points limits the recovery to ~1e-7
    assert_poses_close(T, T_gt, 1e-5)


def test_disconnected_graph_not_pd(M):
    from test_oracle_gn import exact_edge
    rng = np.random.default_rng(4)
    Ti, Tj, Xi, Xj, idx, q = exact_edge(rng, H=16, W=16)
    N = 4
    X = np.concatenate([Xi, Xj, Xi, Xj]).astype(np.float32)
    plan = M.Plan([[16, 16]] * N, [[0, 1], [2, 3]])
    T0 = torch.from_numpy(np.stack([Ti, Tj, Ti, Tj])).cuda()
    P = M.default_params()
    idx2 = torch.from_numpy(np.concatenate([idx, idx])).cuda()
    q2 = torch.from_numpy(np.concatenate([q, q]).astype(np.float32)).cuda()
    H, g, c, nv = M.gn_linearize(plan, P, T0, torch.from_numpy(X).cuda(), idx2, q2)
    T = T0.clone()
    ws = plan.workspace(M._lib.MSLAM_OP_SOLVE)
    tau, st = M.gn_solve(plan, P, H, g, T, workspace=ws)
    torch.cuda.synchronize()
    assert int(st[0]) == 3
    assert torch.equal(T, T0)
    # the mixed-precision kernel declined the singular system (FP32 pivots at
    # rounding level) and the FP64 kernel reported it
    assert solve_flags(plan, ws).tolist() == [0]



def test_degenerate_plans(M):
    P = M.default_params()
    # one keyframe, no edges: nothing to solve, converged at once
    plan = M.Plan([[8, 8]], np.zeros((0, 2), np.int32))
    T = torch.tensor([[0, 0, 0, 0, 0, 0, 1, 1.0]], dtype=torch.float64, device="cuda")
    H = torch.zeros(0, 14, 14, device="cuda")
    g = torch.zeros(0, 14, device="cuda")
    tau, st = M.gn_solve(plan, P, H, g, T)
    torch.cuda.synchronize()
    assert int(st[0]) == 1
    # two graphs in one plan: each keeps its own first keyframe fixed
    from test_oracle_gn import exact_edge
    rng = np.random.default_rng(5)
    Ti, Tj, Xi, Xj, idx, q = exact_edge(rng, H=16, W=16)
    plan2 = M.Plan([[16, 16]] * 4, [[0, 1], [1, 0], [2, 3], [3, 2]], graph_of_kf=[0, 0, 1, 1])
    assert plan2.G == 2 and list(plan2.order) == [-1, 0, -1, 0]
    X = torch.from_numpy(np.concatenate([Xi, Xj, Xi, Xj]).astype(np.float32)).cuda()
    idx4 = torch.from_numpy(np.concatenate([idx] * 4)).cuda()
    q4 = torch.from_numpy(np.concatenate([q] * 4).astype(np.float32)).cuda()
    T0 = np.stack([Ti, Tj, Ti, Tj])
    T0p = T0.copy()
    T0p[1] = oracle.sim3_mul(oracle.sim3_exp(np.r_[0.02, 0, 0.01, 0.01, 0, 0, 0.02]), T0[1])
    T0p[3] = T0p[1]
    gn = M.GaussNewton(plan2, P, X, idx4, q4)
    T = gn.run(torch.from_numpy(T0p).cuda(), 10).cpu()
    assert_poses_close(T, T0, 1e-5)
    assert torch.equal(T[0], torch.from_numpy(T0p[0])) and torch.equal(T[2], torch.from_numpy(T0p[2]))


def test_argument_errors_do_not_launch(M, tiny_wl):
    from paper_2412_12392_gb300 import _lib
    P = M.default_params()
    wd = to_dev(tiny_wl)
    plan = M.Plan(tiny_wl.kf_hw.numpy(), tiny_wl.edges.numpy())
    with pytest.raises(_lib.MslamError) as ei:
        M.match(plan, P, wd.X_ref, wd.X_qry, M.chunk_descriptors(wd.D_ref)[:3].contiguous(),
                M.chunk_descriptors(wd.D_qry)[:3].contiguous(), wd.Q_ref, wd.Q_qry)
    assert ei.value.status == _lib.MSLAM_ERR_ARG
    bad = M.default_params(sigma_ray=0.0)
    idx, q = gpu_match(M, plan, P, wd)
    with pytest.raises(_lib.MslamError):
        M.gn_linearize(plan, bad, tiny_wl.T_init.cuda(), wd.X_canon, idx, q)
    with pytest.raises(_lib.MslamError):
        M.Plan([[16, 16], [16, 16]], [[0, 0]])


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_packed_linearize_parity(M, tiny_wl, dtype):
    """Packed form (gather once, stream records) against the oracle, and the
    plain per-edge and batched packed launches agree bitwise."""
    P = M.default_params()
    par = M.params_dict(P)
    ws = tiny_wl.to_storage(dtype)
    idx_r, q_r, _ = oracle_match_all(ws, par, diag=False)
    q_s = torch.from_numpy(q_r).to(dtype)
    wd = ws.to("cuda")
    plan = M.Plan(ws.kf_hw.numpy(), ws.edges.numpy())
    T = ws.T_init.clone()
    idx_d, q_d = torch.from_numpy(idx_r).cuda(), q_s.cuda()
    packed = M.gn_pack(plan, P, wd.X_canon, idx_d, q_d)
    H, g, c, nv = M.gn_linearize_packed(plan, P, dtype, T.cuda(), packed)
    torch.cuda.synchronize()
    Hr, gr, cr, nvr = oracle_blocks(ws, T.numpy(), idx_r, q_s, par)
    eh, eg = block_rel_err(H, Hr), block_rel_err(g, gr)
    print(f"packed linearize {dtype}: max H rel {eh.max():.2e}, g rel {eg.max():.2e}")
    assert eh.max() <= BLOCK_RTOL and eg.max() <= BLOCK_RTOL
    assert np.allclose(f64(c), cr, rtol=1e-5)
    assert np.array_equal(nv.cpu().numpy(), nvr)
    H2, g2, c2, nv2 = M.gn_linearize_packed(plan, P, dtype, T.cuda(), packed, per_edge=True)
    assert torch.equal(H, H2) and torch.equal(g, g2) and torch.equal(c, c2)
    # against the gathering form: same sums up to FP32 summation order
    H3, g3, c3, nv3 = M.gn_linearize(plan, P, T.cuda(), wd.X_canon, idx_d, q_d)
    assert block_rel_err(H, H3).max() <= 1e-6 and torch.equal(nv, nv3)


@pytest.mark.parametrize("form,tile", [(0, 8192), (1, 8192), (2, 1024), (2, 4096), (3, 1024), (3, 8192)])
def test_packed_linearize_forms(M, tiny_wl, form, tile):
    """Every packed linearisation form of the FP16 ray family (block-streamed,
    register pipeline, warp-streamed) against the oracle at tile sizes that
    give several tiles per edge with ragged record counts; the per-edge and
    batched launches of a form agree bitwise, and the forms agree up to FP32
    summation order."""
    P = M.default_params()
    par = M.params_dict(P)
    ws = tiny_wl.to_storage(torch.float16)
    idx_r, q_r, _ = oracle_match_all(ws, par, diag=False)
    q_s = torch.from_numpy(q_r).to(torch.float16)
    wd = ws.to("cuda")
    T = ws.T_init.clone().cuda()
    idx_d, q_d = torch.from_numpy(idx_r).cuda(), q_s.cuda()
    plan = M.Plan(ws.kf_hw.numpy(), ws.edges.numpy(), opts={"lin_form": form, "lin_tile": tile})
    packed = M.gn_pack(plan, P, wd.X_canon, idx_d, q_d)
    H, g, c, nv = M.gn_linearize_packed(plan, P, torch.float16, T, packed)
    H2, g2, c2, nv2 = M.gn_linearize_packed(plan, P, torch.float16, T, packed, per_edge=True)
    torch.cuda.synchronize()
    assert torch.equal(H, H2) and torch.equal(g, g2) and torch.equal(c, c2) and torch.equal(nv, nv2)
    Hr, gr, cr, nvr = oracle_blocks(ws, ws.T_init.numpy(), idx_r, q_s, par)
    eh, eg = block_rel_err(H, Hr), block_rel_err(g, gr)
    print(f"packed linearize form {form} tile {tile}: max H rel {eh.max():.2e}, g rel {eg.max():.2e}")
    assert eh.max() <= BLOCK_RTOL and eg.max() <= BLOCK_RTOL
    assert np.allclose(f64(c), cr, rtol=1e-5)
    assert np.array_equal(nv.cpu().numpy(), nvr)
    ref_plan = M.Plan(ws.kf_hw.numpy(), ws.edges.numpy(), opts={"lin_form": 1})
    H3, g3, c3, nv3 = M.gn_linearize_packed(ref_plan, P, torch.float16, T,
                                            M.gn_pack(ref_plan, P, wd.X_canon, idx_d, q_d))
    assert block_rel_err(H, H3).max() <= 1e-6 and block_rel_err(g, g3).max() <= 1e-5 and torch.equal(nv, nv3)
    if form == 3:
        # the prefetching form sums the same records in the same order as form 1
        same = M.Plan(ws.kf_hw.numpy(), ws.edges.numpy(), opts={"lin_form": 1, "lin_tile": tile})
        H4, g4, c4, nv4 = M.gn_linearize_packed(same, P, torch.float16, T, M.gn_pack(same, P, wd.X_canon, idx_d, q_d))
        assert torch.equal(H, H4) and torch.equal(g, g4) and torch.equal(c, c4) and torch.equal(nv, nv4)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_packed_gauss_newton_parity(M, tiny_wl, dtype):
    P = M.default_params()
    par = M.params_dict(P)
    ws = tiny_wl.to_storage(dtype)
    idx_r, q_r, _ = oracle_match_all(ws, par, diag=False)
    q_s = torch.from_numpy(q_r).to(dtype)
    wd = ws.to("cuda")
    plan = M.Plan(ws.kf_hw.numpy(), ws.edges.numpy())
    gn = M.GaussNewton(plan, P, wd.X_canon, torch.from_numpy(idx_r).cuda(), q_s.cuda(), packed=True)
    T_g = gn.run(ws.T_init.cuda(), ws.n_gn_iters).cpu()
    st, T_r, hist, done = oracle.gauss_newton(ws.N, ws.edges.numpy(), ws.kf_off.numpy(), ws.e_off.numpy(),
                                              ws.X_canon, idx_r, q_s, ws.T_init.numpy(), ws.n_gn_iters, **par)
    assert st == 0
    assert_poses_close(T_g, T_r)
    # CUDA-graph capture of pack + iterations replays to the same poses
    T_e = T_g.clone()
    gn.capture(ws.n_gn_iters)
    T_c = gn.replay(ws.T_init.cuda()).cpu()
    assert torch.equal(T_e, T_c)


def test_solve_large_graph_uses_workspace_path(M):
    """A 128-keyframe / 600-edge graph (the largest of the batched workload)
    needs more than a CTA's shared memory for its factor, so the solve takes
    the global-memory path; it must agree with the oracle's dense solve."""
    w = synth.global_graph(N=128, n_pairs=300, H=12, W=16, seed=107)
    P = M.default_params()
    par = M.params_dict(P)
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy())
    assert plan.counts[0] * 49 * 8 > 227 * 1024  # factor blocks exceed shared memory
    idx = w.gt_match.numpy()
    q = w.Q_qry.double().numpy()
    T0 = w.T_init.numpy()
    Hr, gr, _, _ = oracle_blocks(w, T0, idx, q, par)
    H32, g32 = torch.from_numpy(Hr).float(), torch.from_numpy(gr).float()
    T = w.T_init.clone().cuda()
    tau = torch.zeros(w.N, 7, dtype=torch.float64, device="cuda")
    tau, st = M.gn_solve(plan, P, H32.cuda(), g32.cuda(), T, tau=tau)
    torch.cuda.synchronize()
    s, T_r, tau_r = oracle.gn_solve(w.N, w.edges.numpy(), H32.double(), g32.double(), T0)
    assert s == 0 and int(st[0]) in (0, 1)
    assert np.abs(f64(tau) - tau_r).max() <= 1e-8 * max(1.0, np.abs(tau_r).max())
    assert_poses_close(T, T_r, 1e-8)


def test_match_tensor_core_form_agrees_with_per_query_form(M):
    """The two window forms take the same decisions except where the FP32
    summation order of a score decides a near tie: on the tracking frame at
    full size (512 x 384, FP16, radial camera) at most 0.01 % of the valid
    pixels may differ, and the tensor-core form alone meets the oracle's bar."""
    import synth
    from parity import check_disagreements, classify_disagreements
    w = synth.tracking().to_storage(torch.float16)
    wd = w.to("cuda")
    P = M.default_params()
    out = {}
    for form in (0, 1):
        plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), opts={"match_form": form, "match_block_w": 16})
        out[form] = gpu_match(M, plan, P, wd)
    torch.cuda.synchronize()
    a, b = out[0][0].cpu().numpy(), out[1][0].cpu().numpy()
    union = (a >= 0) | (b >= 0)
    diff = int((union & (a != b)).sum())
    print(f"tracking: forms differ on {diff} of {int(union.sum())} valid pixels")
    assert diff <= 1e-4 * union.sum()
    par = M.params_dict(P)
    idx_r, q_r, dg = oracle.match_workload(w, 0, diag=True, **par)
    check_disagreements(classify_disagreements(b, idx_r, dg, par), "tracking, tensor-core form:")
    same = (a == b) & (a >= 0)
    assert torch.equal(out[0][1][torch.from_numpy(same).cuda()], out[1][1][torch.from_numpy(same).cuda()])


@pytest.mark.parametrize("dtype,match_form", [(torch.float32, 0), (torch.float16, 0), (torch.float16, 1),
                                              (torch.float16, 2)])
def test_match_ray_image_path_is_identical(M, dtype, match_form):
    """mslam_match with its ray-image workspace (a1 materialised once, FP32)
    and without it (the rays normalised at the taps) give bit-identical
    matches and confidences, on the batched launch, per-edge launches and an
    edge sub-range; the ray pass covers exactly the edges matched."""
    import synth
    w = synth.global_graph(N=6, n_pairs=6, H=48, W=64, seed=7).to_storage(dtype)
    wd = w.to("cuda")
    P = M.default_params()
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), opts={"match_form": match_form})
    a = gpu_match(M, plan, P, wd, workspace=False)
    b = gpu_match(M, plan, P, wd)
    c = gpu_match(M, plan, P, wd, per_edge=True)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert torch.equal(a[0], c[0]) and torch.equal(a[1], c[1])
    ws = plan.workspace(M._lib.MSLAM_OP_MATCH)
    ws.fill_(255)  # NaN rays wherever the pass does not write
    d_idx = torch.full_like(a[0], -7)
    d_q = torch.zeros_like(a[1])
    gpu_match(M, plan, P, wd, idx_out=d_idx, q_out=d_q, edge_range=(2, 4), workspace=ws)
    sl = slice(int(w.e_off[2]), int(w.e_off[4]))
    assert torch.equal(d_idx[sl], a[0][sl]) and torch.equal(d_q[sl], a[1][sl])


def _match_with(M, w, wd, P, **opts):
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), opts=opts)
    return gpu_match(M, plan, P, wd)


@pytest.mark.parametrize("bw,ppt", [(16, 1), (16, 2), (8, 2), (32, 1)])
def test_match_staged_form_is_identical_full_size(M, bw, ppt):
    """match_form 2 scores the same candidates with the same FP32 dot
    products in the same order as the per-query form, from the block's
    staged box or (outside it) from global memory: matches and confidences
    are bit-identical, on the full-size tracking frame (512 x 384, radial
    camera) and on four edges of the global graph's generator, whatever the
    block shape; with a negative wait limit no copy is issued and every
    window is read from global memory, again with identical results."""
    import synth
    P = M.default_params()
    for w in (synth.tracking().to_storage(torch.float16),
              synth.global_graph(N=8, n_pairs=10, seed=2).to_storage(torch.float16)):
        wd = w.to("cuda")
        ref = _match_with(M, w, wd, P, match_form=0, match_block_w=bw, match_ppt=ppt)
        st = _match_with(M, w, wd, P, match_form=2, match_block_w=bw, match_ppt=ppt)
        torch.cuda.synchronize()
        assert torch.equal(ref[0], st[0]) and torch.equal(ref[1], st[1])
        assert int((ref[0] >= 0).sum()) > 0.05 * ref[0].numel()
    nowait = _match_with(M, w, wd, P, match_form=2, match_block_w=bw, match_ppt=ppt, wait_limit=-1)
    assert torch.equal(ref[0], nowait[0]) and torch.equal(ref[1], nowait[1])


@pytest.mark.parametrize("d", [16, 24, 32])
def test_match_staged_form_scattered_centres(M, d):
    """Random pointmaps send the LM centres of a block all over a 96 x 64
    image, so the bounding box of its windows exceeds the staging capacity:
    the cut box around the mean centre serves the queries whose windows it
    holds and the rest read global memory.  Bit-identical to the per-query
    form for every descriptor size, with a ragged image width (96 is not a
    multiple of 64-wide blocks)."""
    rng = np.random.default_rng(11 + d)
    H, W = 64, 96
    X = np.c_[rng.uniform(-1, 1, H * W), rng.uniform(-1, 1, H * W), rng.uniform(2, 4, H * W)].astype(np.float32)
    Xq = np.c_[rng.uniform(-1, 1, H * W), rng.uniform(-1, 1, H * W), rng.uniform(2, 4, H * W)].astype(np.float32)
    Xq[::7] = 0
    D = rng.normal(size=(2 * H * W, d)).astype(np.float32)
    Q = rng.uniform(1, 10, H * W).astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(torch.float16).cuda()
    P = M.default_params()
    Dr, Dq = M.chunk_descriptors(t(D[:H * W])), M.chunk_descriptors(t(D[H * W:]))
    out = {}
    for form, bw in ((0, 16), (2, 16), (2, 64)):
        plan = M.Plan([[H, W], [H, W]], [[0, 1]], opts={"match_form": form, "match_block_w": bw})
        out[(form, bw)] = M.match(plan, P, t(X), t(Xq), Dr, Dq, t(Q), t(Q))
    torch.cuda.synchronize()
    for k in ((2, 16), (2, 64)):
        assert torch.equal(out[(0, 16)][0], out[k][0]) and torch.equal(out[(0, 16)][1], out[k][1]), k
