"""NEXT-stage kernels against the oracle: pointmap fusion (Sec. 3.3), the
keyframe-criterion counts (Sec. 3.4), the point residual family (Eq.
track_point) and the known-calibration pixel + depth family with its
back-projection (Sec. 3.6, Eq. backend_pixel)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import BLOCK_RTOL, assert_poses_close, block_rel_err, f64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available()
    from paper_2412_12392_gb300 import build
    build.build()
    import paper_2412_12392_gb300 as M
    return M


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_ray_image_matches_oracle(M, dtype):
    """mslam_ray_image (a1, Sec. 3.1) against the oracle's ray image on the
    stored values: unit rays within the rounding of the output dtype, and the
    zero ray for zero and non-finite points (a ragged count: not a multiple
    of the block size)."""
    g = torch.Generator().manual_seed(7)
    n = 100003
    X = torch.randn(n, 3, generator=g) * torch.exp(torch.randn(n, 1, generator=g))
    X[::97] = 0.0
    X[5::101, 1] = float("nan")
    X[7::103, 2] = float("inf")
    Xs = X.to(dtype)
    R = M.ray_image(Xs.cuda()).cpu()
    Rr = oracle.ray_image(Xs)
    tol = 4e-7 if dtype == torch.float32 else 5e-4
    err = np.abs(f64(R) - Rr).max()
    print(f"ray image {dtype}: max abs err {err:.2e}")
    assert err <= tol
    bad = ~torch.isfinite(Xs).all(dim=1) | (Xs.float().abs().sum(dim=1) == 0)
    assert bool((R[bad] == 0).all())
    # in place (R may alias X)
    Xd = Xs.cuda()
    M.ray_image(Xd, out=Xd)
    assert torch.equal(Xd.cpu(), R)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_fusion_matches_oracle(M, dtype):
    w = synth.tracking(H=96, W=128)
    rng = np.random.default_rng(1)
    n = int(w.kf_off[1])
    Xc = w.X_canon[:n].to(dtype)
    Cc = w.C_canon[:n].to(dtype)
    # the keyframe's points predicted with the frame, in the frame's
    # coordinates: the canonical points moved by T_fk plus noise
    Tk, Tf = w.T_init[0].numpy(), w.T_init[1].numpy()
    Tfk = oracle.sim3_mul(oracle.sim3_inv(Tf), Tk)
    Xkf = np.array([oracle.sim3_act(Tfk, x) for x in w.X_canon[:n].double().numpy()])
    Xkf += rng.normal(size=Xkf.shape) * 0.01
    Xkf[::17] = 0.0
    Ckf = rng.uniform(1, 10, n)
    Ckf[5::23] = -1.0
    Xkf_t = torch.from_numpy(Xkf).to(dtype)
    Ckf_t = torch.from_numpy(Ckf).to(dtype)
    T = w.T_init.cuda()
    Xg, Cg = Xc.cuda().clone(), Cc.cuda().clone()
    M.fuse(T, 0, 1, Xg, Cg, Xkf_t.cuda(), Ckf_t.cuda())
    torch.cuda.synchronize()
    Xr, Cr = oracle.fuse(oracle.sim3_mul(oracle.sim3_inv(Tk), Tf), Xc, Cc, Xkf_t, Ckf_t)
    tol = 2e-6 if dtype == torch.float32 else 2e-3
    assert np.abs(Xg.double().cpu().numpy() - Xr).max() <= tol * np.abs(Xr).max()
    assert np.abs(Cg.double().cpu().numpy() - Cr).max() <= tol * np.abs(Cr).max()
    # untouched pixels are bit-identical
    bad = np.zeros(n, bool)
    bad[::17] = True
    bad[5::23] = True
    assert torch.equal(Xg.cpu()[torch.from_numpy(bad)], Xc[torch.from_numpy(bad)])


def test_match_stats_match_oracle(M):
    """Sec. 3.4 keyframe-criterion counts on the GPU's matches equal the
    oracle's counts of the same indices (exact integers)."""
    w = synth.global_graph(N=6, n_pairs=8, H=48, W=64, seed=4)
    wd = w.to("cuda")
    P = M.default_params()
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy())
    idx, q = M.match(plan, P, wd.X_ref, wd.X_qry, M.chunk_descriptors(wd.D_ref), M.chunk_descriptors(wd.D_qry),
                     wd.Q_ref, wd.Q_qry)
    nv, nu = M.match_stats(plan, idx)
    torch.cuda.synchronize()
    idx_c = idx.cpu().numpy()
    for e in range(w.E):
        v, u = oracle.match_stats(idx_c[w.edge_slice(e)], 48 * 64)
        assert (int(nv[e]), int(nu[e])) == (v, u), e
    # a second call gives the same counts (the bitmap is cleared each call)
    nv2, nu2 = M.match_stats(plan, idx)
    assert torch.equal(nv, nv2) and torch.equal(nu, nu2)


@pytest.mark.parametrize("dtype,match_form,per_edge", [(torch.float32, 0, False), (torch.float16, 0, True),
                                                        (torch.float16, 1, False)])
def test_match_fused_counts(M, dtype, match_form, per_edge):
    """The keyframe counts taken in mslam_match's epilogue equal those of
    mslam_match_stats on the same matches (exact integers): the whole graph
    in one call, then two edge ranges in two calls that share the workspace
    (every edge's bits start on a word of their own), twice in a row."""
    w = synth.global_graph(N=6, n_pairs=8, H=37, W=53, seed=4).to_storage(dtype)  # ragged: 1961 px per edge
    wd = w.to("cuda")
    P = M.default_params()
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), opts={"match_form": match_form})
    Dr, Dq = M.chunk_descriptors(wd.D_ref), M.chunk_descriptors(wd.D_qry)
    ws = plan.workspace(M._lib.MSLAM_OP_MATCH)
    nv = torch.full((w.E,), -5, dtype=torch.int32, device="cuda")
    nu = torch.full((w.E,), -5, dtype=torch.int32, device="cuda")
    idx, q = M.match(plan, P, wd.X_ref, wd.X_qry, Dr, Dq, wd.Q_ref, wd.Q_qry, workspace=ws, counts=(nv, nu),
                     per_edge=per_edge)
    rv, ru = M.match_stats(plan, idx)
    torch.cuda.synchronize()
    assert torch.equal(nv, rv) and torch.equal(nu, ru)
    assert int(rv.sum()) > 0
    for _ in range(2):
        nv2 = torch.full_like(nv, -5)
        nu2 = torch.full_like(nu, -5)
        half = w.E // 2
        for r in ((0, half), (half, w.E)):
            idx2, _ = M.match(plan, P, wd.X_ref, wd.X_qry, Dr, Dq, wd.Q_ref, wd.Q_qry, workspace=ws,
                              counts=(nv2, nu2), edge_range=r)
        torch.cuda.synchronize()
        assert torch.equal(nv2, rv) and torch.equal(nu2, ru)


def calibration(w):
    """The generator's pinhole camera (tiny workload: k1 = 0)."""
    H, W = int(w.kf_hw[0, 0]), int(w.kf_hw[0, 1])
    return dict(fx=0.8 * W, fy=0.8 * W, cx=(W - 1) / 2.0, cy=(H - 1) / 2.0)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_calib_backproject_matches_oracle(M, tiny_wl, dtype):
    w = tiny_wl
    H, W = int(w.kf_hw[0, 0]), int(w.kf_hw[0, 1])
    K = calibration(w)
    X = w.X_canon.to(dtype).view(w.N, H, W, 3)
    Xg = M.calib_backproject(X.cuda().clone(), **K).cpu()
    for k in range(w.N):
        Xr = oracle.calib_backproject(H, W, K["fx"], K["fy"], K["cx"], K["cy"], X[k].reshape(-1, 3))
        err = np.abs(Xg[k].reshape(-1, 3).double().numpy() - Xr)
        tol = 1e-6 if dtype == torch.float32 else 1e-3
        assert (err <= tol * (np.abs(Xr) + 1e-3)).all(), err.max()
        # the depth is kept bit for bit
        assert torch.equal(Xg[k][..., 2], X[k][..., 2])


def family_params(M, w, fam):
    if fam == "point":
        return M.default_params(residual=M._lib.MSLAM_RES_POINT)
    return M.default_params(residual=M._lib.MSLAM_RES_PIXEL, **calibration(w))


def family_inputs(M, w, fam, dtype):
    """Storage-dtype inputs; the pixel family's keyframes are back-projected
    on the GPU first and both sides consume the stored result."""
    ws = w.to_storage(dtype)
    X = ws.X_canon.cuda().clone()
    if fam == "pixel":
        H, W = int(w.kf_hw[0, 0]), int(w.kf_hw[0, 1])
        M.calib_backproject(X.view(w.N, H, W, 3), **calibration(w))
    idx = ws.gt_match.clone()
    q = (ws.Q_qry.float() * 0.5 + 1.0).to(dtype)
    return ws, X, idx, q


@pytest.mark.parametrize("fam", ["point", "pixel"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_family_linearize_matches_oracle(M, tiny_wl, fam, dtype):
    w = tiny_wl
    P = family_params(M, w, fam)
    par = M.params_dict(P)
    ws, X, idx, q = family_inputs(M, w, fam, dtype)
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy())
    T = ws.T_init.clone()
    H, g, c, nv = M.gn_linearize(plan, P, T.cuda(), X, idx.cuda(), q.cuda())
    packed = M.gn_pack(plan, P, X, idx.cuda(), q.cuda())
    Hp, gp, cp, nvp = M.gn_linearize_packed(plan, P, dtype, T.cuda(), packed)
    torch.cuda.synchronize()
    Xc = X.cpu()
    W = int(w.kf_hw[0, 1])
    Hr, gr, cr, nvr = [], [], [], []
    for e in range(w.E):
        i, j = int(w.edges[e, 0]), int(w.edges[e, 1])
        sl = w.edge_slice(e)
        out = oracle.linearize_edge(T[i], T[j], Xc[w.kf_slice(i)], Xc[w.kf_slice(j)], idx[sl], q[sl], img_w=W, **par)
        Hr.append(out[0]), gr.append(out[1]), cr.append(out[2]), nvr.append(out[3])
    Hr, gr = np.array(Hr), np.array(gr)
    for name, (Hg, gg, cg, ng) in {"gather": (H, g, c, nv), "packed": (Hp, gp, cp, nvp)}.items():
        eh, eg = block_rel_err(Hg, Hr), block_rel_err(gg, gr)
        print(f"{fam} {dtype} {name}: H rel {eh.max():.2e}, g rel {eg.max():.2e}, matches {ng.tolist()}")
        assert eh.max() <= BLOCK_RTOL and eg.max() <= BLOCK_RTOL
        assert np.allclose(f64(cg), cr, rtol=1e-5)
        assert ng.cpu().tolist() == nvr
        assert min(nvr) > 1000


@pytest.mark.parametrize("fam", ["point", "pixel"])
def test_family_gauss_newton_matches_oracle(M, tiny_wl, fam):
    w = tiny_wl
    dtype = torch.float16
    P = family_params(M, w, fam)
    par = M.params_dict(P)
    ws, X, idx, q = family_inputs(M, w, fam, dtype)
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy())
    gn = M.GaussNewton(plan, P, X, idx.cuda(), q.cuda(), packed=True)
    T_g = gn.run(ws.T_init.cuda(), ws.n_gn_iters).cpu()
    W = int(w.kf_hw[0, 1])
    st, T_r, hist, done = oracle.gauss_newton(w.N, w.edges.numpy(), w.kf_off.numpy(), w.e_off.numpy(), X.cpu(),
                                              idx, q, ws.T_init.numpy(), ws.n_gn_iters, img_w=W, **par)
    assert st == 0
    e = assert_poses_close(T_g, T_r)
    print(f"{fam} GN vs oracle (rot, trans, scale): {e.max(axis=0)}")


def test_family_argument_errors(M, tiny_wl):
    w = tiny_wl
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy())
    ws, X, idx, q = family_inputs(M, w, "point", torch.float32)
    T = ws.T_init.cuda()
    with pytest.raises(M._lib.MslamError):
        M.gn_linearize(plan, M.default_params(residual=7), T, X, idx.cuda(), q.cuda())
    with pytest.raises(M._lib.MslamError):  # the pixel family needs a calibration
        M.gn_linearize(plan, M.default_params(residual=M._lib.MSLAM_RES_PIXEL), T, X, idx.cuda(), q.cuda())
    with pytest.raises(M._lib.MslamError):  # the adjoint covers the ray family only
        M.gn_backward(plan, family_params(M, w, "point"), T, X, idx.cuda(), q.cuda(), dL_dcost=1.0)
    # FP16 records carry pixel coordinates exactly only up to 2048
    big = M.Plan(np.array([[2, 4096], [2, 4096]], np.int32), np.array([[0, 1]], np.int32))
    Xb = torch.ones(2 * 8192, 3, dtype=torch.float16, device="cuda")
    with pytest.raises(M._lib.MslamError):
        M.gn_pack(big, family_params(M, w, "pixel"), Xb, torch.zeros(8192, dtype=torch.int32, device="cuda"),
                  torch.full((8192,), 5.0, dtype=torch.float16, device="cuda"))


def test_gn_track_several_frames(M):
    """mslam_gn_track on three tracking problems in one plan (small images,
    ragged tile counts): each frame's poses against the oracle's Gauss-Newton
    run on that problem alone, fed the same matches; a plan that is not of
    the tracking form is refused before any launch."""
    from paper_2412_12392_gb300 import _lib
    ws = [synth.tracking(seed=s, H=96, W=128).to_storage(torch.float16) for s in (1, 5, 9)]
    mw = synth.merge(ws, name="frames")
    P = M.default_params()
    par = M.params_dict(P)
    plan = M.Plan(mw.kf_hw.numpy(), mw.edges.numpy(), mw.graph_of_kf.numpy(), opts={"lin_tile": 1024})
    wd = mw.to("cuda")
    ms = [oracle.match_workload(w, 0, **par) for w in ws]
    idx = torch.from_numpy(np.concatenate([m[0] for m in ms])).cuda()
    q = torch.from_numpy(np.concatenate([m[1] for m in ms])).to(torch.float16).cuda()
    gn = M.GaussNewton(plan, P, wd.X_canon, idx, q, packed=True)
    iters = ws[0].n_gn_iters
    T_f = gn.run_tracking(mw.T_init.cuda(), iters).cpu()
    assert bool((gn.status.cpu() >= 0).all()) and bool((gn.status.cpu() <= 1).all())
    for k, w in enumerate(ws):
        sl = slice(int(mw.e_off[k]), int(mw.e_off[k + 1]))
        st, T_r, _, _ = oracle.gauss_newton(w.N, w.edges.numpy(), w.kf_off.numpy(), w.e_off.numpy(), w.X_canon,
                                            idx[sl].cpu(), q[sl].cpu(), w.T_init.numpy(), iters, **par)
        assert st == 0
        assert_poses_close(T_f[2 * k:2 * k + 2], T_r)
        assert torch.equal(T_f[2 * k], w.T_init[0])  # the keyframe is the fixed gauge
    g = synth.global_graph(N=4, n_pairs=3, H=24, W=32)
    plan_g = M.Plan(g.kf_hw.numpy(), g.edges.numpy())
    gd = g.to("cuda")
    gn_g = M.GaussNewton(plan_g, P, gd.X_canon, torch.full((plan_g.edge_pixels,), -1, dtype=torch.int32, device="cuda"),
                         torch.zeros(plan_g.edge_pixels, device="cuda"), packed=True)
    with pytest.raises(_lib.MslamError):
        gn_g.run_tracking(g.T_init.cuda(), 2)


def test_gn_track_without_matches_is_not_pd(M):
    """A tracking frame with no valid match has a zero 7 x 7 system: the
    mixed-precision solve declines it (no positive diagonal), the FP64
    factorisation reports MSLAM_ERR_NOT_PD, and neither pose moves."""
    from paper_2412_12392_gb300 import _lib
    w = synth.tracking(seed=2, H=96, W=128).to_storage(torch.float16)
    P = M.default_params()
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), opts={"lin_tile": 1024})
    wd = w.to("cuda")
    idx = torch.full((plan.edge_pixels,), -1, dtype=torch.int32, device="cuda")
    q = torch.zeros(plan.edge_pixels, dtype=torch.float16, device="cuda")
    gn = M.GaussNewton(plan, P, wd.X_canon, idx, q, packed=True)
    T = gn.run_tracking(w.T_init.cuda(), 3).cpu()
    assert int(gn.status[0]) == _lib.MSLAM_ERR_NOT_PD
    assert torch.equal(T, w.T_init)


@pytest.mark.parametrize("dtype,d", [(torch.float16, 24), (torch.float32, 16), (torch.float16, 32)])
def test_desc_to_chunked_is_the_permutation(M, dtype, d):
    """mslam_desc_to_chunked (whole pool and a slice of a larger pool) equals
    the [P, d] -> [d / c, P, c] permutation bit for bit."""
    g = torch.Generator(device="cpu").manual_seed(3)
    P = 5003
    D = torch.randn(P, d, generator=g).to(dtype)
    c = 16 // D.element_size()
    ref = D.reshape(P, d // c, c).permute(1, 0, 2).contiguous()
    got = M.chunk_descriptors(D.cuda())
    assert torch.equal(got.cpu(), ref)
    pool = torch.zeros(d // c, P + 300, c, dtype=dtype, device="cuda")
    M.chunk_descriptors(D[1000:2000].cuda(), out=pool, p0=150)
    assert torch.equal(pool[:, 150:1150].cpu(), ref[:, 1000:2000])
    assert not pool[:, :150].any() and not pool[:, 1150:].any()
