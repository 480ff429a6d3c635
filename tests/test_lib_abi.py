"""CPU-only checks of the C ABI: the library builds for sm_103a, loads without
a GPU, exports every function include/mslam.h declares, and its host-side
plan logic (pool offsets, tiles, minimum-degree symbolic factorisation,
argument validation) is right.  No compute call is made."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2412_12392_gb300 import _lib, build
    build.build()
    return _lib.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mslam.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mslam_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    from paper_2412_12392_gb300 import _lib
    names = declared_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(L, n), n
        assert n in _lib.SIGNATURES, f"{n} has no binding signature"


def test_params_struct_layout(L):
    from paper_2412_12392_gb300 import _lib
    p = _lib.Params()
    L.mslam_default_params(C.byref(p))
    assert C.sizeof(p) == 96
    assert _lib.Params.conv_tol.offset == 56 and _lib.Params.residual.offset == 64 and _lib.Params.cy.offset == 92
    assert abs(p.sigma_ray - 0.01) < 1e-8 and p.lm_iters == 10 and list(p.win_dilation)[:2] == [2, 1]
    assert p.residual == _lib.MSLAM_RES_RAY and abs(p.sigma_point - 0.05) < 1e-8 and p.sigma_pixel == 1.0


def plan(kf_hw, edges, graph=None):
    import paper_2412_12392_gb300 as M
    return M.Plan(kf_hw, edges, graph, device="cpu")


def test_plan_offsets_and_tiles(L):
    kf = [[96, 128]] * 3 + [[48, 64]] * 2
    edges = [[0, 1], [1, 2], [2, 0], [3, 4], [4, 3]]
    p = plan(kf, edges, [0, 0, 0, 1, 1])
    assert p.G == 2
    assert list(p.kf_off) == [0, 12288, 24576, 36864, 39936, 43008]
    assert list(p.e_off) == [0, 12288, 24576, 36864, 39936, 43008]
    tiles = sum((h * w + 8191) // 8192 for h, w in [kf[j] for _, j in edges])  # 8192-pixel tiles
    assert p.counts[2] == tiles
    mblocks = sum(((w + 31) // 32) * ((h + 7) // 8) for h, w in [kf[j] for _, j in edges])
    assert p.counts[3] == mblocks
    assert p.order[0] == -1 and p.order[3] == -1


def symbolic_blocks(N, edges, order):
    """Independent symbolic Cholesky: eliminate in the plan's order on a dense
    boolean block pattern; count non-zero blocks of L and update pairs."""
    keep = [k for k in range(N) if order[k] >= 0]
    m = len(keep)
    pos = {k: order[k] for k in keep}
    A = np.zeros((m, m), bool)
    for i, j in edges:
        if i in pos and j in pos:
            A[pos[i], pos[j]] = A[pos[j], pos[i]] = True
    np.fill_diagonal(A, True)
    nnz, trips = 0, 0
    for p in range(m):
        rows = [r for r in range(p + 1, m) if A[r, p]]
        nnz += len(rows)
        trips += len(rows) * (len(rows) + 1) // 2
        for a in rows:
            for b in rows:
                A[a, b] = True
    return m + nnz, trips


@pytest.mark.parametrize("N,n_pairs,seed", [(8, 10, 3), (24, 40, 5), (64, 128, 2), (128, 300, 107)])
def test_symbolic_factorisation_matches_dense_elimination(L, N, n_pairs, seed):
    import synth
    w = synth.global_graph(N=N, n_pairs=n_pairs, H=8, W=8, seed=seed)
    p = plan(w.kf_hw.numpy(), w.edges.numpy())
    nb, nt = symbolic_blocks(N, w.edges.numpy(), p.order)
    assert (p.counts[0], p.counts[1]) == (nb, nt)
    # the ordering is a permutation of the non-fixed keyframes
    assert sorted(p.order[1:]) == list(range(N - 1))
    # minimum degree is no worse than the natural order on these loop
    # graphs, and strictly better once the loop closures give it a choice
    nat = np.r_[-1, np.arange(N - 1)]
    nb_nat, nt_nat = symbolic_blocks(N, w.edges.numpy(), nat)
    assert nt <= nt_nat
    if N >= 64:
        assert nt < nt_nat


@pytest.mark.parametrize("kf,edges,graph", [
    ([[16, 16], [16, 16]], [[0, 0]], None),          # self edge
    ([[16, 16], [16, 16]], [[0, 2]], None),          # out of range
    ([[16, 16], [8, 16]], [[0, 1]], None),           # size mismatch
    ([[16, 16], [16, 16]], [[0, 1]], [0, 1]),        # edge across graphs
    ([[1, 16], [16, 16]], [[0, 1]], None),           # image too small
    ([[16, 16], [16, 16]], [[0, 1]], [0, 2]),        # graph id 1 empty
])
def test_plan_rejects_bad_structure(L, kf, edges, graph):
    from paper_2412_12392_gb300 import _lib
    with pytest.raises(_lib.MslamError) as ei:
        plan(kf, edges, graph)
    assert ei.value.status == _lib.MSLAM_ERR_ARG
    assert _lib.last_error()


def test_calls_reject_unuploaded_plan_and_null_args(L):
    from paper_2412_12392_gb300 import _lib
    p = plan([[16, 16], [16, 16]], [[0, 1]])
    prm = _lib.Params()
    L.mslam_default_params(C.byref(prm))
    st = L.mslam_gn_solve(C.byref(prm), p.handle, None, None, None, None, None, None, 0, None)
    assert st == _lib.MSLAM_ERR_ARG and "uploaded" in _lib.last_error()
    st = L.mslam_match(None, p.handle, 0, 16, *([None] * 11), -1, -1, None, 0, 0, None)
    assert st == _lib.MSLAM_ERR_ARG


def test_every_compute_entry_refuses_bad_arguments_on_the_host(L):
    """Each compute entry point checks its host-visible arguments (NULL
    parameter block, plan or device pointer, a plan never uploaded, an
    unsupported dtype or size) and returns MSLAM_ERR_ARG with a message
    before it touches the device.  (The allocation-free linearisation looks
    up its device first and is covered on the GPU.)"""
    from paper_2412_12392_gb300 import _lib
    p = plan([[8, 16], [8, 16]], [[0, 1]])
    prm = _lib.Params()
    L.mslam_default_params(C.byref(prm))
    P = C.byref(prm)
    N = None
    calls = {
        "gn_linearize": lambda: L.mslam_gn_linearize(P, p.handle, 0, *[N] * 8, N, 0, 0, N),
        "gn_linearize, NULL params": lambda: L.mslam_gn_linearize(N, p.handle, 0, *[N] * 8, N, 0, 0, N),
        "gn_pack": lambda: L.mslam_gn_pack(P, p.handle, 0, N, N, N, N, 0, N),
        "gn_linearize_packed": lambda: L.mslam_gn_linearize_packed(P, p.handle, 1, N, N, 0, *[N] * 6, 0, 0, N),
        "match_stats": lambda: L.mslam_match_stats(p.handle, N, N, N, N, 0, N),
        "gn_backward": lambda: L.mslam_gn_backward(P, p.handle, 0, *[N] * 7, 1.0, N, N, N, N, 0, N),
        "gn_step_backward": lambda: L.mslam_gn_step_backward(P, p.handle, 0, *[N] * 8, 1.0, *[N] * 5, 0, N),
        "gn_solve, NULL plan": lambda: L.mslam_gn_solve(P, N, *[N] * 6, 0, N),
        "match, NULL plan": lambda: L.mslam_match(P, N, 0, 16, *[N] * 11, -1, -1, N, 0, 0, N),
        "desc_to_chunked, d = 8": lambda: L.mslam_desc_to_chunked(0, 8, 16, N, N, 16, N),
        "ray_image, dtype 7": lambda: L.mslam_ray_image(7, 4, N, N, N),
        "ray_image, NULL": lambda: L.mslam_ray_image(0, 4, N, N, N),
        "calib_backproject, NULL": lambda: L.mslam_calib_backproject(0, 1, 8, 8, 1.0, 1.0, 4.0, 4.0, N, N),
        "fuse, NULL": lambda: L.mslam_fuse(0, N, 0, 1, 16, N, N, N, N, N),
        "keyframe_criterion, E < 0": lambda: L.mslam_keyframe_criterion(-1, N, N, N, 0.3, N),
        "keyframe_criterion, NULL": lambda: L.mslam_keyframe_criterion(2, N, N, N, 0.3, N),
        "plan_upload, NULL buffer": lambda: L.mslam_plan_upload(p.handle, N, 0, N),
    }
    for name, call in calls.items():
        assert call() == _lib.MSLAM_ERR_ARG, name
        assert _lib.last_error(), name
    # the size queries answer 0 for a NULL plan or an unknown op
    assert L.mslam_workspace_bytes(N, 0) == 0 and L.mslam_workspace_bytes(p.handle, 99) == 0
    assert L.mslam_plan_kf_pixels(N) == 0 and L.mslam_gn_solve_launches(N) == 0


def test_workspace_sizes_of_each_op(L):
    """mslam_workspace_bytes: the tracking op holds the tile partials (40
    floats per tile, 256-byte aligned) and one counter per edge; unknown ops
    need nothing; a tracking call on a plan that was never uploaded is
    refused before anything is enqueued."""
    from paper_2412_12392_gb300 import _lib
    p = plan([[96, 128], [96, 128]], [[0, 1]])
    n_tiles = int(p.counts[2])
    part = (4 * 40 * n_tiles + 255) // 256 * 256
    assert p.workspace_bytes(_lib.MSLAM_OP_TRACK) == part + 256
    assert p.workspace_bytes(_lib.MSLAM_OP_LINEARIZE) >= part
    assert p.workspace_bytes(99) == 0
    # the match op holds one float4 ray per edge-pool pixel
    bits = (96 * 128 + 32 * 1 + 63) // 32 + 1
    assert p.workspace_bytes(_lib.MSLAM_OP_MATCH) == (16 * 96 * 128 + 255) // 256 * 256 + (4 * bits + 255) // 256 * 256
    prm = _lib.Params()
    L.mslam_default_params(C.byref(prm))
    st = L.mslam_gn_track(C.byref(prm), p.handle, 1, None, None, 0, 1, None, None, 0, None)
    assert st == _lib.MSLAM_ERR_ARG  # not uploaded (no GPU here)


def test_plan_opts_struct_layout(L):
    from paper_2412_12392_gb300 import _lib
    o = _lib.PlanOpts()
    L.mslam_default_plan_opts(C.byref(o))
    assert C.sizeof(o) == 32 and _lib.PlanOpts.match_form.offset == 20 and _lib.PlanOpts.wait_limit.offset == 28
    assert o.match_ppt == 1
    assert o.wait_limit == 0 and o.lin_form == 3 and o.solve_form == 0 and o.match_form == 0
    # every wait limit is accepted: < 0 gives up at once (for the timeout tests), 0 is the default
    for wl in (-1, 0, 1, 1 << 24):
        p = plan([[16, 16]] * 2, [[0, 1]], None) if wl == 0 else None
        import paper_2412_12392_gb300 as M
        q = M.Plan([[16, 16]] * 2, [[0, 1]], device="cpu", opts={"wait_limit": wl})
        assert q.opts["wait_limit"] == wl
        del p, q
