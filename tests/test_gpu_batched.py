"""Batched form over several independent keyframe graphs (the structure of
the batched workload: 8 graphs with 16..128 keyframes and 40..600 directed
edges, mixed resolutions, here at reduced image sizes): one launch per stage
for all graphs, each graph against the oracle run on that graph alone; and
the autotuner's choice gives the same poses as the default launch shapes."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import MATCH_AGREE, assert_poses_close, match_agreement

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available()
    from paper_2412_12392_gb300 import build
    build.build()
    import paper_2412_12392_gb300 as M
    return M


@pytest.fixture(scope="module")
def graphs():
    return synth.batched(device="cuda", scale=8)


def test_batched_graphs_against_oracle_per_graph(M, graphs):
    P = M.default_params()
    par = M.params_dict(P)
    mw = synth.merge(graphs)
    plan = M.Plan(mw.kf_hw.numpy(), mw.edges.numpy(), mw.graph_of_kf.numpy())
    assert plan.G == 8
    wd = mw.to("cuda")
    idx_g, q_g = M.match(plan, P, wd.X_ref, wd.X_qry, M.chunk_descriptors(wd.D_ref), M.chunk_descriptors(wd.D_qry),
                         wd.Q_ref, wd.Q_qry)
    # oracle matches per graph, stitched into the merged pools
    idx_all, q_all = [], []
    tot_dis = tot_union = 0
    for w in graphs:
        for e in range(w.E):
            i_r, q_r = oracle.match_workload(w, e, **par)
            idx_all.append(i_r)
            q_all.append(q_r)
    idx_r = np.concatenate(idx_all)
    q_r = np.concatenate(q_all)
    agree, ndis, nunion, _ = match_agreement(idx_g, idx_r)
    assert agree >= MATCH_AGREE, agree
    gn = M.GaussNewton(plan, P, wd.X_canon, torch.from_numpy(idx_r).cuda(),
                       torch.from_numpy(q_r).float().cuda(), packed=True)
    T_g = gn.run(mw.T_init.cuda(), 10).cpu()
    assert bool((gn.status.cpu() >= 0).all()) and bool((gn.status.cpu() <= 1).all())
    base = 0
    eb = 0
    for w in graphs:
        sl = slice(int(w.e_off[0]) + int(mw.e_off[eb]), int(mw.e_off[eb + w.E]))
        st, T_r, _, _ = oracle.gauss_newton(w.N, w.edges.numpy(), w.kf_off.numpy(), w.e_off.numpy(), w.X_canon,
                                            idx_r[sl], q_r[sl].astype(np.float32), w.T_init.numpy(), 10, **par)
        assert st == 0
        assert_poses_close(T_g[base:base + w.N], T_r)
        assert torch.equal(T_g[base], w.T_init[0])  # each graph's first keyframe is fixed
        base += w.N
        eb += w.E


def test_autotuner_choice_is_equivalent(M, graphs):
    from paper_2412_12392_gb300.autotune import LIN_TILES, MATCH_WIDTHS, WARP_STREAM_TILES, autotune
    P = M.default_params()
    mw = synth.merge(graphs[:4])
    wd = mw.to("cuda")
    Dr, Dq = M.chunk_descriptors(wd.D_ref), M.chunk_descriptors(wd.D_qry)
    T0 = mw.T_init.cuda()
    rep = autotune(mw.kf_hw.numpy(), mw.edges.numpy(), mw.graph_of_kf.numpy(), P, wd.X_ref, wd.X_qry, Dr, Dq,
                   wd.Q_ref, wd.Q_qry, wd.X_canon, T0, reps=2)
    opts = rep["opts"]
    assert opts["match_block_w"] in MATCH_WIDTHS
    assert opts["lin_tile"] in set(LIN_TILES) | {32768, 65536} | set(WARP_STREAM_TILES)
    assert opts["lin_form"] in (0, 1, 2, 3)
    out = []
    for o in (None, opts):
        plan = M.Plan(mw.kf_hw.numpy(), mw.edges.numpy(), mw.graph_of_kf.numpy(), opts=o)
        idx, q = M.match(plan, P, wd.X_ref, wd.X_qry, Dr, Dq, wd.Q_ref, wd.Q_qry)
        gn = M.GaussNewton(plan, P, wd.X_canon, idx, q, packed=True)
        out.append((idx.clone(), gn.run(T0, 10).cpu()))
    assert torch.equal(out[0][0], out[1][0])  # matching does not depend on the block shape
    assert_poses_close(out[1][1], out[0][1], 1e-6)
