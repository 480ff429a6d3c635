"""The batched workload at full size (8 independent graphs, 488 keyframes,
1,926 directed edges, 512 x 384 and 256 x 192, FP16 storage) in one plan, in
the launch configuration the benchmark keeps for it (the prefetching
register-pipeline linearisation with 16384-pixel tiles, 8 x 32 match blocks
with two query pixels per thread); the warp-streamed linearisation with
4096-pixel tiles, an earlier choice, gives the same poses within the pose
bar (the two forms add the Hessian sums in different FP32 orders; measured
2e-8 rad and 1.7e-6 relative translation apart):

* the batched matching launch on sampled query pixels of three edges per
  graph against the oracle: agreement over all sampled pixels valid on
  either side >= 99.9 %, with disagreements explained only by an LM iterate
  still moving (the loop trajectories of these graphs leave more of them
  than the single 64-keyframe graph) and unexplained ones each capped
  (tests/parity.py);
* the poses of graph 0 (16 keyframes, 40 edges, 512 x 384) and graph 1 (24
  keyframes, 64 edges, 256 x 192) after 10 Gauss-Newton iterations of the
  one batched plan, against the oracle's Gauss-Newton run on that graph
  alone and fed the same matches.  The plan's largest graph (128 keyframes,
  600 edges) has an FP32 factor too large for one SM's shared memory, so
  the mixed-precision solve factors every graph in place in the workspace
  (with FP64 refinement); the oracle on that graph would take minutes of
  host time, so its solve is covered by the structure test in
  test_gpu_fullsize.py instead.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import add_counts, assert_poses_close, check_disagreements, classify_disagreements

pytestmark = pytest.mark.gpu

OPTS = {"lin_form": 3, "lin_tile": 16384, "lin_blocks_per_sm": 2, "match_block_w": 8, "match_ppt": 2}
OPTS_WARP = {"lin_form": 2, "lin_tile": 4096, "match_block_w": 16}


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available()
    from paper_2412_12392_gb300 import build
    build.build()
    import paper_2412_12392_gb300 as M
    return M


@pytest.fixture(scope="module")
def batched_wl():
    return synth.batched_storage("cuda", torch.float16)


def _graph_slices(w, g):
    """Keyframe and edge ranges of graph g in the merged pools."""
    kf0 = int(sum(w.meta["graph_kf"][:g]))
    e0 = int(sum(w.meta["graph_edges"][:g]))
    return kf0, kf0 + w.meta["graph_kf"][g], e0, e0 + w.meta["graph_edges"][g]


def test_batched_full_size(M, batched_wl):
    w = batched_wl
    assert len(w.meta["graphs"]) == 8 and w.E == 1926
    P = M.default_params()
    par = M.params_dict(P)
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), w.graph_of_kf.numpy(), opts=OPTS)
    assert plan.G == 8
    Dr, Dq = M.chunk_descriptors(w.D_ref), M.chunk_descriptors(w.D_qry)
    idx_g, q_g = M.match(plan, P, w.X_ref, w.X_qry, Dr, Dq, w.Q_ref, w.Q_qry)  # one launch for all graphs
    torch.cuda.synchronize()
    del Dr, Dq

    # matching: 16384 sampled query pixels of three edges of every graph
    rng = np.random.default_rng(1)
    tot = {}
    for g in range(8):
        kf0, kf1, e0, e1 = _graph_slices(w, g)
        for e in rng.choice(np.arange(e0, e1), 3, replace=False):
            e = int(e)
            H, W = int(w.kf_hw[int(w.edges[e, 1]), 0]), int(w.kf_hw[int(w.edges[e, 1]), 1])
            sl = w.edge_slice(e)
            cpu = {k: getattr(w, k)[sl].cpu() for k in ("X_ref", "X_qry", "D_ref", "D_qry", "Q_ref", "Q_qry")}
            pix = np.sort(rng.choice(H * W, 16384, replace=False))
            idx_r, q_r, dg = oracle.match(H, W, cpu["X_ref"], cpu["X_qry"], cpu["D_ref"], cpu["D_qry"], cpu["Q_ref"],
                                          cpu["Q_qry"], pix=pix, diag=True, **par)
            c = classify_disagreements(idx_g[sl].cpu().numpy()[pix], idx_r, dg, par)
            print(f"graph {g} edge {e} ({W}x{H}): {c}")
            tot = add_counts(tot, c)
    check_disagreements(tot, "sampled total:")

    # Gauss-Newton of all eight graphs in the one plan
    gn = M.GaussNewton(plan, P, w.X_canon, idx_g, q_g, packed=True)
    T_g = gn.run(w.T_init.cuda(), w.n_gn_iters).cpu()
    status = gn.status.cpu()
    assert bool((status >= 0).all()) and bool((status <= 1).all()), status
    # the warp-streamed linearisation on the same matches: the same poses up
    # to the FP32 summation order of the Hessian sums
    plan_w = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), w.graph_of_kf.numpy(), opts=OPTS_WARP)
    gn_w = M.GaussNewton(plan_w, P, w.X_canon, idx_g, q_g, packed=True)
    T_w = gn_w.run(w.T_init.cuda(), w.n_gn_iters).cpu()
    e_w = assert_poses_close(T_w, T_g)
    print(f"warp-streamed against prefetching linearisation, all poses (rot, trans, scale): {e_w.max(axis=0)}")
    del gn_w, plan_w
    idx_c, q_c = idx_g.cpu(), q_g.cpu()
    for g in (0, 1):
        kf0, kf1, e0, e1 = _graph_slices(w, g)
        edges = w.edges[e0:e1].numpy() - kf0
        kf_off = w.kf_off[kf0:kf1 + 1] - w.kf_off[kf0]
        e_off = w.e_off[e0:e1 + 1] - w.e_off[e0]
        pool = slice(int(w.e_off[e0]), int(w.e_off[e1]))
        Xc = w.X_canon[int(w.kf_off[kf0]):int(w.kf_off[kf1])].cpu()
        st, T_r, hist, done = oracle.gauss_newton(kf1 - kf0, edges, kf_off.numpy(), e_off.numpy(), Xc, idx_c[pool],
                                                  q_c[pool], w.T_init[kf0:kf1].numpy(), w.n_gn_iters, **par)
        assert st == 0
        e = assert_poses_close(T_g[kf0:kf1], T_r)
        assert torch.equal(T_g[kf0], w.T_init[kf0])  # each graph's first keyframe is fixed
        print(f"graph {g} ({kf1 - kf0} keyframes, {e1 - e0} edges): poses vs oracle (rot, trans, scale) "
              f"{e.max(axis=0)}")
