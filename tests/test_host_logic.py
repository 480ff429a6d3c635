"""Host-side logic of the benchmark and the workload generator (CPU only)."""
import sys
import types

import torch

import synth


def test_batched_storage_equals_merged_graphs():
    """The batched workload made graph by graph in FP16 equals merging the
    eight FP32 graphs and casting afterwards (the cast is exact either way)."""
    a = synth.batched_storage("cpu", torch.float16, scale=32)
    b = synth.merge([g.to_storage(torch.float16) for g in synth.batched("cpu", scale=32)], name="batched")
    assert a.N == b.N == sum(synth.gen.BATCHED_KF) and a.E == b.E == sum(synth.gen.BATCHED_EDGES)
    for k in ("kf_hw", "edges", "graph_of_kf", "kf_off", "e_off", "T_init", "X_canon", "X_ref", "X_qry", "D_ref",
              "D_qry", "Q_ref", "Q_qry", "gt_match"):
        assert torch.equal(getattr(a, k), getattr(b, k)), k
    assert a.meta["graph_kf"] == synth.gen.BATCHED_KF and a.meta["graph_edges"] == synth.gen.BATCHED_EDGES


def _bench():
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        import bench
    finally:
        sys.argv = argv
    return bench


def test_workload_names():
    bench = _bench()
    t = synth.tiny()
    assert bench.workload_name(t) == "tiny: 4 keyframes, 3 directed edges, 128x96, d=16, 10 GN iters"
    m = synth.merge([synth.tiny(), synth.tiny(seed=3)], name="batched")
    assert bench.workload_name(m).startswith("batched: 2 graphs, 8 keyframes (4/4), 6 directed edges (3/3), 128x96")


def test_pipelined_shape_check_needs_a_streamed_choice():
    """The pipelined shape check runs only when the autotuner chose a
    linearisation form other than the plain register pipeline (a streamed
    form, or the prefetching one: both hold shared memory while the next
    batch's matching runs beside them); it compares against the best plain
    register-pipeline shape by the autotuner's own score (iterations x
    linearise + pack)."""
    bench = _bench()
    assert bench.pick_pipelined_shapes(types.SimpleNamespace(tuning=None), 1) is None
    regs = types.SimpleNamespace(tuning={"opts": {"lin_form": 1}})
    assert bench.pick_pipelined_shapes(regs, 1) is None


def test_bench_pose_errors_agree_with_the_oracle_algebra():
    """The benchmark's pose-accuracy figures (quaternion algebra in numpy)
    equal those of the test helper built on the oracle's Sim(3) product and
    inverse, on random poses."""
    import numpy as np

    from parity import pose_errors as oracle_pose_errors
    bench = _bench()
    rng = np.random.default_rng(4)
    A, B = [], []
    for _ in range(16):
        for L in (A, B):
            q = rng.normal(size=4)
            q /= np.linalg.norm(q)
            L.append(np.concatenate([rng.normal(size=3), q, [rng.uniform(0.5, 2.0)]]))
    A, B = np.array(A), np.array(B)
    B[:4] = A[:4]  # identical poses give zero error
    e1 = bench.pose_errors(A, B)
    e2 = oracle_pose_errors(A, B)
    assert np.allclose(e1, e2, rtol=1e-9, atol=1e-12)
    assert np.all(e1[:4] <= 1e-12)


def test_valid_query_pixels_counts_finite_nonzero_points():
    bench = _bench()
    X = torch.tensor([[0.0, 0.0, 0.0], [1.0, 2.0, 3.0], [float("nan"), 1.0, 1.0], [0.0, 0.0, -1e-3],
                      [float("inf"), 0.0, 0.0]], dtype=torch.float16)
    assert bench.valid_query_pixels(X) == 2
