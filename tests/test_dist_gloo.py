"""Replica (weak-scaling) logic of bench.py across ranks, on CPU with the gloo
backend and world size 2: each rank builds an independent graph replica,
runs its own work (here the oracle's Gauss-Newton on a small replica), and
the job reports max-over-ranks time and summed matched pixels, with no
collective on the data path."""
import os
import socket
from argparse import Namespace

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    args = Namespace(workload="global", small=True)
    w = bench.make_workload(args, rank, "cpu", hw=(24, 32))
    par = dict(oracle.DEFAULT_PARAMS)
    idx = w.gt_match.numpy()
    q = w.Q_qry.double().numpy()
    st, T, hist, done = oracle.gauss_newton(w.N, w.edges.numpy(), w.kf_off.numpy(), w.e_off.numpy(), w.X_canon,
                                            idx, q, w.T_init.numpy(), 3, **par)
    n_matched = int((idx >= 0).sum())
    fake_ms = 10.0 * (rank + 1)
    ms = bench.max_over_ranks(fake_ms, world)
    tot = bench.sum_over_ranks(float(n_matched), world)
    # gather a fingerprint of each replica's data to check independence
    fp = torch.tensor([float(w.X_canon.double().sum())], dtype=torch.float64)
    fps = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(fps, fp)
    out[rank] = dict(status=st, ms=ms, tot=tot, n=n_matched, fps=[float(f) for f in fps],
                     improved=bool(hist[-1] < hist[0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    assert r0["status"] == 0 and r1["status"] == 0 and r0["improved"] and r1["improved"]
    assert r0["ms"] == r1["ms"] == 20.0                      # max over ranks
    assert r0["tot"] == r1["tot"] == r0["n"] + r1["n"]       # whole-job work
    assert r0["fps"][0] != r0["fps"][1]                      # independent replicas
