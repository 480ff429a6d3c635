"""Benchmark of the hot path: projective matching over every edge of a keyframe
graph followed by Gauss-Newton iterations (linearise + gauge-fixed Cholesky
solve + retraction), on seeded synthetic 512 x 384 pointmaps.

One step = mslam_match over all edges + n_gn x (mslam_gn_linearize,
mslam_gn_solve).  value = matched-pixel GN iterations per second over the
whole step (matching time included), summed over ranks.  Prints one JSON
line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mslam|reference]
                  [--workload global|tracking|batched] [--form batched|plain]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "matched-pixel GN iters/s + matches/s @512x384, batched vs plain, % HBM peak"
FP32_LANES_PER_SM = 128
L1_BYTES_PER_CLK = 128  # one 128-byte data-stage wavefront per clock and SM


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mslam", choices=["mslam", "reference"])
    ap.add_argument("--workload", default="global", choices=["global", "tracking", "batched"],
                    help="batched: 8 independent graphs (16-128 keyframes, 40-600 edges, 1,926 in all) in one plan; "
                         "reports the device-resident step only (no plain, end-to-end or CPU legs)")
    ap.add_argument("--form", default="batched", choices=["batched", "plain"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 per-edge comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--small", action="store_true", help="a reduced graph (8 keyframes) for profiling")
    ap.add_argument("--hw", default="384x512", help="image size HxW (smaller sizes keep the graph for profiling)")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes instead of the autotuner's")
    ap.add_argument("--opts", default="",
                    help="fixed plan launch shapes instead of the autotuner, e.g. match_block_w=16,lin_tile=32768")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay timing")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the tracking-frame and adjoint measurements reported beside the headline")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="only the adjoint measurement on the differentiation graph at --hw (for profiling)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- setup

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def workload_name(w) -> str:
    if "graphs" in w.meta:
        sizes = sorted({f"{int(W)}x{int(H)}" for H, W in w.kf_hw.tolist()}, reverse=True)
        return (f"{w.name}: {len(w.meta['graphs'])} graphs, {w.N} keyframes ({'/'.join(map(str, w.meta['graph_kf']))}), "
                f"{w.E} directed edges ({'/'.join(map(str, w.meta['graph_edges']))}), {' and '.join(sizes)}, d={w.d}, "
                f"{w.n_gn_iters} GN iters")
    return (f"{w.name}: {w.N} keyframes, {w.E} directed edges, {int(w.kf_hw[0, 1])}x{int(w.kf_hw[0, 0])}, d={w.d}, "
            f"{w.n_gn_iters} GN iters")


def make_workload(args, rank: int, device, hw=None):
    """This rank's replica: an independent graph (seed offset by rank), so the
    per-GPU work is fixed as ranks are added (weak scaling)."""
    import synth
    H, W = hw if hw is not None else (384, 512)
    if args.workload == "tracking":
        return synth.tracking(device=device, seed=1 + 1000 * rank, H=H, W=W)
    if args.workload == "batched":
        return synth.batched_storage(device, torch.float16, seed_offset=1000 * rank)
    if args.small:
        return synth.global_graph(device=device, seed=2 + 1000 * rank, N=8, n_pairs=12, H=H, W=W)
    return synth.global_graph(device=device, seed=2 + 1000 * rank, H=H, W=W)


# DRAM bytes (read + write) per query pixel of one batched matching launch,
# from one ncu capture of match_kernel<__half, 24, 3, 2> (8 keyframes, 24
# edges, 512x384, the FP32 ray image: 344,033,024 bytes for 4,718,592 query
# pixels), scaled to a launch by its query pixels.  Remove an entry when its
# kernel changes.
NCU_DRAM_BYTES_PER_QUERY_PX = {("match", 2, 24): 344033024 / 4718592}
# DRAM bytes per matched pixel of one packed linearisation launch, FP16
# records, scaled to a launch by its matches (1,637,856 matches in each
# capture, 8 keyframes / 24 edges at 512x384): lin_packed_kernel (16384-record
# tiles, 2 CTAs per SM: 26,254,592 bytes), its prefetching form (lin_form 3,
# the same shape: 26,256,128 bytes) and lin_warp_stream_kernel (4096-record
# tiles: 26,328,064 bytes).
NCU_DRAM_BYTES_PER_MATCH = {("lin_packed", 2): 26254592 / 1637856, ("lin_packed_prefetch", 2): 26256128 / 1637856,
                            ("lin_warp_stream", 2): 26328064 / 1637856}


def valid_query_pixels(X_qry: torch.Tensor) -> int:
    """Query points the matching kernel works on: finite and not zero."""
    x = X_qry.float()
    ok = torch.isfinite(x).all(dim=1) & ((x * x).sum(dim=1) > 0)
    return int(ok.sum())


def _qmul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Hamilton product of quaternions stored x y z w."""
    ax, ay, az, aw = a[..., 0], a[..., 1], a[..., 2], a[..., 3]
    bx, by, bz, bw = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([aw * bx + ax * bw + ay * bz - az * by, aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw, aw * bw - ax * bx - ay * by - az * bz], axis=-1)


def pose_errors(T_a, T_b) -> np.ndarray:
    """Per pose of two [N, 8] Sim(3) arrays (t, q xyzw, s): rotation angle of
    R_a R_b^T (rad), |t_a - t_b| / max(|t_b|, 0.1 m), |s_a - s_b| / s_b (the
    parity tests' definition)."""
    A = np.asarray(T_a.cpu() if torch.is_tensor(T_a) else T_a, dtype=np.float64).reshape(-1, 8)
    B = np.asarray(T_b.cpu() if torch.is_tensor(T_b) else T_b, dtype=np.float64).reshape(-1, 8)
    qb_inv = B[:, 3:7] * np.array([-1.0, -1.0, -1.0, 1.0])
    dq = _qmul(A[:, 3:7], qb_inv)
    rot = 2.0 * np.arcsin(np.minimum(1.0, np.linalg.norm(dq[:, :3], axis=1)))
    tr = np.linalg.norm(A[:, :3] - B[:, :3], axis=1) / np.maximum(np.linalg.norm(B[:, :3], axis=1), 0.1)
    sc = np.abs(A[:, 7] - B[:, 7]) / np.abs(B[:, 7])
    return np.stack([rot, tr, sc], axis=1)


def _err_summary(e: np.ndarray) -> dict:
    """Max and median over poses of (rotation rad, relative translation, relative scale)."""
    return {"rot_rad_max": float(e[:, 0].max()), "trans_rel_max": float(e[:, 1].max()),
            "scale_rel_max": float(e[:, 2].max()), "rot_rad_median": float(np.median(e[:, 0])),
            "trans_rel_median": float(np.median(e[:, 1])), "scale_rel_median": float(np.median(e[:, 2]))}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = open(os.path.join(ROOT, f".clocks_{os.getpid()}.csv"), "w+")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        res = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return res
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [r.strip().split(",") for r in self.out.read().strip().splitlines() if r.strip()]
        name = self.out.name
        self.out.close()
        os.remove(name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip() == "Active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if sm:
            res = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return res


# ----------------------------------------------------------------------------- GPU arm

class Arm:
    """Device-resident inputs and buffers of one launch form."""

    def __init__(self, M, w, dtype, per_edge: bool, autotune: bool = False, opts=None):
        self.M, self.w, self.per_edge = M, w, per_edge
        self.P = M.default_params()
        self.wd = w if w.X_canon.dtype == dtype else w.to_storage(dtype)
        # descriptors in the kernel's chunk-planar layout (a one-off layout change)
        self.Dr = M.chunk_descriptors(self.wd.D_ref)
        self.Dq = M.chunk_descriptors(self.wd.D_qry)
        self.tuning = None
        if autotune:
            from paper_2412_12392_gb300.autotune import autotune as tune
            wd = self.wd
            self.tuning = tune(w.kf_hw.numpy(), w.edges.numpy(), w.graph_of_kf.numpy(), self.P, wd.X_ref, wd.X_qry,
                               self.Dr, self.Dq, wd.Q_ref, wd.Q_qry, wd.X_canon, w.T_init.to(wd.X_canon.device))
            opts = self.tuning["opts"]
        dev = self.wd.X_canon.device
        self.T0 = w.T_init.to(dev)
        self.iters = w.n_gn_iters
        self.set_opts(opts, dtype)

    def set_opts(self, opts, dtype=None):
        """(Re)build the plan with these launch shapes, on the same inputs."""
        M, w = self.M, self.w
        dtype = dtype or self.q.dtype
        dev = self.wd.X_canon.device
        self.plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy(), w.graph_of_kf.numpy(), opts=opts)
        self.idx = torch.empty(self.plan.edge_pixels, dtype=torch.int32, device=dev)
        self.q = torch.empty(self.plan.edge_pixels, dtype=dtype, device=dev)
        self.ws_match = self.plan.workspace(M._lib.MSLAM_OP_MATCH)
        # the batched form gathers the used matches once per step and streams
        # them in every iteration; the plain form gathers in every iteration
        self.gn = M.GaussNewton(self.plan, self.P, self.wd.X_canon, self.idx, self.q, per_edge=self.per_edge,
                                packed=not self.per_edge)

    def match(self):
        wd = self.wd
        self.M.match(self.plan, self.P, wd.X_ref, wd.X_qry, self.Dr, self.Dq, wd.Q_ref, wd.Q_qry,
                     idx_out=self.idx, q_out=self.q, per_edge=self.per_edge, workspace=self.ws_match)

    def step(self, ev=None):
        """One pass of the hot path; ev = optional list collecting
        (match_start, match_end, [(lin_start, lin_end)]) CUDA events."""
        self.gn.T.copy_(self.T0)
        self.gn.status.zero_()
        if ev is None:
            self.match()
            self.gn.pack()
            for _ in range(self.iters):
                self.gn.step()
            return
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        self.match()
        e[1].record()
        self.gn.pack()
        e[2].record()
        lins = []
        for _ in range(self.iters):
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record()
            self.gn.linearize()
            b.record()
            self.gn.solve()
            c.record()
            lins.append((a, b, c))
        ev.append((e[0], e[1], e[2], lins))

    def capture(self):
        """Capture one whole step (pose reset, matching, packing and the GN
        iterations) into a CUDA graph; step_graph() replays it."""
        dev = self.wd.X_canon.device
        s = torch.cuda.Stream(dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            self.step()  # warm-up outside capture
        torch.cuda.current_stream(dev).wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step()
        self.graph = g

    def step_graph(self, ev=None):
        self.graph.replay()

    def run_pipelined(self, n: int):
        """n whole steps with two batches in flight: batch k+1's matching
        runs on a low-priority stream beside batch k's Gauss-Newton loop
        (whose solve occupies one SM per graph), and packing waits for both
        its batch's matches and the previous loop.  Every step does all of
        its work; only the ordering across steps changes."""
        if not hasattr(self, "streams"):
            dev = self.wd.X_canon.device
            lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -1)
            self.streams = (torch.cuda.Stream(dev, priority=lo), torch.cuda.Stream(dev, priority=hi))
        sm, sg = self.streams
        cur = torch.cuda.current_stream()
        sm.wait_stream(cur)
        sg.wait_stream(cur)
        packed = None
        for _ in range(n):
            with torch.cuda.stream(sm):
                if packed is not None:
                    sm.wait_event(packed)  # the previous batch's matches are packed
                self.match()
                matched = torch.cuda.Event()
                matched.record(sm)
            with torch.cuda.stream(sg):
                sg.wait_event(matched)
                self.gn.T.copy_(self.T0)
                self.gn.status.zero_()
                self.gn.pack()
                packed = torch.cuda.Event()
                packed.record(sg)
                for _ in range(self.iters):
                    self.gn.step()
        cur.wait_stream(sm)
        cur.wait_stream(sg)

    def launches_per_step(self) -> int:
        """Kernels of this library launched per step: the ray image and match; (batched) pack;
        per iteration the relative-pose, tile and finalize kernels of the
        linearisation (per edge in the plain form) and the solve."""
        E = self.plan.E
        sl = self.plan.solve_launches
        if self.per_edge:
            return 2 * E + self.iters * (1 + 2 * E + sl)
        return 2 + 1 + self.iters * (3 + sl)


def pick_pipelined_shapes(arm, world, steps: int = 5, warmup: int = 3):
    """The autotuner ranks the linearisation shapes one stage at a time.  With
    two batches in flight the linearisation also shares the SMs with the next
    batch's matching, and the shared memory a streamed or prefetching form
    holds shrinks the L1 the matching kernel reads its windows from.  Time
    the autotuner's choice and its best plain register-pipeline shape as
    pipelined steps and keep the faster (the same work either way; only the
    launch shapes differ)."""
    rep = arm.tuning
    need = rep is not None and rep["opts"].get("lin_form") != 1
    if world > 1:
        # every rank takes part in the timing collectives if any rank needs them
        need = max_over_ranks(1.0 if need else 0.0, world) > 0.0
    if not need or rep is None:
        return None
    best, key_best = float("inf"), None
    for key, ms in rep["lin_ms"].items():
        tile, bps, form = key.split("/")
        if form != "regs":
            continue
        score = arm.iters * ms + rep["pack_ms"][int(tile) if int(tile) in rep["pack_ms"] else tile]
        if score < best:
            best, key_best = score, (int(tile), int(bps))
    if key_best is None:
        return None
    chosen = dict(rep["opts"])
    alt = dict(chosen, lin_tile=key_best[0], lin_blocks_per_sm=key_best[1], lin_form=1)
    times = {}
    for name, o in (("autotuned", chosen), ("register_pipeline", alt)):
        arm.set_opts(o)
        times[name], _, _ = time_steps(arm, steps, warmup, world, None, pipelined=True)
        times[name] = max_over_ranks(times[name], world)
    keep = min(times, key=times.get)
    arm.set_opts(chosen if keep == "autotuned" else alt)
    arm.step()
    torch.cuda.synchronize()
    return {"pipelined_ms": times, "kept": keep, "opts": dict(arm.plan.opts)}


def time_steps(arm, steps, warmup, world, sampler=None, with_events=True, graph=False, pipelined=False):
    """Mean time of a step over `steps` steps after `warmup` untimed steps;
    with events, also the mean time of each stage (eager launches); with
    graph, the steps are replays of the captured CUDA graph; pipelined, the
    steps run with two batches in flight (Arm.run_pipelined)."""
    step = arm.step_graph if graph else arm.step
    if pipelined:
        arm.run_pipelined(warmup)
    else:
        for _ in range(warmup):
            step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ev = [] if with_events and not pipelined else None
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    if sampler:
        sampler.start()
    t0.record()
    if pipelined:
        arm.run_pipelined(steps)
    else:
        for _ in range(steps):
            step(ev)
    t1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    barrier(world)
    ms = t0.elapsed_time(t1) / steps
    stats = None
    if ev:
        match_ms = np.mean([a.elapsed_time(b) for a, b, _, _ in ev])
        pack_ms = np.mean([b.elapsed_time(c) for _, b, c, _ in ev])
        lin_ms = np.mean([a.elapsed_time(b) for _, _, _, L in ev for a, b, c in L])
        solve_ms = np.mean([b.elapsed_time(c) for _, _, _, L in ev for a, b, c in L])
        stats = dict(match_ms=float(match_ms), pack_ms=float(pack_ms), lin_ms=float(lin_ms),
                     solve_ms=float(solve_ms))
    return ms, stats, clocks


def run_gpu(args, world, rank, local):
    import paper_2412_12392_gb300 as M
    from paper_2412_12392_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hw = tuple(int(v) for v in args.hw.lower().split("x"))
    w = make_workload(args, rank, dev, hw=hw)
    dtype = torch.float16 if args.form == "batched" else torch.float32
    fixed = {k: int(v) for k, v in (kv.split("=") for kv in args.opts.split(",") if kv)} or None
    arm = Arm(M, w, dtype, per_edge=(args.form == "plain"),
              autotune=(args.form == "batched" and not args.no_autotune and fixed is None), opts=fixed)
    arm.step()
    torch.cuda.synchronize()
    n_matched = int(((arm.idx >= 0) & (arm.q.float() > arm.P.q_min)).sum())
    n_query = int(arm.plan.edge_pixels)
    peaks, peak_src = measured_peaks()
    sampler = ClockSampler(local) if rank == 0 else None
    pipe_pick = None
    if args.form == "batched" and arm.tuning is not None:
        pipe_pick = pick_pipelined_shapes(arm, world)
    # one step at a time, with CUDA events between the stages
    serial_ms, stats, _ = time_steps(arm, args.steps, args.warmup, world, None)
    serial_ms = max_over_ranks(serial_ms, world)
    T_serial = arm.gn.T.clone()
    # the headline: the same steps with two batches in flight
    ms, _, clocks = time_steps(arm, args.steps, args.warmup, world, sampler, pipelined=True)
    ms = max_over_ranks(ms, world)
    same_result = bool(torch.equal(arm.gn.T, T_serial))
    graph_ms = None
    if args.form == "batched" and not args.no_graph:
        # the same step captured once as a CUDA graph and replayed
        arm.capture()
        graph_ms, _, _ = time_steps(arm, args.steps, args.warmup, world, None, with_events=False, graph=True)
        graph_ms = max_over_ranks(graph_ms, world)
    tot_matched = sum_over_ranks(n_matched, world)
    tot_query = sum_over_ranks(n_query, world)
    value = tot_matched * arm.iters / (ms * 1e-3)
    # per-kernel rooflines (algorithmic bytes / flops per launch over the
    # CUDA-event duration of that launch in the timed region)
    d = w.d
    esz = 2 if dtype == torch.float16 else 4
    lin_bytes = n_matched * (6 * esz + 4 + esz)      # X_i[m], X_j[n], idx, q
    # the matching kernel returns at once (idx -1, q 0) for a query point that
    # is zero or not finite (the overlap band of each edge zeroes whole
    # columns): such a query moves X_qry, idx and q only and does no
    # arithmetic; every other query runs the LM iterations and the windows
    n_valid_query = valid_query_pixels(arm.wd.X_qry)
    per_valid_flop = w.n_match_iters * 80 + arm.P.n_levels * (2 * arm.P.win_radius + 1) ** 2 * 2 * d
    match_bytes = n_query * (3 * esz + 4 + esz) + n_valid_query * (3 * esz + 2 * d * esz + 2 * esz)
    match_flop = n_valid_query * per_valid_flop
    hbm = float(peaks["hbm_gbs"])
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = nsm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    lin_gbs = lin_bytes / (stats["lin_ms"] * 1e-3) / 1e9
    match_tfs = match_flop / (stats["match_ms"] * 1e-3) / 1e12
    lf = arm.plan.opts.get("lin_form")
    lin_kernel = ("lin_tiles" if args.form != "batched" else "lin_packed" if (esz == 4 or lf == 1)
                  else "lin_packed_prefetch" if lf == 3 else "lin_stream" if lf == 0 else "lin_warp_stream")
    traffic_m = NCU_DRAM_BYTES_PER_MATCH.get((lin_kernel, esz))
    rl_lin = {"kernel": "gn_linearize", "launch": lin_kernel, "bound": "hbm", "achieved": round(lin_gbs, 1),
              "peak": hbm, "unit": "GB/s", "frac": round(lin_gbs / hbm, 4),
              "traffic": int(traffic_m * n_matched) if traffic_m else None,
              "algorithmic_bytes": int(lin_bytes), "ms": round(stats["lin_ms"], 4),
              "peak_source": f"{peak_src} hbm_gbs",
              "note": "ms and achieved: the whole linearisation call (relative poses, tile kernel, finalize)"}
    if args.form == "batched":
        c_ms, k_ms = lin_kernel_only_ms(M, arm)
        k_gbs = lin_bytes / (k_ms * 1e-3) / 1e9
        rl_lin["kernel_only"] = {"ms": round(k_ms, 4), "achieved": round(k_gbs, 1), "frac": round(k_gbs / hbm, 4),
                                 "call_ms_in_graph": round(c_ms, 4),
                                 "method": "20 calls replayed as one CUDA graph, minus the same calls on a packed "
                                           "buffer with zero records (relative-pose and finalize launches, empty "
                                           "tile loop)"}
    traffic_px = NCU_DRAM_BYTES_PER_QUERY_PX.get(("match", esz, d)) if args.form == "batched" else None
    rl_match = {"kernel": "match", "bound": "alu", "achieved": round(match_tfs, 2), "peak": round(fp32_peak, 1),
                "unit": "TFLOP/s", "frac": round(match_tfs / fp32_peak, 4),
                "traffic": int(traffic_px * n_query) if traffic_px else None,
                "algorithmic_flop": int(match_flop), "algorithmic_bytes": int(match_bytes),
                "valid_query_pixels": int(n_valid_query), "flop_per_valid_query": int(per_valid_flop),
                "dense_frac_if_every_query_ran": round(n_query * per_valid_flop / (stats["match_ms"] * 1e-3) / 1e12
                                                       / fp32_peak, 4),
                "hbm_frac": round(match_bytes / (stats["match_ms"] * 1e-3) / 1e9 / hbm, 4),
                "ms": round(stats["match_ms"], 4),
                "peak_source": f"FP32 FMA: {nsm} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_mhz:.0f} MHz"}
    # the unit that actually limits the kernel: the L1 data stage serving the
    # window candidates (n_levels x (2r+1)^2 descriptors of d elements) and
    # the LM taps (lm_iters x 4 unit rays of 16 bytes) of every valid query
    l1_per_query = arm.P.n_levels * (2 * arm.P.win_radius + 1) ** 2 * d * esz + w.n_match_iters * 4 * 16
    l1_peak = nsm * L1_BYTES_PER_CLK * sm_mhz * 1e6 / 1e9
    l1_gbs = n_valid_query * l1_per_query / (stats["match_ms"] * 1e-3) / 1e9
    rl_match["l1"] = {"bound": "l1", "achieved": round(l1_gbs, 1), "peak": round(l1_peak, 1), "unit": "GB/s",
                      "frac": round(l1_gbs / l1_peak, 4), "bytes_per_valid_query": int(l1_per_query),
                      "peak_source": f"L1 data stage: {nsm} SMs x {L1_BYTES_PER_CLK} B x {sm_mhz:.0f} MHz"}
    lin_share = stats["lin_ms"] * arm.iters
    dominant = rl_match if stats["match_ms"] >= lin_share else rl_lin
    out = {
        "metric": METRIC, "value": value, "unit": "matched-pixel GN iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16-storage/f32-math/f64-solve" if esz == 2 else
        "f32/f64-solve", "data": "synthetic (seeded box-room pointmaps, no network or dataset)",
        "config": {"workload": workload_name(w),
                   "form": args.form, "launch_shapes": arm.plan.opts, "global_batch": w.E, "seq_len": None,
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (per-step edge pools of several GB)"},
        "matches_per_s": tot_query / (stats["match_ms"] * 1e-3) if stats else None,
        "gn_iters_per_s_gn_only": tot_matched * arm.iters / (((stats["lin_ms"] + stats["solve_ms"]) * arm.iters
                                                              + stats["pack_ms"]) * 1e-3),
        "stage_ms": {k: round(v, 4) for k, v in stats.items()},
        "matched_pixels": n_matched, "query_pixels": n_query,
        "roofline": dominant, "roofline_kernels": [rl_match, rl_lin],
        "pipelining": {"serial_ms_per_step": serial_ms, "serial_value": tot_matched * arm.iters / (serial_ms * 1e-3),
                       "same_result_as_serial": same_result, "shape_check": pipe_pick,
                       "note": "headline steps run with two batches in flight: batch k+1's matching on a "
                               "low-priority stream beside batch k's Gauss-Newton loop; serial = one step "
                               "at a time (the stage times are from the serial run)"},
        "cuda_graph": None if graph_ms is None else {
            "ms_per_step": graph_ms, "value": tot_matched * arm.iters / (graph_ms * 1e-3),
            "note": "the whole step captured once as a CUDA graph and replayed"},
        "gpu_launches": arm.launches_per_step() * args.steps,
        "clocks": clocks,
    }
    return out, arm, w


def lin_kernel_only_ms(M, arm, reps: int = 20):
    """The tile kernel's share of a linearisation call, free of host launch
    gaps: `reps` calls captured in one CUDA graph, replayed, against the same
    calls on a copy of the packed buffer whose per-tile record counts are
    zero (the relative-pose and finalize launches and an empty persistent
    tile loop).  Returns (call ms, kernel ms), both per call."""
    gn, plan = arm.gn, arm.plan
    empty = gn.pack_buf.clone()
    n_tiles = int(plan.counts[2])
    cnt_bytes = (4 * n_tiles + 255) // 256 * 256
    nb = M.pack_bytes(plan, arm.wd.X_canon.dtype)
    empty[nb - cnt_bytes:nb].zero_()

    def graph_ms(buf):
        call = lambda: M.gn_linearize_packed(plan, arm.P, arm.wd.X_canon.dtype, gn.T, buf, gn.H, gn.g, gn.cost,
                                             gn.n_valid, gn.ws_lin)
        call()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(reps):
                call()
        return _event_ms(g.replay, 3) / reps

    full, over = graph_ms(gn.pack_buf), graph_ms(empty)
    gn.linearize()  # the blocks of the real records again
    torch.cuda.synchronize()
    return full, max(full - over, 1e-6)


def accuracy_report(M, arm, plain, w):
    """Final poses of the two forms after a whole step, against each other
    and the synthetic ground truth, and what FP16 storage changes against
    the FP32-storage form (whose matches, blocks and poses the parity tests
    hold to the FP64 oracle within 99.9 % / 1e-5 / 1e-5).  The FP16 form's
    error against the FP64 oracle is therefore within the parity bars of
    this difference."""
    arm.step()
    plain.step()
    torch.cuda.synchronize()
    Tb, Tp, Tgt = arm.gn.T.cpu(), plain.gn.T.cpu(), w.T_gt
    acc = {"batched_fp16_vs_ground_truth": _err_summary(pose_errors(Tb, Tgt)[1:]),
           "plain_fp32_vs_ground_truth": _err_summary(pose_errors(Tp, Tgt)[1:]),
           "batched_fp16_vs_plain_fp32": _err_summary(pose_errors(Tb, Tp)[1:]),
           "init_vs_ground_truth": _err_summary(pose_errors(w.T_init, Tgt)[1:]),
           "note": "poses after one whole step (matching + 10 GN iterations) of each form; keyframe 0 is "
                   "fixed in both and left out"}
    # storage error: matches of the two forms, then both linearisations at the
    # initial poses on the FP32 form's matches (q rounded to FP16 for the FP16 form)
    gi, pi = arm.idx.cpu().numpy(), plain.idx.cpu().numpy()
    union = (gi >= 0) | (pi >= 0)
    agree = 1.0 - float(np.sum(union & (gi != pi))) / max(int(union.sum()), 1)
    T0 = arm.T0
    Hp, gp, _, _ = M.gn_linearize(plain.plan, plain.P, T0, plain.wd.X_canon, plain.idx, plain.q)
    Hb, gbb, _, _ = M.gn_linearize(arm.plan, arm.P, T0, arm.wd.X_canon, plain.idx, plain.q.half())
    torch.cuda.synchronize()

    def rel(a, b):
        a, b = a.double().reshape(a.shape[0], -1), b.double().reshape(b.shape[0], -1)
        return (torch.linalg.norm(a - b, dim=1) / torch.linalg.norm(b, dim=1).clamp_min(1e-300)).cpu().numpy()

    eh, eg = rel(Hb, Hp), rel(gbb, gp)
    st = {"match_agreement_fp16_vs_fp32": agree, "union_valid_pixels": int(union.sum()),
          "H_block_rel_median": float(np.median(eh)), "H_block_rel_max": float(eh.max()),
          "g_block_rel_median": float(np.median(eg)), "g_block_rel_max": float(eg.max()),
          "poses": acc["batched_fp16_vs_plain_fp32"],
          "note": "FP16-storage form against the FP32-storage form on the same workload; the blocks are "
                  "both linearisations at the initial poses on the FP32 form's matches"}
    return acc, st


def e2e_measure(args, M, w, dtype, world, rank, local, opts=None, n_chunks: int = 8, n_copy_streams: int = 4):
    """Same metric through the public API with host (pinned) inputs copied in
    and the poses copied out inside the timed region.  The copies run on a
    copy stream into two alternating device input sets, in edge chunks, so
    that a step's matching starts on its first chunk while the rest is still
    arriving and the next step's inputs arrive during this step's
    Gauss-Newton loop (double buffering); every byte of every step is still
    copied inside the timed region."""
    dev = torch.device("cuda", local)
    wh = w.to_storage(dtype).to("cpu")
    pools = ["X_ref", "X_qry", "D_ref", "D_qry", "Q_ref", "Q_qry"]
    # host inputs as a network writes them (descriptors [P, d]); the copies
    # land in natural-layout staging buffers and mslam_desc_to_chunked builds
    # the kernel's chunk-planar layout on the device, inside the timed region
    host = {k: getattr(wh, k).pin_memory() for k in pools + ["X_canon"]}
    T_host = w.T_init.cpu().pin_memory()
    arm = Arm(M, w, dtype, per_edge=False, opts=opts)
    sets = [{k: torch.empty_like(host[k], device=dev) for k in host} for _ in range(2)]
    c_el = 16 // host["D_ref"].element_size()
    chunked = [{k: torch.empty(w.d // c_el, host[k].shape[0], c_el, dtype=host[k].dtype, device=dev)
                for k in ("D_ref", "D_qry")} for _ in range(2)]
    T_out = [torch.empty_like(T_host).pin_memory() for _ in range(2)]
    h2d = sum(t.numel() * t.element_size() for t in host.values()) + T_host.numel() * 8
    d2h = T_out[0].numel() * 8
    e_off = w.e_off.numpy()
    bounds = np.linspace(0, w.E, n_chunks + 1).round().astype(int)
    chunks = [(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
    # copy streams take chunks in turn, so that several copy engines run
    copy_streams = [torch.cuda.Stream(device=dev) for _ in range(n_copy_streams)]
    compute = torch.cuda.current_stream(dev)
    free = [torch.cuda.Event(), torch.cuda.Event()]  # a set's inputs are no longer read
    for ev in free:
        ev.record(compute)

    def copy_inputs(si):
        """Copy stream: one step's inputs into set si, chunk by chunk."""
        dst = sets[si]
        done = []
        for cs in copy_streams:
            cs.wait_event(free[si])
        with torch.cuda.stream(copy_streams[-1]):
            dst["X_canon"].copy_(host["X_canon"], non_blocking=True)
            xev = torch.cuda.Event()
            xev.record(copy_streams[-1])
        for ci, (e0, e1) in enumerate(chunks):
            cs = copy_streams[ci % len(copy_streams)]
            with torch.cuda.stream(cs):
                p0, p1 = int(e_off[e0]), int(e_off[e1])
                for k in pools:
                    dst[k][p0:p1].copy_(host[k][p0:p1], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(cs)
                done.append(ev)
        return done, xev

    def compute_step(si, copies, out):
        done, xev = copies
        src = sets[si]
        arm.gn.T.copy_(T_host, non_blocking=True)
        arm.gn.status.zero_()
        dch = chunked[si]
        for (e0, e1), ev in zip(chunks, done):
            compute.wait_event(ev)
            p0, p1 = int(e_off[e0]), int(e_off[e1])
            for k in ("D_ref", "D_qry"):
                M.chunk_descriptors(src[k][p0:p1], out=dch[k], p0=p0)
            M.match(arm.plan, arm.P, src["X_ref"], src["X_qry"], dch["D_ref"], dch["D_qry"], src["Q_ref"],
                    src["Q_qry"], idx_out=arm.idx, q_out=arm.q, edge_range=(e0, e1), workspace=arm.ws_match)
        compute.wait_event(xev)
        arm.gn.X.copy_(src["X_canon"], non_blocking=True)
        arm.gn.pack()
        free[si].record(compute)
        for _ in range(arm.iters):
            arm.gn.step()
        out.copy_(arm.gn.T, non_blocking=True)

    def run(n):
        for s in range(n):
            done = copy_inputs(s % 2)
            compute_step(s % 2, done, T_out[s % 2])

    run(max(1, args.warmup))
    torch.cuda.synchronize()
    # the host-to-device copy rate of this machine, for context: one large
    # pinned copy of the reference descriptors
    probe = host["D_ref"]
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(compute)
    sets[0]["D_ref"].copy_(probe, non_blocking=True)
    c1.record(compute)
    torch.cuda.synchronize()
    h2d_gbs = probe.numel() * probe.element_size() / (c0.elapsed_time(c1) * 1e-3) / 1e9
    barrier(world)
    steps = max(2, args.steps)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(compute)
    for cs in copy_streams:
        cs.wait_event(t0)
    run(steps)
    t1.record(compute)
    torch.cuda.synchronize()
    ms = max_over_ranks(t0.elapsed_time(t1) / steps, world)
    # the result of the last step against the same step run without the pipeline
    arm.step()
    torch.cuda.synchronize()
    same = bool(torch.equal(T_out[(steps - 1) % 2].to(dev), arm.gn.T))
    n_matched = int(((arm.idx >= 0) & (arm.q.float() > arm.P.q_min)).sum())
    val = sum_over_ranks(n_matched, world) * arm.iters / (ms * 1e-3)
    return {"value": val, "unit": "matched-pixel GN iters/s", "ms_per_step": ms, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "copy": f"pinned host, {len(chunks)} edge chunks per step on "
            f"{len(copy_streams)} copy streams, double-buffered device inputs; descriptors arrive as [P, d] and "
            f"are put in the kernel's chunk-planar layout by mslam_desc_to_chunked inside the timed region",
            "same_result_as_device_resident_step": same, "h2d_gbs_single_copy": round(h2d_gbs, 1)}


# ----------------------------------------------------------------------------- oracle arm

def oracle_sample(w, seconds: float, n_gn_iters: int, par: dict, seed: int = 0):
    """Time the FP64 oracle on a bounded sample of the workload: matching of
    sampled query pixels, then linearisation + solve on whole edges.  Returns
    (matched-pixel GN iters/s for the whole step at the workload's mix,
    matches/s, details)."""
    import oracle
    rng = np.random.default_rng(seed)
    # matching: sampled pixels of the first edges
    e = 0
    H, W = int(w.kf_hw[0, 0]), int(w.kf_hw[0, 1])
    t_match, n_match = 0.0, 0
    budget = seconds * 0.5
    idx_all = {}
    while t_match < budget and e < w.E:
        pix = np.sort(rng.choice(H * W, size=min(H * W, 32768), replace=False))
        t = time.perf_counter()
        idx, q = oracle.match_workload(w, e, pix=pix, **par)
        t_match += time.perf_counter() - t
        n_match += len(pix)
        e += 1
    # GN: full linearisation of whole edges with ground-truth matches + one solve
    t_gn, n_px_it = 0.0, 0
    T = w.T_init.numpy()
    e = 0
    H14, g14 = [], []
    while t_gn < seconds * 0.5 and e < w.E:
        i, j = int(w.edges[e, 0]), int(w.edges[e, 1])
        sl = w.edge_slice(e)
        idx = w.gt_match[sl].numpy()
        q = w.Q_qry[sl].double().numpy()
        t = time.perf_counter()
        Hb, gb, c, nv = oracle.linearize_edge(T[i], T[j], w.X_canon[w.kf_slice(i)], w.X_canon[w.kf_slice(j)], idx,
                                              q, **par)
        t_gn += time.perf_counter() - t
        n_px_it += nv
        H14.append(Hb)
        g14.append(gb)
        e += 1
    t = time.perf_counter()
    oracle.gn_solve(w.N, w.edges.numpy()[:e], np.array(H14), np.array(g14), T)
    t_solve = time.perf_counter() - t
    t_match_px = t_match / max(n_match, 1)
    t_gn_px = t_gn / max(n_px_it, 1)
    return t_match_px, t_gn_px, t_solve, dict(match_pixels=n_match, gn_pixel_iters=n_px_it, edges_linearised=e)


def cpu_baseline(w, seconds, n_matched_total, n_query_total, iters, par):
    import oracle
    tm, tg, ts, det = oracle_sample(w, seconds, iters, par)
    step_s = n_query_total * tm + n_matched_total * iters * tg + iters * ts
    val = n_matched_total * iters / step_s
    return {"value": val, "unit": "matched-pixel GN iters/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"FP64 C oracle (OpenMP): matching of {det['match_pixels']} sampled query pixels and "
                       f"linearisation of {det['edges_linearised']} whole edges ({det['gn_pixel_iters']} matched "
                       f"pixel-iterations) plus one solve, scaled to the full step's pixel counts"),
            "matches_per_s": 1.0 / tm}


def run_reference(args, world, rank):
    """The oracle as the reference arm, on the host cores."""
    if rank != 0:
        return None
    import oracle
    import synth
    oracle.build()
    # the synthetic inputs are made with torch on the GPU when there is one
    # (minutes of host time otherwise) and handed to the oracle on the host;
    # no kernel of this library runs in this arm
    gen_dev = "cuda" if torch.cuda.is_available() else "cpu"
    w = make_workload(args, 0, gen_dev).to("cpu")
    if gen_dev == "cuda":
        torch.cuda.empty_cache()
    par = dict(oracle.DEFAULT_PARAMS)
    n_query = int(w.e_off[-1])
    n_matched = int((w.gt_match >= 0).sum())
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(w, per_step, w.n_gn_iters, par)
    times = []
    t0 = time.perf_counter()
    for k in range(args.steps):
        tm, tg, ts, det = oracle_sample(w, per_step, w.n_gn_iters, par, seed=k)
        times.append(n_query * tm + n_matched * w.n_gn_iters * tg + w.n_gn_iters * ts)
    wall = time.perf_counter() - t0
    step_s = float(np.mean(times))
    val = n_matched * w.n_gn_iters / step_s
    cb = {"value": val, "unit": "matched-pixel GN iters/s", "cores": oracle.num_threads(), "kind": "oracle",
          "sample": f"each step: about {per_step:.0f} s of FP64 oracle matching and linearisation on sampled "
                    f"pixels/edges, scaled to the full step"}
    return {"metric": METRIC, "value": val, "unit": "matched-pixel GN iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(w), "parallelism": "host cores (OpenMP)"},
            "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": val, "unit": "matched-pixel GN iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}, "wall_s": wall,
            "ms_per_step_kind": "projected: the oracle's measured time per matched query pixel and per matched "
                                "pixel-iteration (on the sampled pixels and edges of each step) times the full "
                                "step's pixel counts; a whole step is not run"}


def _event_ms(fn, reps: int) -> float:
    """Mean CUDA-event time of fn() on the current stream after one warm-up."""
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tracking_frame(M, dev, peaks) -> dict:
    """One tracking frame (Sec. 3.3) at 512 x 384, FP16 storage, radial
    camera: matching of the frame against its keyframe, packing, and 20
    Gauss-Newton iterations on the ray error (1 edge, the keyframe fixed)."""
    import synth
    w = synth.tracking(device=dev)
    arm = Arm(M, w, torch.float16, per_edge=False, autotune=True)
    ms = _event_ms(arm.step, 20)
    ev = []
    arm.step(ev)
    torch.cuda.synchronize()
    m0, m1, p1, lins = ev[0]
    n_matched = int(((arm.idx >= 0) & (arm.q.float() > arm.P.q_min)).sum())
    # the frame's launches (a few microseconds of work each) replayed as one CUDA graph
    arm.capture()
    gms = _event_ms(arm.step_graph, 20)
    # the fused tracking loop: match, pack, then one launch per GN iteration,
    # with 2048-pixel tiles (96 tiles: fewer partials for the finishing block to add)
    M_ = arm.M
    plan_t = M_.Plan(w.kf_hw.numpy(), w.edges.numpy(), opts=dict(arm.plan.opts, lin_tile=2048))
    gn_t = M_.GaussNewton(plan_t, arm.P, arm.wd.X_canon, arm.idx, arm.q, packed=True)

    def fused():
        arm.match()
        gn_t.run_tracking(arm.T0, arm.iters)
    fms = _event_ms(fused, 20)
    T_fused = gn_t.T.clone()
    dev_ = arm.wd.X_canon.device
    s_ = torch.cuda.Stream(dev_)
    s_.wait_stream(torch.cuda.current_stream(dev_))
    with torch.cuda.stream(s_):
        fused()
    torch.cuda.current_stream(dev_).wait_stream(s_)
    torch.cuda.synchronize()
    fg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(fg):
        fused()
    fgms = _event_ms(fg.replay, 20)
    fused_same = bool(torch.equal(gn_t.T, T_fused))
    return {"workload": "tracking: 1 frame against 1 keyframe, 512x384, radial camera, d=24, 20 GN iters",
            "ms_per_frame": ms, "ms_per_frame_cuda_graph": gms,
            "ms_per_frame_fused": fms, "ms_per_frame_fused_cuda_graph": fgms, "fused_replay_same_result": fused_same,
            "match_ms": m0.elapsed_time(m1),
            "pack_ms": m1.elapsed_time(p1), "gn_iter_ms": float(np.mean([a.elapsed_time(c) for a, b, c in lins])),
            "matched_pixels": n_matched, "launches_per_frame": arm.launches_per_step(),
            "launch_shapes": arm.plan.opts}


def adjoint_measure(M, dev, peaks, img_h=384, img_w=512) -> dict:
    """The adjoint (a9) on the differentiation workload (32 keyframes, 96
    edges, 512 x 384 unless smaller, FP16 storage): gradient of c E_g +
    a . tau (one GN step) with respect to the canonical pointmaps and the
    confidences."""
    import synth
    w = synth.differentiation(device=dev, H=img_h, W=img_w)
    arm = Arm(M, w, torch.float16, per_edge=False)
    arm.step()
    torch.cuda.synchronize()
    P, plan, wd = arm.P, arm.plan, arm.wd
    T = arm.T0.clone()
    H, g, cost, nv = M.gn_linearize(plan, P, T, wd.X_canon, arm.idx, arm.q)
    a = torch.full((plan.N, 7), 1e-3, dtype=torch.float64, device=dev)
    ws = plan.workspace(M._lib.MSLAM_OP_BACKWARD)
    dX = torch.empty(plan.kf_pixels, 3, dtype=torch.float32, device=dev)
    dq = torch.empty(plan.edge_pixels, dtype=torch.float32, device=dev)
    st = torch.zeros(plan.G, dtype=torch.int32, device=dev)

    def run():
        st.zero_()
        M.gn_backward(plan, P, T, wd.X_canon, arm.idx, arm.q, H, g, dL_dtau=a, dL_dcost=1.0, dL_dX=dX, dL_dq=dq,
                      dev_status=st, workspace=ws)

    ms = _event_ms(run, 10)
    n_matched = int(((arm.idx >= 0) & (arm.q.float() > P.q_min)).sum())
    # per matched pixel: X_i[m], X_j[n] (6 B each), idx (4), q (2) read; the
    # two point gradients (12 B each) and dq (4 B) written
    alg = n_matched * (6 + 6 + 4 + 2 + 12 + 12 + 4)
    gbs = alg / (ms * 1e-3) / 1e9
    hbm = float(peaks["hbm_gbs"])
    return {"workload": f"differentiation: 32 keyframes, 96 directed edges, {img_w}x{img_h}, FP16 storage",
            "ms": ms, "matched_pixels": n_matched, "status": int(st[0]),
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(gbs / hbm, 4), "algorithmic_bytes": int(alg)}}


def main():
    args = parse()
    if args.workload == "batched":
        # tens of GB of device pools: the FP32 plain form, the pinned host
        # copies and the host-side oracle sample are measured on the global graph
        args.no_plain = args.no_e2e = args.no_cpu = True
    world, rank, local = dist_setup(args)
    if args.adjoint_only:
        import paper_2412_12392_gb300 as M
        torch.cuda.set_device(local)
        H, W = (int(v) for v in args.hw.lower().split("x"))
        out = adjoint_measure(M, torch.device("cuda", local), measured_peaks()[0], H, W)
        if rank == 0:
            print(json.dumps(out))
        return
    if args.impl == "reference":
        out = run_reference(args, world, rank)
        if out is not None:
            print(json.dumps(out))
        return
    out, arm, w = run_gpu(args, world, rank, local)
    import paper_2412_12392_gb300 as M
    if not args.no_plain and args.form == "batched":
        plain = Arm(M, w, torch.float32, per_edge=True)
        pms, pstats, _ = time_steps(plain, max(2, args.steps // 3), 1, world)
        pms = max_over_ranks(pms, world)
        n_m = int(((plain.idx >= 0) & (plain.q > plain.P.q_min)).sum())
        out["plain_fp32_per_edge"] = {
            "value": sum_over_ranks(n_m, world) * plain.iters / (pms * 1e-3), "ms_per_step": pms,
            "stage_ms": {k: round(v, 4) for k, v in pstats.items()},
            "speedup_of_batched": pms / out["pipelining"]["serial_ms_per_step"],
            "speedup_of_batched_pipelined": pms / out["ms_per_step"]}
        out["pose_accuracy"], out["storage_error"] = accuracy_report(M, arm, plain, w)
        del plain
    if not args.no_e2e:
        out["e2e"] = e2e_measure(args, M, w, arm.wd.X_canon.dtype, world, rank, local, opts=arm.plan.opts)
    if arm.tuning is not None:
        out["autotune"] = {"opts": arm.tuning["opts"], "match_ms": arm.tuning["match_ms"],
                           "lin_ms": arm.tuning["lin_ms"], "pack_ms": arm.tuning["pack_ms"]}
    if not args.no_extra and args.workload == "global" and not args.small:
        peaks, _ = measured_peaks()
        dev = arm.wd.X_canon.device
        del arm.gn
        torch.cuda.empty_cache()
        out["tracking_frame"] = tracking_frame(M, dev, peaks)
        out["adjoint"] = adjoint_measure(M, dev, peaks)
    if rank == 0 and not args.no_cpu:
        wc = w.to_storage(arm.wd.X_canon.dtype).to("cpu")
        out["cpu_baseline"] = cpu_baseline(wc, args.cpu_seconds, out["matched_pixels"], out["query_pixels"],
                                           w.n_gn_iters, M.params_dict(arm.P))
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
