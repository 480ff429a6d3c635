"""Autotuner for the plan's launch shapes: the linearisation tile size and
form, blocks per SM, the match block shape (pixels per block row) and the
match window form (per-query FP32 or grouped tensor-core scoring) and the
query pixels per match thread.

Each candidate is timed on the caller's device-resident inputs with CUDA
events -- the match block shape on mslam_match, the linearisation tile size
and persistent-grid blocks per SM on mslam_gn_pack + mslam_gn_linearize_packed
-- and the fastest of each stage is kept.  Results are identical for every
shape up to FP32 summation order.
"""
from __future__ import annotations

import itertools
from typing import Dict, Optional, Sequence

import torch

from . import api

MATCH_WIDTHS = (8, 16, 32, 64)
MATCH_PPTS = (1, 2)
LIN_TILES = (4096, 8192, 16384)
LIN_BLOCKS = (0, 2, 3, 4)
WARP_STREAM_TILES = (1024, 2048, 4096)
FORM_NAMES = {0: "stream", 1: "regs", 2: "warp", 3: "regs_ring"}


def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(kf_hw, edges, graph_of_kf, params, X_ref, X_qry, D_ref, D_qry, Q_ref, Q_qry, X_canon, T_wc,
             match_widths: Sequence[int] = MATCH_WIDTHS, lin_tiles: Sequence[int] = LIN_TILES,
             match_ppts: Sequence[int] = MATCH_PPTS,
             lin_blocks: Sequence[int] = LIN_BLOCKS, reps: int = 3, gn_iters: int = 10) -> Dict:
    """Returns {"opts": best plan options, "match_ms": {...}, "lin_ms": {...},
    "pack_ms": {...}}.  A linearisation shape is scored by gn_iters
    linearisations plus one packing (the tile size sets both).  D_ref / D_qry
    are chunk-planar (api.chunk_descriptors)."""
    report = {"match_ms": {}, "lin_ms": {}, "pack_ms": {}}
    best_w, best_t = None, float("inf")
    idx = q = None
    # the tensor-core and staged window forms exist for FP16 storage
    forms = (0, 1, 2) if X_ref.dtype == torch.float16 else (0,)
    for wdt, form, ppt in itertools.product(match_widths, forms, match_ppts):
        plan = api.Plan(kf_hw, edges, graph_of_kf, opts={"match_block_w": wdt, "match_form": form,
                                                        "match_ppt": ppt})
        ws = plan.workspace(api._lib.MSLAM_OP_MATCH)

        def run_match():
            return api.match(plan, params, X_ref, X_qry, D_ref, D_qry, Q_ref, Q_qry, workspace=ws)

        ms = _time(run_match, reps)
        report["match_ms"][f"{wdt}/{form}/{ppt}"] = ms
        if ms < best_t:
            best_w, best_t = (wdt, form, ppt), ms
        del ws
    idx, q = api.match(api.Plan(kf_hw, edges, graph_of_kf), params, X_ref, X_qry, D_ref, D_qry, Q_ref, Q_qry)
    best_lin, best_lt = None, float("inf")
    shapes = [(tile, bps, form) for tile, bps in itertools.product(lin_tiles, lin_blocks)
              for form in ((1, 3) if X_canon.dtype == torch.float16 else (1,))]
    # the block-streamed form runs one CTA per SM and favours large tiles;
    # the warp-streamed form gives each warp whole tiles and favours small ones
    shapes += [(tile, 0, 0) for tile in sorted(set(lin_tiles) | {32768, 65536})]
    shapes += [(tile, 0, 2) for tile in WARP_STREAM_TILES]
    for tile, bps, form in shapes:
        plan = api.Plan(kf_hw, edges, graph_of_kf, opts={"lin_tile": tile, "lin_blocks_per_sm": bps,
                                                        "lin_form": form})
        packed = api.gn_pack(plan, params, X_canon, idx, q)
        ws = plan.workspace(api._lib.MSLAM_OP_LINEARIZE)

        def run_lin():
            api.gn_linearize_packed(plan, params, X_canon.dtype, T_wc, packed, workspace=ws)

        def run_pack():
            api.gn_pack(plan, params, X_canon, idx, q, packed)

        ms = _time(run_lin, reps)
        pms = report["pack_ms"].setdefault(tile, _time(run_pack, reps))
        report["lin_ms"][f"{tile}/{bps}/{FORM_NAMES[form]}"] = ms
        score = gn_iters * ms + pms
        if score < best_lt:
            best_lin, best_lt = (tile, bps, form), score
    report["opts"] = {"match_block_w": best_w[0], "match_form": best_w[1], "match_ppt": best_w[2],
                      "lin_tile": best_lin[0],
                      "lin_blocks_per_sm": best_lin[1], "lin_form": best_lin[2]}
    return report
