"""The constants the paper states (tests/golden/paper_constants.txt, each
with its passage) against the library's and the oracle's defaults, the
workload generator and the keyframe criterion (CPU only)."""
import os

import numpy as np
import torch

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_constants.txt")


def _constants():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                name, value, _ = line.split(" ", 2)
                out[name] = float(value)
    return out


def test_iteration_counts_follow_the_paper():
    c = _constants()
    import paper_2412_12392_gb300 as M
    assert M.default_params().lm_iters == c["lm_iters"] == oracle.DEFAULT_PARAMS["lm_iters"]
    g = synth.global_graph(N=4, n_pairs=3, H=24, W=32)
    assert g.n_match_iters == c["lm_iters"] and 1 <= g.n_gn_iters <= c["gn_iters_max"]


def test_keyframe_criterion():
    c = _constants()
    import paper_2412_12392_gb300 as M
    assert M.api.OMEGA_K == c["omega_k"]
    n_query = 1000
    # valid fraction, unique fraction -> keyframe needed
    cases = [(0.9, 0.9, False), (0.2, 0.9, True), (0.9, 0.2, True), (0.333, 0.333, False), (0.332, 0.5, True)]
    nv = torch.tensor([round(a * n_query) for a, _, _ in cases])
    nu = torch.tensor([round(b * n_query) for _, b, _ in cases])
    got = M.keyframe_needed(nv, nu, n_query).tolist()
    assert got == [want for _, _, want in cases]
    assert bool(M.keyframe_needed(np.array([0]), np.array([0]), 0)[0])  # an empty frame always needs a keyframe
