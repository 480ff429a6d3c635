"""Storage error of the FP16 precision form: the GPU path on FP16-stored
pointmaps, descriptors and confidences against the FP64 oracle on the
unrounded FP32 inputs (the parity tests compare on the same stored values;
this reports what the FP16 storage itself costs).  Loose sanity bounds; the
printed numbers are the report."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import pose_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available()
    from paper_2412_12392_gb300 import build
    build.build()
    import paper_2412_12392_gb300 as M
    return M


def test_fp16_storage_error_report(M, tiny_wl):
    w = tiny_wl
    P = M.default_params()
    par = M.params_dict(P)
    # GPU path: FP16 storage, batched packed form
    ws = w.to_storage(torch.float16)
    wd = ws.to("cuda")
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy())
    idx_g, q_g = M.match(plan, P, wd.X_ref, wd.X_qry, M.chunk_descriptors(wd.D_ref), M.chunk_descriptors(wd.D_qry),
                         wd.Q_ref, wd.Q_qry)
    gn = M.GaussNewton(plan, P, wd.X_canon, idx_g, q_g, packed=True)
    T_g = gn.run(w.T_init.cuda(), w.n_gn_iters).cpu()
    # oracle on the FP32 inputs
    idx_r, q_r = [], []
    for e in range(w.E):
        out = oracle.match_workload(w, e, diag=False, **par)
        idx_r.append(out[0])
        q_r.append(out[1])
    idx_r, q_r = np.concatenate(idx_r), np.concatenate(q_r)
    st, T_r, hist, done = oracle.gauss_newton(w.N, w.edges.numpy(), w.kf_off.numpy(), w.e_off.numpy(), w.X_canon,
                                              idx_r, q_r, w.T_init.numpy(), w.n_gn_iters, **par)
    assert st == 0
    ig = idx_g.cpu().numpy()
    union = (ig >= 0) | (idx_r >= 0)
    agree = float((ig[union] == idx_r[union]).mean())
    e = pose_errors(T_g, torch.from_numpy(T_r)).max(axis=0)
    e_gt_g = pose_errors(T_g, w.T_gt)[1:].max(axis=0)
    e_gt_r = pose_errors(torch.from_numpy(T_r), w.T_gt)[1:].max(axis=0)
    print(f"FP16 storage vs FP32-input oracle: index agreement {agree:.5f}; poses (rot rad, rel trans, rel scale) "
          f"{e}; error to ground truth: FP16 GPU {e_gt_g}, FP32 oracle {e_gt_r}")
    assert agree >= 0.98
    assert e[0] <= 1e-3
    # the storage error is far below the distance to the ground truth
    assert e[0] <= 0.5 * max(e_gt_r[0], 1e-6) + 1e-4
