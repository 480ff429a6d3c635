"""mslam_gn_linearize_noalloc, the workspace-free linearisation for callers
that cannot allocate device memory (a real-time tracking loop where
cudaMalloc may stall the frame, or host code whose device memory belongs to
another allocator).  Called through the C ABI, twice in a row, it must give
exactly the blocks of the workspace form (it runs the same kernels in the
same order on the same inputs), and a call after the first must leave the
device's allocations unchanged; a plan needing more than its built-in
scratch is refused with MSLAM_ERR_RANGE.  This file is collected last."""
import ctypes as C

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_noalloc_linearize_matches_workspace_form():
    assert torch.cuda.is_available()
    import synth
    import paper_2412_12392_gb300 as M
    from paper_2412_12392_gb300 import _lib, build
    build.build()
    L = _lib.lib()
    w = synth.tiny()
    wd = w.to("cuda")
    P = M.default_params()
    plan = M.Plan(w.kf_hw.numpy(), w.edges.numpy())
    idx, q = M.match(plan, P, wd.X_ref, wd.X_qry, M.chunk_descriptors(wd.D_ref), M.chunk_descriptors(wd.D_qry),
                     wd.Q_ref, wd.Q_qry)
    T = w.T_init.cuda()
    H0, g0, c0, n0 = M.gn_linearize(plan, P, T, wd.X_canon, idx, q)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        H = torch.full_like(H0, float("nan"))
        g = torch.full_like(g0, float("nan"))
        c = torch.full_like(c0, float("nan"))
        n = torch.full_like(n0, -1)
        torch.cuda.synchronize()
        alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
        st = L.mslam_gn_linearize_noalloc(C.byref(P), plan.handle, _lib.MSLAM_F32, T.data_ptr(),
                                          wd.X_canon.data_ptr(), idx.data_ptr(), q.data_ptr(), H.data_ptr(),
                                          g.data_ptr(), c.data_ptr(), n.data_ptr(), 0, stream)
        assert st == _lib.MSLAM_OK, _lib.last_error()
        torch.cuda.synchronize()
        if call > 0:
            # the first call looked up the array's address; later calls allocate nothing
            assert torch.cuda.memory_allocated() == alloc0
            assert torch.cuda.mem_get_info()[0] == free0
        assert torch.equal(H, H0), call
        assert torch.equal(g, g0), call
        assert torch.equal(c, c0), call
        assert torch.equal(n, n0), call


def test_noalloc_rejects_plans_beyond_its_scratch():
    assert torch.cuda.is_available()
    import paper_2412_12392_gb300 as M
    from paper_2412_12392_gb300 import _lib
    L = _lib.lib()
    # 8 keyframes of 8192 x 8192 with 7 edges: 57,344 tiles, more than the scratch's 26,214
    plan = M.Plan([[8192, 8192]] * 8, [[k, k + 1] for k in range(7)])
    P = M.default_params()
    st = L.mslam_gn_linearize_noalloc(C.byref(P), plan.handle, _lib.MSLAM_F32, None, None, None, None, None,
                                      None, None, None, 0, None)
    assert st == _lib.MSLAM_ERR_RANGE
    assert "scratch" in _lib.last_error()
