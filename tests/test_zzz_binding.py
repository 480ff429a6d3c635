"""The binding refuses buffers the C ABI cannot check: a host tensor, a
tensor of the wrong dtype or size handed over as a device pointer (an output,
a gradient, a status array or a workspace) raises ValueError before any
launch, so that no kernel is ever given a host address or a short buffer."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2412_12392_gb300 import build
    build.build()
    import paper_2412_12392_gb300 as M
    return M


def test_binding_rejects_unusable_buffers(M):
    from paper_2412_12392_gb300 import _lib, api
    H, W = 8, 16
    n = H * W
    plan = M.Plan([[H, W], [H, W]], [[0, 1]])
    P = M.default_params()
    dev = "cuda"
    T = torch.zeros(2, 8, dtype=torch.float64, device=dev)
    X = torch.ones(2 * n, 3, device=dev)
    idx = torch.full((n,), -1, dtype=torch.int32, device=dev)
    q = torch.zeros(n, device=dev)
    Hb = torch.zeros(1, 14, 14, device=dev)
    gb = torch.zeros(1, 14, device=dev)
    lin_bytes = plan.workspace_bytes(_lib.MSLAM_OP_LINEARIZE)
    host_ws = torch.empty(max(lin_bytes, 256), dtype=torch.uint8)
    f32_ws = torch.empty(max(lin_bytes, 256) // 4 + 1, dtype=torch.float32, device=dev)
    cases = {
        "host linearize workspace": lambda: M.gn_linearize(plan, P, T, X, idx, q, workspace=host_ws),
        "FP32 linearize workspace": lambda: M.gn_linearize(plan, P, T, X, idx, q, workspace=f32_ws),
        "host solve workspace": lambda: M.gn_solve(plan, P, Hb, gb, T.clone(), workspace=host_ws),
        "host match workspace": lambda: M.match(plan, P, X[:n], X[:n], M.chunk_descriptors(X.new_zeros(n, 16)),
                                                M.chunk_descriptors(X.new_zeros(n, 16)), q, q,
                                                workspace=host_ws),
        "host ray-image output": lambda: M.ray_image(X, out=torch.empty(2 * n, 3)),
        "FP64 ray-image input": lambda: M.ray_image(X.double()),
        "short packed outputs": lambda: M.gn_linearize_packed(plan, P, torch.float16, T,
                                                              torch.zeros(256, dtype=torch.uint8, device=dev),
                                                              H=torch.zeros(13, 14, device=dev)),
        "host gradient": lambda: M.gn_backward(plan, P, T, X, idx, q, dL_dX=torch.empty(2 * n, 3)),
        "FP32 pose gradient": lambda: api.gn_step_backward(plan, P, T, X, idx, q, Hb, gb,
                                                           dL_dT=torch.empty(2, 8, device=dev)),
        "host tracking status": lambda: M.gn_track(plan, P, torch.float16, T,
                                                   torch.zeros(256, dtype=torch.uint8, device=dev), 1,
                                                   dev_status=torch.zeros(1, dtype=torch.int32)),
    }
    for name, call in cases.items():
        with pytest.raises(ValueError):
            call()
            pytest.fail(f"{name}: accepted")
    # the same calls with usable buffers go through
    R = M.ray_image(X, out=torch.empty_like(X))
    torch.cuda.synchronize()
    assert torch.allclose(R, X / 3 ** 0.5)
