"""The solve's FP64 inverse square root (Newton-Raphson from the FP32
hardware estimate) against CUDA's own 1/sqrt in FP64, over the range the
pivots take and beyond (the fallback branch)."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_rsqrt_newton_matches_cuda(tmp_path):
    assert torch.cuda.is_available()
    so = str(tmp_path / "rsqrt_probe.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler", "-fPIC",
                    "-std=c++17", "-o", so, os.path.join(HERE, "kernels", "rsqrt_probe.cu")], check=True)
    lib = C.CDLL(so)
    lib.rsqrt_probe.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
    rng = np.random.default_rng(0)
    x = np.concatenate([10.0 ** rng.uniform(-40, 40, 200000), rng.uniform(0.5, 2.0, 100000),
                        [1.0, 4.0, 1e-30, 1e30, 2.0 ** -60, 3.0e35]])
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    torch.cuda.synchronize()
    assert lib.rsqrt_probe(xd.data_ptr(), yd.data_ptr(), xd.numel()) == 0
    ref = 1.0 / torch.sqrt(xd)
    rel = ((yd - ref).abs() / ref).max().item()
    assert rel <= 4 * 2.0 ** -53, rel
