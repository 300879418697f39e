"""The paired FP32 FMA and add (__ffma2_rn, __fadd2_rn) the FP32 compositing kernels use in their
subcarrier loops are two IEEE single-precision fused multiply-adds / additions: on random operands
(normal values, mixed magnitudes and signs, signed zeros, subnormals) they agree bit for bit with
two scalar fmaf / additions."""
import ctypes
import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("add", [0, 1])
def test_paired_fma_is_two_fmaf_bit_for_bit(add):
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2511_22793_gb300", "libgsparc_probe.so"))
    lib.gsparc_probe_fma2_check.restype = ctypes.c_int
    lib.gsparc_probe_fma2_check.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 6
    rng = np.random.default_rng(8)
    n = 1 << 20
    ops = []
    for _ in range(3):
        x = rng.normal(size=2 * n) * np.exp(rng.uniform(-30, 30, size=2 * n))
        x[rng.integers(0, 2 * n, 1000)] = 0.0
        x[rng.integers(0, 2 * n, 1000)] = -0.0
        x[rng.integers(0, 2 * n, 1000)] = 1e-40      # subnormal in FP32
        ops.append(torch.tensor(x.astype(np.float32), device="cuda"))
    pair = torch.empty_like(ops[0])
    scal = torch.empty_like(ops[0])
    rc = lib.gsparc_probe_fma2_check(n, add, *[ctypes.c_void_p(t.data_ptr()) for t in ops], ctypes.c_void_p(pair.data_ptr()),
                                     ctypes.c_void_p(scal.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0
    assert torch.equal(pair.view(torch.int32), scal.view(torch.int32))
