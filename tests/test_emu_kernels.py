"""CPU check of plain CUDA kernels' logic: the kernel's own source, compiled for the host under a
test-only shim (tests/emu/cuda_emu.h: one thread per CUDA thread, real barriers and warp
exchanges), run with the launch shape of its entry point and compared with the FP64 oracle.
This checks index arithmetic, warp sums and summation order before the GPU parity tests; it
is not a parity claim for the GPU (those are the `-m gpu` tests)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from extras_cases import conf_case, conf_oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2511_22793_gb300", "csrc")
EMU = os.path.join(ROOT, "tests", "emu")


@pytest.fixture(scope="module")
def emu_bin(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    out = tmp_path_factory.mktemp("emu")

    def build(name):
        exe = out / name
        if not exe.exists():
            subprocess.run([gxx, "-std=c++20", "-O1", "-pthread", "-I", CSRC, "-I", EMU,
                            os.path.join(EMU, name + ".cpp"), "-o", str(exe)], check=True)
        return str(exe)

    return build


def _run(exe, tmp_path, payload: bytes, timeout=120):
    src, dst = tmp_path / "in.bin", tmp_path / "out.bin"
    src.write_bytes(payload)
    subprocess.run([exe, str(src), str(dst)], check=True, timeout=timeout)
    return dst.read_bytes()


@pytest.mark.parametrize("B,hidden", [(1, 32), (4, 32), (37, 32), (300, 8), (9, 1)])
def test_confidence_kernel_logic(emu_bin, tmp_path, B, hidden):
    exe = emu_bin("confidence_emu")
    pos, L, w = conf_case(B, hidden, 100 + B + hidden)
    dw0 = np.linspace(-1, 1, 5 * hidden + 1).astype(np.float32)     # the kernel accumulates into it
    payload = np.array([B, hidden], np.int32).tobytes() + np.array([0.3], np.float32).tobytes() + \
        pos.tobytes() + L.tobytes() + w.tobytes() + dw0.tobytes()
    raw = _run(exe, tmp_path, payload)
    nw = 5 * hidden + 1
    out = np.frombuffer(raw[:-4], dtype=np.float32)
    violations = int(np.frombuffer(raw[-4:], dtype=np.int32)[0])
    assert violations == 0
    obj, C, dL, dw = out[0], out[1:1 + B], out[1 + B:1 + 2 * B], out[1 + 2 * B:1 + 2 * B + nw]
    o_obj, o_C, o_dL, o_dw, kink = conf_oracle(pos, L, w, hidden)
    assert kink > 1e-5            # no ReLU decision within FP32 rounding of the kink
    assert abs(obj - o_obj) <= 1e-5 * abs(o_obj)
    assert np.allclose(C, o_C, rtol=2e-6, atol=0)
    assert np.allclose(dL, o_dL, rtol=2e-6, atol=0)
    g = dw.astype(np.float64) - dw0
    assert np.linalg.norm(g - o_dw) <= 1e-5 * np.linalg.norm(o_dw)
