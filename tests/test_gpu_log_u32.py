"""The FP32 log u of the tensor-core kernel's MH draws (App. B.1: u = (w + 1/2)
2^-32 from the chain's Philox word).  The first-level MH decision adds
2^-20 (1 + |log u|) to its margin for this value; here the bound is checked
against the FP64 log on the device's special-function unit: every draw below
2^20, the top 2^20 and 2^22 random words.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from _common import ROOT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = str(tmp_path_factory.mktemp("logu") / "liblogu.so")
    cmd = ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler", "-fPIC",
           "--expt-relaxed-constexpr", "-std=c++17",
           "-I", os.path.join(ROOT, "paper_2008_05401_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "csrc", "log_u32_check.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.log_u32_eval.argtypes = [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_float), ctypes.c_int]
    return lib


def test_log_u32_within_the_margin_term(lib):
    g = np.random.default_rng(11)
    w = np.concatenate([np.arange(1 << 20, dtype=np.uint32),
                        (np.uint64(2**32) - 1 - np.arange(1 << 20, dtype=np.uint64)).astype(np.uint32),
                        g.integers(0, 2**32, 1 << 22, dtype=np.uint64).astype(np.uint32)])
    out = np.empty(len(w), dtype=np.float32)
    assert lib.log_u32_eval(w.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), len(w)) == 0
    ref = np.log((w.astype(np.float64) + 0.5) * 2.0 ** -32)
    got = out.astype(np.float64)
    bound = 2.0 ** -20 * (1.0 + np.abs(got))
    ratio = np.abs(got - ref) / bound
    worst = int(np.argmax(ratio))
    assert ratio[worst] <= 1.0, (int(w[worst]), float(got[worst]), float(ref[worst]))
