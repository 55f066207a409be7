"""The FP32 error bounds behind the mixed path's certified margins.

The library assumes (host constants of crbm_load_model): ex2.approx relative
error <= 2^-22 on the arguments it receives, rcp.approx relative error <=
2^-23, lg2.approx absolute error <= 2^-22 on [1, 2].  Each is checked here on
EVERY float of its range against FP64, so the assumption is a measured fact
of the device the tests run on.  So is the precision of the mixed path's
conditionals: the FP32 sigmoid those units compose is within 1e-6 relative of
the FP64 one wherever sigma >= 1.1e-7, and within 1.1e-6 down to 2^-32.
"""
import ctypes
import os
import struct
import subprocess

import pytest

from _common import ROOT

pytestmark = pytest.mark.gpu


def _bits(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = str(tmp_path_factory.mktemp("sfu") / "libsfu.so")
    cmd = ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "paper_2008_05401_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "csrc", "sfu_bounds.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.sfu_max_error.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double)]
    return lib


def _max_err(lib, which, b0, b1):
    r = ctypes.c_double()
    assert lib.sfu_max_error(which, b0, b1, ctypes.byref(r)) == 0
    return r.value


def test_ex2_relative_error(lib):
    # arguments -|x| log2 e (softplus) and -x log2 e (sigmoid) with normal results:
    # every float in [-125.9, 127.9]
    worst = max(_max_err(lib, 0, _bits(0.0), _bits(127.9)),              # +0 .. 127.9
                _max_err(lib, 0, _bits(-0.0), _bits(-125.9)))            # -0 .. -125.9
    assert worst <= 2.0 ** -22, worst


def test_rcp_relative_error(lib):
    # relative error is scale-free: every mantissa, [1, 2) and [2, 4)
    worst = max(_max_err(lib, 1, _bits(1.0), _bits(2.0)), _max_err(lib, 1, _bits(2.0), _bits(4.0)))
    assert worst <= 2.0 ** -23, worst


def test_lg2_absolute_error_on_1_2(lib):
    worst = _max_err(lib, 2, _bits(1.0), _bits(2.0) + 1)
    assert worst <= 2.0 ** -22, worst


def test_fp32_conditional_relative_error(lib):
    # every float of [-16, 40] (sigma >= 1.1e-7; above 40 both sides give 1):
    # within 1e-6 relative.  Down to sigma = 2^-32 (x = -22.18; a uniform
    # (w + 1/2) 2^-32 never falls below it) the FP32 product x log2(e) adds up
    # to |x| 2^-24 ln 2 relative: within 1.1e-6.  (Decisions are certified on
    # the absolute error and take the FP64 path's result either way.)
    assert _max_err(lib, 3, _bits(0.0), _bits(40.0)) <= 1e-6
    assert _max_err(lib, 3, _bits(-0.0), _bits(-16.0)) <= 1e-6
    assert _max_err(lib, 3, _bits(-0.0), _bits(-22.18)) <= 1.1e-6
