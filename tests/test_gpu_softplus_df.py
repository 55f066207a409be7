"""The double-FP32 softplus behind the mixed path's second-level MH decision.

The library bounds its error per unit by 1e-12 + 2^-44 softplus(x) (the
constant in free_sum_df); here it is measured against a long-double reference
on a dense grid over the argument range the free energy meets and on random
df64 arguments (hi + lo pairs with a non-zero low word).
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
    out = str(tmp_path_factory.mktemp("spdf") / "libspdf.so")
    cmd = ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler", "-fPIC",
           "--expt-relaxed-constexpr", "-std=c++17",
           "-I", os.path.join(ROOT, "paper_2008_05401_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "csrc", "softplus_df_check.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    fp = ctypes.POINTER(ctypes.c_float)
    lib.softplus_df_eval.argtypes = [fp, fp, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    return lib


def _eval(lib, hi, lo):
    hi = np.ascontiguousarray(hi, dtype=np.float32)
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    out = np.empty(len(hi), dtype=np.float64)
    fp = ctypes.POINTER(ctypes.c_float)
    assert lib.softplus_df_eval(hi.ctypes.data_as(fp), lo.ctypes.data_as(fp),
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(hi)) == 0
    return out


def _reference(hi, lo):
    x = hi.astype(np.longdouble) + lo.astype(np.longdouble)
    return np.maximum(x, 0) + np.log1p(np.exp(-np.abs(x)))


def _check(lib, hi, lo):
    got = _eval(lib, hi, lo).astype(np.longdouble)
    ref = _reference(hi, lo)
    excess = np.abs(got - ref) - (1e-12 + 2.0 ** -44 * ref)
    worst = int(np.argmax(excess))
    assert excess[worst] <= 0, (float(hi[worst]), float(lo[worst]), float(got[worst]), float(ref[worst]))
    return float(np.max(np.abs(got - ref)))


def test_softplus_df_on_a_dense_grid(lib):
    x = np.linspace(-60.0, 60.0, 2_000_001)
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    assert _check(lib, hi, lo) < 4e-12


def test_softplus_df_random_df64_arguments(lib):
    g = np.random.default_rng(7)
    x = np.concatenate([g.normal(0, 3, 500_000), g.uniform(-45, 45, 500_000), g.normal(0, 1e-3, 100_000)])
    hi = x.astype(np.float32)
    lo = (g.uniform(-0.5, 0.5, len(x)) * np.spacing(np.abs(hi).astype(np.float32))).astype(np.float32)
    _check(lib, hi, lo)


def test_softplus_df_near_the_branch_and_table_edges(lib):
    # a = 40 (switch to the ex2 tail), m/64 boundaries, multiples of ln 2, 0
    pts = [40.0, 40.0001, 39.9999, 0.0, -0.0, 1e-30, -1e-30]
    pts += [m / 64 + d for m in range(0, 46) for d in (-1e-7, 0.0, 1e-7)]
    pts += [n * np.log(2) + d for n in range(0, 59) for d in (-1e-6, 0.0, 1e-6)]
    x = np.array(pts + [-p for p in pts])
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    _check(lib, hi, lo)
