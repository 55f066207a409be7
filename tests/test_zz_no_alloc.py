"""crbm_autocorr_noalloc (fixed device scratch, no allocation) against
crbm_autocorr on the same device series, two calls in a row; oversize
requests are rejected before any launch."""
import numpy as np
import pytest

from _common import gpu_ctx

pytestmark = pytest.mark.gpu


def _series(rng, n, cols):
    X = np.empty((n, cols))
    for c in range(cols):
        rho = 0.9 * c / max(cols - 1, 1)
        e = rng.normal(size=n)
        X[0, c] = e[0]
        for t in range(1, n):
            X[t, c] = rho * X[t - 1, c] + e[t]
    return X


def test_noalloc_equals_allocating_entry_twice():
    import torch
    from paper_2008_05401_gb300 import binding
    ctx = gpu_ctx()
    try:
        rng = np.random.default_rng(7)
        for n, cols in ((3000, 40), (1500, 9)):       # the second call reuses the scratch
            x = torch.tensor(_series(rng, n, cols), device="cuda:0")
            ref_tau, ref_w = binding.crbm_autocorr(ctx.h, x.data_ptr(), cols, n)
            tau, w = binding.crbm_autocorr_noalloc(ctx.h, x.data_ptr(), cols, n)
            np.testing.assert_array_equal(w, ref_w)
            np.testing.assert_array_equal(tau, ref_tau)
    finally:
        ctx.close()


def test_noalloc_at_the_largest_size_allocates_nothing():
    """At CRBM_AUTOCORR_NOALLOC_MAX_SERIES series (the window results then fill
    the scratch array's second half up to its end) the results equal
    crbm_autocorr's, and a warm call leaves the device's free memory as it
    was: the entry point allocates nothing."""
    import torch
    from paper_2008_05401_gb300 import binding
    ctx = gpu_ctx()
    try:
        cols, n = 16384, 48
        rng = np.random.default_rng(11)
        x = torch.tensor(np.cumsum(rng.normal(size=(n, cols)), axis=0) * 0.1 + rng.normal(size=(n, cols)),
                         device="cuda:0")
        ref_tau, ref_w = binding.crbm_autocorr(ctx.h, x.data_ptr(), cols, n)
        binding.crbm_autocorr_noalloc(ctx.h, x.data_ptr(), cols, n)        # warm: module and scratch set up
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        tau, w = binding.crbm_autocorr_noalloc(ctx.h, x.data_ptr(), cols, n)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 >= free0, (free0, free1)
        np.testing.assert_array_equal(w, ref_w)
        np.testing.assert_array_equal(tau, ref_tau)
    finally:
        ctx.close()


def test_noalloc_rejects_oversize():
    import torch
    from paper_2008_05401_gb300 import binding
    ctx = gpu_ctx()
    try:
        x = torch.zeros(2, 1, dtype=torch.float64, device="cuda:0")
        with pytest.raises(binding.CrbmError):
            binding.crbm_autocorr_noalloc(ctx.h, x.data_ptr(), 16385, 2)
    finally:
        ctx.close()
