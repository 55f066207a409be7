"""Bounded device-side waits (failure handling of the GPU pipeline; the paper
has no counterpart).

The tensor-core kernel's warp-specialised pipeline waits on shared-memory
mbarriers.  Every such wait gives up after the context's cycle limit, raises
the CTA's abort flag and the context's error flag, and the CTA drains its MMAs
and ends.  crbm_probe_wait runs that wait routine in one CTA on an mbarrier
that nothing arrives on (the failure is made by leaving a barrier without
arrivals: no fault, trap or endless loop is involved): the wait must give up,
crbm_sync must report CRBM_ETIMEOUT once, and the context must run normal
jobs, bit-exact with the oracle, afterwards.
"""
import numpy as np
import pytest

import crbm_workloads as wl
from _common import gpu_ctx, oracle_chains, run_oracle

pytestmark = pytest.mark.gpu

SEED = 2008054010


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


def test_wait_with_an_arrival_succeeds(ctx):
    from paper_2008_05401_gb300 import ISING, MIXED, binding
    W, hb, vb = wl.gaussian_crbm(2, 3, 0.2)
    mid = ctx.load_model(ISING, W, vb, hb)
    job = ctx.new_job(mid, ISING, 16, np.full(2, 2.3), (1.0,), SEED, 0, None, MIXED)
    binding.crbm_probe_wait(ctx.h, 10_000, 1)
    job.sync()
    job.release()


def test_wait_that_nothing_completes_gives_up_and_the_context_recovers(ctx):
    from paper_2008_05401_gb300 import ISING, MIXED, binding
    W, hb, vb = wl.gaussian_crbm(4, 5, 0.12, seed=4)
    L, n, S = 64, 5, 6
    T = wl.ising_ladder(n, 4)
    bits0 = wl.pack_bits(wl.random_lattices(n, L, seed=12))
    mid = ctx.load_model(ISING, W, vb, hb)
    job = ctx.new_job(mid, ISING, L, T, (1.0,), SEED, 0, bits0, MIXED)
    binding.crbm_probe_wait(ctx.h, 10_000, 0)          # about 5 us of waiting, then the error flag
    with pytest.raises(binding.CrbmError) as e:
        job.sync()
    assert e.value.code == -4                            # CRBM_ETIMEOUT
    job.sync()                                           # reported once, then cleared
    # the context still runs the tensor-core kernel, with the oracle's chains
    job.run(S, precision=MIXED)
    ref = oracle_chains("ising", W, hb, vb, L, T, (1.0,), SEED, n, bits0)
    run_oracle(ref, S)
    bits, step = job.state()
    _, acc, _ = job.observables()
    assert step == S
    np.testing.assert_array_equal(bits, wl.pack_bits(ref.v))
    np.testing.assert_array_equal(acc, ref.accepts)
    job.release()


def test_wait_limit_arguments(ctx):
    from paper_2008_05401_gb300 import binding
    for bad in (999, 2 ** 40 + 1):
        with pytest.raises(binding.CrbmError):
            binding.crbm_set_wait_limit(ctx.h, bad)
        with pytest.raises(binding.CrbmError):
            binding.crbm_probe_wait(ctx.h, bad, 0)
    with pytest.raises(binding.CrbmError):
        binding.crbm_probe_wait(ctx.h, 10_000, 2)
    binding.crbm_set_wait_limit(ctx.h, 2 ** 28)
