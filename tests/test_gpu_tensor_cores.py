"""The tensor-core form of the Ising proposal kernel (L = 128: one chain per
CTA; L = 64, 32 and 16: two, four and eight chains per CTA with interleaved
rows; mixed precision).

Its chain is the FP64 path's: lattices and accept counts identical to the
oracle's and to the table kernel's, bit for bit, on the same Philox streams;
the lattice sums (log pi, E, observable sums) are exact integers times
constants and identical too; the free energy read back (in FP64) agrees with
the oracle's to 1e-10.  Cases cover the four sides (chain counts that
leave the last CTA partly empty), K < 4 (unused filter slots), k = 3..5,
g > 1 Gibbs steps (ping-pong lattice operands), uncorrected Gibbs, a batch
mixing the tensor-core form with the table kernel, CUDA-graph replay, and the
analytic CRBM (log r = 0: every MH decision sits within the FP32 bound and is
redone in FP64).
"""
import numpy as np
import pytest

import crbm_workloads as wl
from _common import decisions_are_clear, gpu_ctx, oracle_chains, run_oracle

pytestmark = pytest.mark.gpu

SEED = 2008054010


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


def _run(ctx, mid, L, T, bits0, S, g, correct, tc, prec):
    from paper_2008_05401_gb300 import ISING
    ctx.set_tensor_cores(tc)
    job = ctx.new_job(mid, ISING, L, T, (1.0,), SEED, 0, bits0, prec)
    job.run(S, g=g, correct=correct, precision=prec)
    bits, step = job.state()
    lp, F, E = job.energies()
    sums, acc, rec = job.observables()
    job.release()
    ctx.set_tensor_cores(True)
    return dict(bits=bits, step=step, lp=lp, F=F, E=E, sums=sums, acc=acc, rec=rec)


TC_CASES = [
    # L, K, k, n, g, correct, std
    (128, 4, 5, 8, 1, True, 0.1),       # the batch Ising workload's filter bank
    (128, 4, 4, 4, 1, True, 0.15),      # k = 4
    (128, 2, 3, 6, 2, True, 0.3),       # K < 4, g = 2
    (128, 3, 4, 4, 3, False, 0.25),     # uncorrected, g = 3
    (128, 1, 5, 4, 1, True, 0.4),       # one filter
    (64, 4, 5, 9, 1, True, 0.12),       # two chains per CTA, the last CTA half empty
    (64, 2, 3, 6, 2, True, 0.3),        # g = 2 with two chains per CTA
    (64, 3, 4, 5, 3, False, 0.25),      # uncorrected, g = 3
    (32, 4, 5, 11, 1, True, 0.12),      # four chains per CTA, the last CTA three
    (32, 2, 3, 6, 2, True, 0.3),        # g = 2 with four chains per CTA
    (32, 3, 4, 9, 3, False, 0.25),      # uncorrected, g = 3, one chain in the last CTA
    (32, 1, 5, 4, 1, True, 0.4),        # one filter
    (16, 4, 5, 13, 1, True, 0.12),      # eight chains per CTA, the last CTA five
    (16, 2, 3, 8, 2, True, 0.3),        # g = 2 with eight chains per CTA
    (16, 3, 4, 9, 3, False, 0.25),      # uncorrected, g = 3, one chain in the last CTA
]


@pytest.mark.parametrize("L,K,k,n,g,correct,std", TC_CASES)
def test_tensor_core_form_matches_oracle_and_table_kernel(ctx, L, K, k, n, g, correct, std):
    from paper_2008_05401_gb300 import FP64, ISING, MIXED
    W, hb, vb = wl.gaussian_crbm(K, k, std, seed=1000 + 10 * K + k)
    T = wl.ising_ladder(n, 8)
    bits0 = wl.pack_bits(wl.random_lattices(n, L, seed=K + k + L))
    S = 10
    ref = oracle_chains("ising", W, hb, vb, L, T, (1.0,), SEED, n, bits0)
    worst = run_oracle(ref, S, g=g, correct=correct)
    if not decisions_are_clear(worst):
        pytest.skip(f"oracle reports a decision inside the FP64 margin: {worst}")
    mid = ctx.load_model(ISING, W, vb, hb)
    tc = _run(ctx, mid, L, T, bits0, S, g, correct, True, MIXED)
    tab = _run(ctx, mid, L, T, bits0, S, g, correct, False, MIXED)
    f64 = _run(ctx, mid, L, T, bits0, S, g, correct, True, FP64)
    assert tc["step"] == S
    np.testing.assert_array_equal(tc["bits"], wl.pack_bits(ref.v))
    np.testing.assert_array_equal(tc["acc"], ref.accepts)
    for key in ("bits", "acc", "lp", "E", "sums"):
        np.testing.assert_array_equal(tc[key], tab[key])
        np.testing.assert_array_equal(tc[key], f64[key])
    np.testing.assert_allclose(tc["E"], ref.E_phys, rtol=1e-12)
    # free energies read back in FP64 (|F| ~ 4.5e4 here): the FP64 path's and the oracle's
    np.testing.assert_allclose(tc["F"], ref.F, rtol=1e-10, atol=1e-10)
    np.testing.assert_array_equal(tc["F"], tab["F"])
    np.testing.assert_allclose(f64["F"], ref.F, rtol=1e-10, atol=1e-10)


def test_tensor_core_form_batched_with_table_kernel_jobs(ctx):
    """A batch holding L = 128, 64, 32 and 16 jobs (tensor-core form, side
    streams) and L = 8 jobs (table kernel) gives every job the results it has
    alone."""
    from paper_2008_05401_gb300 import ISING, MIXED
    W, hb, vb = wl.gaussian_crbm(4, 5, 0.1, seed=77)
    mid = ctx.load_model(ISING, W, vb, hb)
    specs = [(128, 6, 1), (64, 5, 2), (128, 3, 3), (32, 7, 4), (16, 5, 5), (8, 6, 6)]

    def make():
        return [ctx.new_job(mid, ISING, Lj, wl.ising_ladder(n, 4), (1.0,), SEED, base * 1000,
                            wl.pack_bits(wl.random_lattices(n, Lj, seed=base)), MIXED)
                for Lj, n, base in specs]

    alone = make()
    for j in alone:
        j.run(6, precision=MIXED)
    batch = make()
    ctx.run_batch(batch, 6, precision=MIXED)
    for a, b in zip(alone, batch):
        np.testing.assert_array_equal(a.state()[0], b.state()[0])
        for x, y in zip(a.energies(), b.energies()):
            np.testing.assert_array_equal(x, y)
        for x, y in zip(a.observables(), b.observables()):
            np.testing.assert_array_equal(x, y)
    for j in alone + batch:
        j.release()


@pytest.mark.parametrize("L", [128, 64, 32, 16])
def test_tensor_core_form_graph_replay_equals_direct_runs(ctx, L):
    from paper_2008_05401_gb300 import ISING, MIXED
    W, hb, vb = wl.gaussian_crbm(4, 5, 0.12, seed=78)
    mid = ctx.load_model(ISING, W, vb, hb)
    T = wl.ising_ladder(4, 4)
    bits0 = wl.pack_bits(wl.random_lattices(4, L, seed=9))
    direct = ctx.new_job(mid, ISING, L, T, (1.0,), SEED, 0, bits0, MIXED)
    for _ in range(3):
        direct.run(4, precision=MIXED)
    replay = ctx.new_job(mid, ISING, L, T, (1.0,), SEED, 0, bits0, MIXED)
    gr = ctx.graph([replay], 4, precision=MIXED)
    for _ in range(3):
        gr.launch()
    replay.sync()
    np.testing.assert_array_equal(direct.state()[0], replay.state()[0])
    for x, y in zip(direct.observables(), replay.observables()):
        np.testing.assert_array_equal(x, y)
    gr.destroy()
    direct.release()
    replay.release()


@pytest.mark.parametrize("L", [128, 64, 32, 16])
def test_tensor_core_form_mh_redo_on_the_analytic_crbm(ctx, L):
    """App. C: log r = 0 exactly, so the FP32 bound straddles it whenever
    |log u| is small and the FP64 redo decides; every proposal is accepted and
    F after the run is the FP64 value wherever a redo happened last."""
    from oracle import ising
    from paper_2008_05401_gb300 import ISING, MIXED
    beta = 1 / 2.269
    W, hb, vb = ising.analytic_crbm(beta, 3)
    mid = ctx.load_model(ISING, W, vb, hb)
    # the FP32 bound shrinks with the lattice (K N units): more draws at small L
    # so that some |log u| fall inside it
    n, S = 16 * (128 // L), 24
    job = ctx.new_job(mid, ISING, L, np.full(n, 1 / beta), (1.0,), SEED, 0, None, MIXED)
    job.run(S, precision=MIXED)
    _, acc, rec = job.observables()
    assert np.all(acc == S)
    assert rec[:, 1].sum() > 0
    job.release()
