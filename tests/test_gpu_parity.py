"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every case runs the same chains, from the same packed lattices and Philox
streams, on both sides.  Lattices and accept counts must match bit for bit
unless the oracle reports a Bernoulli draw within 1e-12 of its threshold or an
MH decision within 1e-10 (relative) -- FP64 on the two sides uses different
exp/log implementations and summation orders, so only such draws may differ.
Floating results (log pi, F, observable sums) must agree to 1e-9 relative:
FP64 rounding over <= 2^16 terms of size O(1), well inside that.
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


def _compare(job, ref, worst, S, exact_floats=True):
    bits, step = job.state()
    lp, F, E = job.energies()
    sums, acc, rec = job.observables()
    assert step == S
    if not decisions_are_clear(worst):
        pytest.skip(f"oracle reports a decision inside the FP64 margin: {worst}")
    np.testing.assert_array_equal(bits, wl.pack_bits(ref.v))
    np.testing.assert_array_equal(acc, ref.accepts)
    np.testing.assert_allclose(lp, ref.logpi, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(E, ref.E_phys, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(sums, ref.obs, rtol=1e-9, atol=1e-9)
    if exact_floats:
        np.testing.assert_allclose(F, ref.F, rtol=1e-10, atol=1e-10)
    return bits, acc, rec, F


ISING_CASES = [
    # L, K, k, n, g, correct, std
    (4, 2, 3, 40, 1, True, 0.6),
    (6, 1, 2, 24, 1, True, 0.5),      # L % 4 != 0: ragged units across rows, N % 32 != 0
    (8, 2, 3, 16, 1, True, 0.1),      # the small Ising workload
    (8, 4, 5, 33, 2, True, 0.3),      # g = 2, ragged chain tail
    (12, 3, 4, 10, 1, False, 0.4),    # uncorrected Gibbs
    (16, 4, 5, 20, 1, True, 0.2),
    (24, 2, 7, 5, 1, True, 0.2),      # widest kernel
    (32, 4, 5, 6, 1, True, 0.15),
    (64, 4, 5, 3, 1, True, 0.1),      # several tiles of 4-site units, multi-word rows
    (96, 2, 3, 2, 1, True, 0.1),      # row of 3 words
    (256, 8, 6, 2, 1, True, 0.05),    # the largest lattice, K = 8 filters, K k 2^k = 3072 table entries
    (20, 4, 7, 3, 3, True, 0.1),      # k = 7 (largest kernel), g = 3
]


@pytest.mark.parametrize("L,K,k,n,g,correct,std", ISING_CASES)
def test_ising_matches_oracle(ctx, L, K, k, n, g, correct, std):
    from paper_2008_05401_gb300 import FP64, ISING, MIXED
    W, hb, vb = wl.gaussian_crbm(K, k, std, seed=L * 100 + K)
    T = wl.ising_ladder(n, 8)
    bits0 = wl.pack_bits(wl.random_lattices(n, L, seed=L))
    S = 12
    ref = oracle_chains("ising", W, hb, vb, L, T, (1.0,), SEED, n, bits0)
    worst = run_oracle(ref, S, g=g, correct=correct)
    mid = ctx.load_model(ISING, W, vb, hb)
    job = ctx.new_job(mid, ISING, L, T, (1.0,), SEED, 0, bits0, FP64)
    job.run(S, g=g, correct=correct, precision=FP64)
    bits64, acc64, rec64, F64 = _compare(job, ref, worst, S)
    assert rec64.sum() == 0
    # the mixed path takes exactly the FP64 path's decisions
    jm = ctx.new_job(mid, ISING, L, T, (1.0,), SEED, 0, bits0, MIXED)
    jm.run(S, g=g, correct=correct, precision=MIXED)
    bm, _ = jm.state()
    np.testing.assert_array_equal(bm, bits64)
    _, accm, recm = jm.observables()
    np.testing.assert_array_equal(accm, acc64)
    # read back in FP64 (crbm_read_energies re-evaluates a mixed job's lattices)
    lpm, Fm, Em = jm.energies()
    np.testing.assert_allclose(Fm, ref.F, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(lpm, ref.logpi, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(Em, ref.E_phys, rtol=1e-10, atol=1e-10)
    job.release()
    jm.release()


KITAEV_CASES = [
    # L, K, k, n, correct
    (2, 2, 2, 6, True),
    (3, 4, 3, 8, True),    # odd L: N = 9, ragged units
    (4, 4, 3, 8, True),
    (6, 4, 3, 12, True),   # the small Kitaev workload geometry
    (5, 2, 3, 4, False),
    (8, 2, 5, 4, True),
    (12, 4, 3, 2, True),   # N = 144: largest matrix
]


@pytest.mark.parametrize("L,K,k,n,correct", KITAEV_CASES)
def test_kitaev_matches_oracle(ctx, L, K, k, n, correct):
    from paper_2008_05401_gb300 import FP64, KITAEV, MIXED
    W, hb, vb = wl.gaussian_crbm(K, k, 0.05, seed=L + 17)
    T = wl.kitaev_ladder(n, 24)
    J = (1.0, 1.0, 1.0) if L % 2 == 0 else (0.8, 1.1, 1.3)
    bits0 = wl.pack_bits(wl.random_lattices(n, L, seed=L + 3))
    S = 4
    ref = oracle_chains("kitaev", W, hb, vb, L, T, J, SEED, n, bits0)
    worst = run_oracle(ref, S, correct=correct)
    mid = ctx.load_model(KITAEV, W, vb, hb)
    job = ctx.new_job(mid, KITAEV, L, T, J, SEED, 0, bits0, FP64)
    job.run(S, correct=correct, precision=FP64)
    bits64, acc64, _, F64 = _compare(job, ref, worst, S)
    jm = ctx.new_job(mid, KITAEV, L, T, J, SEED, 0, bits0, MIXED)
    jm.run(S, correct=correct, precision=MIXED)
    bm, _ = jm.state()
    np.testing.assert_array_equal(bm, bits64)
    lpm, Fm, _ = jm.energies()
    np.testing.assert_allclose(Fm, ref.F, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(lpm, ref.logpi, rtol=1e-10, atol=1e-9)
    job.release()
    jm.release()


@pytest.mark.parametrize("J", [(0.0, 0.0, 1.0), (0.7, 0.0, 1.2), (0.0, 0.9, 1.1)])
@pytest.mark.parametrize("L", [4, 6])
def test_kitaev_degenerate_couplings_match_oracle(ctx, L, J):
    """Vanishing couplings: with J_x = J_y = 0 the matrix M^T M is diagonal,
    so every column of the Householder reduction is already reduced (the
    step without a reflection) and the spectrum is N-fold degenerate; with
    one of them zero the lattice falls apart into chains (repeated
    eigenvalues, columns that vanish part-way through the reduction).  Both
    precisions against the oracle's singular values."""
    from paper_2008_05401_gb300 import FP64, KITAEV, MIXED
    W, hb, vb = wl.gaussian_crbm(4, 3, 0.05, seed=L + 29)
    n, S = 24, 3
    T = wl.kitaev_ladder(n, 24)
    bits0 = wl.pack_bits(wl.random_lattices(n, L, seed=L + 11))
    ref = oracle_chains("kitaev", W, hb, vb, L, T, J, SEED, n, bits0)
    worst = run_oracle(ref, S)
    mid = ctx.load_model(KITAEV, W, vb, hb)
    for prec in (FP64, MIXED):
        job = ctx.new_job(mid, KITAEV, L, T, J, SEED, 0, bits0, prec)
        job.run(S, precision=prec)
        _compare(job, ref, worst, S)
        job.release()


def test_random_init_matches_oracle(ctx):
    """init = 0 draws the lattices from the stream's init tag on the device."""
    from oracle import chain
    from paper_2008_05401_gb300 import FP64, ISING
    W, hb, vb = wl.gaussian_crbm(2, 3, 0.1)
    mid = ctx.load_model(ISING, W, vb, hb)
    for L, n, base in ((8, 5, 0), (6, 3, 1000), (64, 2, 2 ** 32 - 2)):
        job = ctx.new_job(mid, ISING, L, np.full(n, 2.0), (1.0,), 99, base, None, FP64)
        bits, _ = job.state()
        np.testing.assert_array_equal(bits, wl.pack_bits(chain.random_init(99, np.arange(base, base + n), L)))
        job.release()


def test_analytic_crbm_accepts_everything(ctx):
    """App. C: the analytic CRBM equals the Ising distribution, so every
    proposal is accepted, at any lattice size (here L = 128)."""
    from oracle import ising
    from paper_2008_05401_gb300 import FP64, ISING, MIXED
    beta = 1 / 2.269
    W, hb, vb = ising.analytic_crbm(beta, 3)
    mid = ctx.load_model(ISING, W, vb, hb)
    for prec in (FP64, MIXED):
        job = ctx.new_job(mid, ISING, 128, np.full(4, 1 / beta), (1.0,), SEED, 0, None, prec)
        job.run(10, precision=prec)
        _, acc, _ = job.observables()
        assert np.all(acc == 10)
        job.release()


@pytest.mark.parametrize("L,n,S", [(6, 24, 4), (10, 24, 4), (12, 24, 4), (6, 1024, 3), (12, 682, 2)])
def test_kitaev_mixed_df64_stage_matches_fp64(ctx, L, n, S):
    """The mixed path's df64 eigen-stage: lattices and acceptances identical to
    the FP64 path over the whole temperature ladder (down to T = 0.005), also
    at the Kitaev workloads' chain counts, and log-weights (read back in FP64)
    within 1e-10."""
    from paper_2008_05401_gb300 import FP64, KITAEV, MIXED
    W, hb, vb = wl.gaussian_crbm(4, 3, 0.05, seed=L + 99)
    T = wl.kitaev_ladder(n, 24)
    bits0 = wl.pack_bits(wl.random_lattices(n, L, seed=L + 5))
    mid = ctx.load_model(KITAEV, W, vb, hb)
    a = ctx.new_job(mid, KITAEV, L, T, (1.0, 1.0, 1.0), SEED, 0, bits0, FP64)
    b = ctx.new_job(mid, KITAEV, L, T, (1.0, 1.0, 1.0), SEED, 0, bits0, MIXED)
    a.run(S, precision=FP64)
    b.run(S, precision=MIXED)
    np.testing.assert_array_equal(a.state()[0], b.state()[0])
    _, acc_a, _ = a.observables()
    _, acc_b, rec_b = b.observables()
    np.testing.assert_array_equal(acc_a, acc_b)
    lp_a, _, E_a = a.energies()
    lp_b, _, E_b = b.energies()
    np.testing.assert_allclose(lp_b, lp_a, rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(E_b, E_a, rtol=1e-9, atol=1e-9)
    assert rec_b[:, 1].sum() <= n * S // 2          # MH recomputes stay the exception
    a.release()
    b.release()
