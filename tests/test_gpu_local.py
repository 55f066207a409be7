"""Parity of the CUDA local-update Metropolis sweeps (crbm_local_run), the
E_phys trace (crbm_set_trace) and the autocorrelation time (crbm_autocorr)
with the oracle (the paper's baselines, Sec. III and IV).

Lattices, flip counts and step counters must match bit for bit unless the
oracle reports a decision within 1e-12 (Ising: |u - p|) or 1e-10 (Kitaev and
exchanges: relative |log u - log r|) of its threshold; FP64 values to 1e-9
relative.
"""
import numpy as np
import pytest

import crbm_workloads as wl
from _common import gpu_ctx, oracle_chains

pytestmark = pytest.mark.gpu

SEED = 2008054010


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


def _run_oracle(ch, sweeps, exchange, trace=None):
    from oracle import metropolis
    worst = {"ising": np.inf, "rel": np.inf}

    def rec(c, d):
        key = "ising" if c.model == 0 else "rel"
        worst[key] = min(worst[key], float(np.min(d["margin"])))
        worst["rel"] = min(worst["rel"], float(np.min(d["temp_margin"])))
        if trace is not None:
            trace.append(c.E_phys.copy())

    metropolis.run(ch, sweeps, exchange, record=rec)
    return worst


def _clear(worst):
    return worst["ising"] > 1e-12 and worst["rel"] > 1e-10


def _compare(job, ref, worst):
    if not _clear(worst):
        pytest.skip(f"oracle reports a decision inside the FP64 margin: {worst}")
    bits, step = job.state()
    assert step == ref.step
    np.testing.assert_array_equal(bits, wl.pack_bits(ref.v))
    sums, acc, _ = job.observables()
    np.testing.assert_array_equal(acc, ref.accepts)
    np.testing.assert_allclose(sums, ref.obs, rtol=1e-9, atol=1e-9)
    lp, F, E = job.energies()
    np.testing.assert_allclose(lp, ref.logpi, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(E, ref.E_phys, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(F, ref.F, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("L,n,sweeps,exchange", [(2, 6, 4, False), (4, 12, 6, True), (8, 9, 5, True),
                                                 (16, 8, 4, False), (64, 3, 3, True), (32, 33, 3, False)])
def test_ising_local_matches_oracle(ctx, L, n, sweeps, exchange):
    from paper_2008_05401_gb300 import FP64, ISING
    W, hb, vb = wl.gaussian_crbm(2, min(3, L), 0.2, seed=L)
    T = wl.ising_ladder(n, n, 1.8, 3.2)
    bits0 = wl.pack_bits(wl.random_lattices(n, L, seed=L + 4))
    ref = oracle_chains("ising", W, hb, vb, L, T, (1.0,), SEED, n, bits0)
    worst = _run_oracle(ref, sweeps, exchange)
    mid = ctx.load_model(ISING, W, vb, hb)
    job = ctx.new_job(mid, ISING, L, T, (1.0,), SEED, 0, bits0, FP64)
    job.local_run(sweeps, exchange=exchange)
    _compare(job, ref, worst)
    job.release()


@pytest.mark.parametrize("L,n,sweeps,exchange,J", [(2, 6, 3, False, (1.0, 1.0, 1.0)),
                                                   (3, 5, 2, True, (0.8, 1.1, 1.3)),
                                                   (4, 4, 2, False, (1.0, 1.0, 1.0)),
                                                   (4, 6, 2, True, (1.0, 1.0, 1.0))])
@pytest.mark.parametrize("prec_name", ["FP64", "MIXED"])
def test_kitaev_local_matches_oracle(ctx, L, n, sweeps, exchange, J, prec_name):
    import paper_2008_05401_gb300 as P
    prec = getattr(P, prec_name)
    W, hb, vb = wl.gaussian_crbm(2, 2, 0.1, seed=L)
    T = wl.kitaev_ladder(n, n, 0.05, 1.0)
    bits0 = wl.pack_bits(wl.random_lattices(n, L, seed=L + 9))
    ref = oracle_chains("kitaev", W, hb, vb, L, T, J, SEED, n, bits0)
    worst = _run_oracle(ref, sweeps, exchange)
    mid = ctx.load_model(P.KITAEV, W, vb, hb)
    job = ctx.new_job(mid, P.KITAEV, L, T, J, SEED, 0, bits0, prec)
    job.local_run(sweeps, exchange=exchange, precision=prec)
    _compare(job, ref, worst)
    job.release()


def test_trace_and_autocorr_match_oracle(ctx):
    """The E trace of CRBM proposals then local sweeps equals the oracle's,
    and crbm_autocorr on it equals the oracle's tau and window."""
    from oracle import autocorr, chain
    from paper_2008_05401_gb300 import FP64, ISING
    L, n = 8, 16
    W, hb, vb = wl.gaussian_crbm(2, 3, 0.1, seed=3)
    T = np.full(n, 2.5)
    bits0 = wl.pack_bits(wl.random_lattices(n, L, seed=2))
    ref = oracle_chains("ising", W, hb, vb, L, T, (1.0,), SEED, n, bits0)
    tr = []
    chain.run(ref, 20, record=lambda c, d: tr.append(c.E_phys.copy()))
    worst = _run_oracle(ref, 60, False, trace=tr)
    mid = ctx.load_model(ISING, W, vb, hb)
    job = ctx.new_job(mid, ISING, L, T, (1.0,), SEED, 0, bits0, FP64)
    buf = job.set_trace(100)
    job.run(20)
    job.local_run(60)
    job.sync()
    if not _clear(worst):
        pytest.skip("decision inside the FP64 margin")
    got = buf.cpu().numpy()
    np.testing.assert_array_equal(got[:80], np.array(tr))
    assert np.isnan(got[80:]).all()
    tau, win = ctx.autocorr(buf[:80])
    t_ref, w_ref = autocorr.tau_int_columns(np.array(tr))
    np.testing.assert_array_equal(win, w_ref)
    np.testing.assert_allclose(tau, t_ref, rtol=1e-9)
    job.release()


def test_autocorr_of_host_series(ctx):
    """AR(1) series with known tau, a constant and an alternating series."""
    import torch
    from oracle import autocorr
    rng = np.random.default_rng(1)
    n, cols = 4000, 5
    X = np.empty((n, cols))
    for c, rho in enumerate((0.0, 0.5, 0.9)):
        e = rng.normal(size=n)
        X[0, c] = e[0]
        for t in range(1, n):
            X[t, c] = rho * X[t - 1, c] + e[t]
    X[:, 3] = 2.0
    X[:, 4] = np.tile([1.0, -1.0], n // 2)
    tau, win = ctx.autocorr(torch.tensor(X, device="cuda:0"))
    t_ref, w_ref = autocorr.tau_int_columns(X)
    np.testing.assert_array_equal(win, w_ref)
    np.testing.assert_allclose(tau, t_ref, rtol=1e-9)
    assert tau[3] == 0.5 and win[3] == 0


def test_local_rejects_odd_ising_lattice(ctx):
    from paper_2008_05401_gb300 import ISING, CrbmError
    W, hb, vb = wl.gaussian_crbm(2, 3, 0.1)
    mid = ctx.load_model(ISING, W, vb, hb)
    job = ctx.new_job(mid, ISING, 5, np.full(2, 2.0), (1.0,), 1)
    with pytest.raises(CrbmError):
        job.local_run(1)
    job.release()
