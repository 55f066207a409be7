"""Statistical and full-size checks of the CUDA path against exact results.

* stationarity: chains started from an exact draw of the target distribution
  (enumerated on a tiny lattice) keep it after several proposals (chi^2 over
  independent chains) -- the MH correction of Eq. (B5) is exact;
* Kaufman's closed-form <E> of the 8 x 8 torus at T = 2.269 (the small Ising
  workload) within 4 sigma, with the analytic CRBM of App. C;
* full-size parity: the 4096-chain L = 128 launch of the batch workload,
  sampled chains replayed by the oracle.
"""
import numpy as np
import pytest

import crbm_workloads as wl
from _common import decisions_are_clear, gpu_ctx, oracle_chains, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


def _chi2_ok(idx, probs, C):
    cnt = np.bincount(idx, minlength=len(probs)).astype(float)
    m = probs * C > 5
    obs = np.append(cnt[m], cnt[~m].sum())
    exp = np.append(probs[m] * C, probs[~m].sum() * C)
    keep = exp > 0
    chi2 = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    df = keep.sum() - 1
    return chi2, df, chi2 < df + 6 * np.sqrt(2 * df)


@pytest.mark.parametrize("prec", [0, 1])
def test_ising_chains_keep_the_boltzmann_distribution(ctx, prec):
    from oracle import ising
    from paper_2008_05401_gb300 import ISING
    L, beta, C = 4, 0.35, 16384
    W, hb, vb = ising.analytic_crbm(beta, 3)
    g = np.random.default_rng(3)
    W = W + g.normal(0, 0.4, W.shape)
    hb = hb + g.normal(0, 0.4, 2)
    vb = vb + 0.3
    vs = ising.all_states(L)
    E = ising.energy(vs)
    p = np.exp(-beta * E - (-beta * E).max())
    p /= p.sum()
    v0 = vs[np.random.default_rng(12).choice(len(vs), size=C, p=p)]
    mid = ctx.load_model(ISING, W, vb, hb)
    job = ctx.new_job(mid, ISING, L, np.full(C, 1 / beta), (1.0,), 99, 0, wl.pack_bits(v0), prec)
    job.run(10, precision=prec)
    bits, _ = job.state()
    _, acc, _ = job.observables()
    assert 0.1 < acc.mean() / 10 < 0.95
    levels, inv = np.unique(E, return_inverse=True)
    pe = np.bincount(inv, weights=p)
    idx = np.searchsorted(levels, ising.energy(wl.unpack_bits(bits, L)))
    chi2, df, ok = _chi2_ok(idx, pe, C)
    assert ok, (chi2, df)
    job.release()


def test_kitaev_chains_keep_the_target_distribution(ctx):
    from oracle import ising, kitaev
    from paper_2008_05401_gb300 import KITAEV, MIXED
    L, beta, C = 3, 4.0, 8192
    J = (1.0, 1.0, 1.0)
    vs = ising.all_states(L)
    lw = kitaev.log_weight(vs, np.full(len(vs), beta), J)
    p = np.exp(lw - lw.max())
    p /= p.sum()
    g = np.random.default_rng(L)
    W, hb, vb = g.normal(0, 0.3, (4, 3, 3)), g.normal(0, 0.3, 4), 0.1
    v0 = vs[g.choice(len(vs), size=C, p=p)]
    mid = ctx.load_model(KITAEV, W, vb, hb)
    job = ctx.new_job(mid, KITAEV, L, np.full(C, 1 / beta), J, 21, 0, wl.pack_bits(v0), MIXED)
    job.run(5, precision=MIXED)
    bits, _ = job.state()
    v = wl.unpack_bits(bits, L).reshape(C, -1).astype(np.int64)
    idx = (v << np.arange(L * L)).sum(1)
    chi2, df, ok = _chi2_ok(idx, p, C)
    assert ok, (chi2, df)
    job.release()


def test_small_ising_workload_matches_kaufman(ctx):
    """L = 8, T = 2.269 (the small Ising workload geometry): the analytic CRBM
    accepts every proposal; after burn-in the mean energy per chain agrees with
    Kaufman's exact finite-torus <E> within 4 standard errors."""
    from oracle import ising
    from paper_2008_05401_gb300 import ISING, MIXED
    L, T, C, S = 8, 2.269, 1024, 400
    W, hb, vb = ising.analytic_crbm(1 / T, 2)
    mid = ctx.load_model(ISING, W, vb, hb)
    warm = ctx.new_job(mid, ISING, L, np.full(C, T), (1.0,), 2008054010, 0, None, MIXED)
    warm.run(100, precision=MIXED)
    bits, _ = warm.state()
    job = ctx.new_job(mid, ISING, L, np.full(C, T), (1.0,), 2008054010, 0, bits, MIXED)
    job.write_state(bits, 100)
    job.run(S, precision=MIXED)
    sums, acc, _ = job.observables()
    assert np.all(acc == S)
    per_chain = sums[:, 0] / S
    mean, err = per_chain.mean(), per_chain.std(ddof=1) / np.sqrt(C)
    exact = ising.kaufman_moments(L, 1 / T)["E"]
    assert abs(mean - exact) < 4 * err, (mean, err, exact)
    warm.release()
    job.release()


def test_full_size_batch_launch_sampled_parity(ctx):
    """The L = 128 job of the batch workload in its bench launch configuration
    (4096 chains, K = 4 filters 5 x 5, mixed precision): chains sampled across
    the grid are replayed by the oracle from the same initial lattices."""
    from paper_2008_05401_gb300 import ISING, MIXED
    L, n, S = 128, 4096, 2
    W, hb, vb = wl.gaussian_crbm(4, 5, 0.1)
    T = wl.ising_ladder(n, 32)
    bits0 = wl.pack_bits(wl.random_lattices(n, L, seed=2008054010 + L))
    mid = ctx.load_model(ISING, W, vb, hb)
    job = ctx.new_job(mid, ISING, L, T, (1.0,), 2008054010, 0, bits0, MIXED)
    job.run(S, precision=MIXED)
    bits, _ = job.state()
    lp, F, E = job.energies()
    _, acc, _ = job.observables()
    for c in (0, 1, 1517, 4095):
        ref = oracle_chains("ising", W, hb, vb, L, T[c:c + 1], (1.0,), 2008054010, 1, bits0[c:c + 1], cid_base=c)
        worst = run_oracle(ref, S)
        if not decisions_are_clear(worst):
            continue
        np.testing.assert_array_equal(bits[c:c + 1], wl.pack_bits(ref.v))
        assert acc[c] == ref.accepts[0]
        np.testing.assert_allclose(E[c], ref.E_phys[0], rtol=1e-12)
        # F is the FP32-path value unless a recompute made it exact: within its bound
        np.testing.assert_allclose(F[c], ref.F[0], rtol=2e-6)
    job.release()
