"""Pins for the oracle's proposal + Metropolis-Hastings chain (App. B, Eq. B5).

Each stationarity test starts every chain from an exact draw of the target
distribution (enumerated on a tiny lattice) and checks, by a chi^2 test on
independent chains, that a few proposals leave that distribution unchanged.
Dropping the F(v') - F(v) term, flipping its sign or losing the visible bias
each fails these tests by hundreds of chi^2 units.
"""
import numpy as np
import pytest

from oracle import chain, crbm, ising, kitaev


def _chi2_ok(samples_idx, probs, n_bins_min=5.0):
    C = len(samples_idx)
    cnt = np.bincount(samples_idx, minlength=len(probs)).astype(float)
    m = probs * C > n_bins_min
    # pool the rare bins into one
    obs = np.append(cnt[m], cnt[~m].sum())
    exp = np.append(probs[m] * C, probs[~m].sum() * C)
    keep = exp > 0
    chi2 = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    df = keep.sum() - 1
    return chi2, df, chi2 < df + 6.0 * np.sqrt(2.0 * df)


def _state_index(v):
    C = v.shape[0]
    bits = v.reshape(C, -1).astype(np.int64)
    return (bits << np.arange(bits.shape[1])).sum(axis=1)


def _perturbed_analytic(beta, k, seed):
    W, hb, vb = ising.analytic_crbm(beta, k)
    g = np.random.default_rng(seed)
    return W + g.normal(0, 0.4, W.shape), hb + g.normal(0, 0.4, 2), vb + 0.3


def test_analytic_crbm_accepts_every_proposal():
    """App. C: P_CRBM == P_Ising, so log r == 0 and every proposal is accepted."""
    beta = 1 / 2.269
    W, hb, vb = ising.analytic_crbm(beta, 3)
    ch = chain.make_chains(chain.ISING, W, hb, vb, 6, 1 / beta, (1.0,), 17, np.arange(32))
    logs = []
    chain.run(ch, 25, record=lambda c, d: logs.append(d["log_r"]))
    assert np.all(ch.accepts == 25)
    assert np.abs(np.array(logs)).max() < 1e-10


@pytest.mark.parametrize("g_steps", [1, 2])
def test_ising_mh_chain_keeps_target_distribution(g_steps):
    L, beta = 4, 0.35
    W, hb, vb = _perturbed_analytic(beta, 3, seed=3)
    vs = ising.all_states(L)
    lw = -beta * ising.energy(vs)
    p = np.exp(lw - lw.max())
    p /= p.sum()
    rng = np.random.default_rng(11)
    C = 8192
    ch = chain.make_chains(chain.ISING, W, hb, vb, L, 1 / beta, (1.0,), 5, np.arange(C),
                           v0=vs[rng.choice(len(vs), size=C, p=p)])
    chain.run(ch, 8, g=g_steps)
    acc = ch.accepts.mean() / ch.step
    assert 0.1 < acc < 0.95
    # energy levels
    E = ising.energy(vs)
    levels, inv = np.unique(E, return_inverse=True)
    pe = np.bincount(inv, weights=p)
    idx = np.searchsorted(levels, ising.energy(ch.v))
    chi2, df, ok = _chi2_ok(idx, pe)
    assert ok, (chi2, df)


def test_uncorrected_chain_keeps_crbm_distribution():
    """correct=False is plain Gibbs sampling: its stationary law is exp(-F)/Z (App. B.1)."""
    L = 3
    g = np.random.default_rng(4)
    W, hb, vb = g.normal(0, 0.6, (2, 2, 2)), g.normal(0, 0.6, 2), 0.2
    vs = ising.all_states(L)
    F = crbm.free_energy(vs, W, hb, vb)
    q = np.exp(-(F - F.min()))
    q /= q.sum()
    C = 16384
    ch = chain.make_chains(chain.ISING, W, hb, vb, L, 1.0, (1.0,), 8, np.arange(C),
                           v0=vs[g.choice(len(vs), size=C, p=q)])
    chain.run(ch, 4, correct=False)
    assert np.all(ch.accepts == 4)
    chi2, df, ok = _chi2_ok(_state_index(ch.v), q)
    assert ok, (chi2, df)


@pytest.mark.parametrize("L,beta", [(2, 2.0), (3, 4.0)])
def test_kitaev_mh_chain_keeps_target_distribution(L, beta):
    J = (1.0, 1.0, 1.0)
    vs = ising.all_states(L)
    lw = kitaev.log_weight(vs, np.full(len(vs), beta), J)
    p = np.exp(lw - lw.max())
    p /= p.sum()
    g = np.random.default_rng(L)
    W, hb, vb = g.normal(0, 0.3, (4, 3, 3)), g.normal(0, 0.3, 4), 0.1
    C = 8192
    ch = chain.make_chains(chain.KITAEV, W, hb, vb, L, 1 / beta, J, 21, np.arange(C),
                           v0=vs[g.choice(len(vs), size=C, p=p)])
    chain.run(ch, 5)
    assert 0.02 < ch.accepts.mean() / ch.step < 0.99
    chi2, df, ok = _chi2_ok(_state_index(ch.v), p)
    assert ok, (chi2, df)


def test_observable_sums_and_resume():
    """Sums add the observables of the post-decision state; splitting a run in
    two (counter-based RNG) gives the identical chain."""
    W, hb, vb = _perturbed_analytic(0.4, 3, seed=1)
    a = chain.make_chains(chain.ISING, W, hb, vb, 6, 2.5, (1.0,), 3, np.arange(8))
    b = chain.make_chains(chain.ISING, W, hb, vb, 6, 2.5, (1.0,), 3, np.arange(8))
    E_trace = []
    chain.run(a, 12, record=lambda c, d: E_trace.append(ising.energy(c.v)))
    chain.run(b, 5)
    b2 = chain.make_chains(chain.ISING, W, hb, vb, 6, 2.5, (1.0,), 3, np.arange(8), v0=b.v)
    b2.step = b.step
    chain.run(b2, 7)
    np.testing.assert_array_equal(a.v, b2.v)
    np.testing.assert_allclose(a.obs[:, 0], np.sum(E_trace, axis=0))
    np.testing.assert_allclose(a.obs[:, 1], np.sum(np.square(E_trace), axis=0))
