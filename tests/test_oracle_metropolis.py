"""Pins for the oracle's local-update Metropolis baselines and its integrated
autocorrelation time.

Metropolis: chains started in the exact distribution (enumerated on a tiny
lattice) must keep it (chi^2 on independent chains), alone and with the
neighbour temperature exchange; a planted sign error in dE, or a dropped beta,
fails the same test.  tau: closed forms -- an AR(1) series has
tau = (1 + rho) / (2 (1 - rho)); independent samples 1/2; an alternating series
gives tau = 1/2 - (n-1)/n at W = 1 exactly.
"""
import numpy as np
import pytest

from oracle import autocorr, chain, ising, kitaev, metropolis
from test_oracle_chain import _chi2_ok, _state_index


def _ising_start(L, betas, per_T, seed):
    vs = ising.all_states(L)
    E = ising.energy(vs)
    rng = np.random.default_rng(seed)
    v0 = np.empty((per_T * len(betas), L, L), dtype=np.uint8)
    for t, b in enumerate(betas):
        p = np.exp(-b * E - (-b * E).max())
        v0[t::len(betas)] = vs[rng.choice(len(vs), size=per_T, p=p / p.sum())]
    return vs, E, v0


def _ising_chi2(betas, per_T, sweeps, exchange, seed=3):
    L = 4
    vs, E, v0 = _ising_start(L, betas, per_T, seed)
    W, hb, vb = np.zeros((1, 2, 2)), np.zeros(1), 0.0
    T = np.tile(1 / np.asarray(betas), per_T)
    ch = chain.make_chains(chain.ISING, W, hb, vb, L, T, (1.0,), 11, np.arange(len(T)), v0=v0)
    n_temp = 0
    for _ in range(sweeps):
        d = metropolis.sweep(ch, exchange)
        n_temp += d["temp"].sum()
    levels, inv = np.unique(E, return_inverse=True)
    Ec = ising.energy(ch.v)
    res = []
    for t, b in enumerate(betas):
        p = np.exp(-b * E - (-b * E).max())
        pe = np.bincount(inv, weights=p / p.sum())
        res.append(_chi2_ok(np.searchsorted(levels, Ec[t::len(betas)]), pe))
    return res, ch, n_temp


def test_ising_checkerboard_keeps_boltzmann():
    res, ch, _ = _ising_chi2([0.3, 0.44], 4096, 3, False)
    for chi2, df, ok in res:
        assert ok, (chi2, df)
    assert 0.1 < ch.accepts.sum() / (ch.step * 16 * len(ch.chain_ids)) < 0.9


def test_ising_checkerboard_with_exchange_keeps_boltzmann():
    res, _, n_temp = _ising_chi2([0.25, 0.32, 0.4, 0.48], 2048, 4, True)
    assert n_temp > 500
    for chi2, df, ok in res:
        assert ok, (chi2, df)


@pytest.mark.parametrize("plant", ["sign", "beta"])
def test_planted_metropolis_mistakes_fail(monkeypatch, plant):
    dE = metropolis._delta_E
    if plant == "sign":
        monkeypatch.setattr(metropolis, "_delta_E", lambda s, J: -dE(s, J))
    else:   # the Boltzmann factor at beta = 1 instead of the chain's beta
        monkeypatch.setattr(metropolis, "_delta_E", lambda s, J: dE(s, J) * 0.4 / np.array([0.3, 0.44])[
            np.arange(s.shape[0]) % 2][:, None, None])
    res, _, _ = _ising_chi2([0.3, 0.44], 4096, 3, False)
    assert sum(chi2 for chi2, _, _ in res) > 500


def test_ising_sweep_is_a_checkerboard():
    """Sites of one colour are updated from the lattice left by the other
    colour: a lattice whose even sites all flip must present the odd sites
    with the flipped neighbours (zero-temperature limit, deterministic)."""
    L = 4
    v0 = np.ones((1, L, L), dtype=np.uint8)
    v0[0, ::2, ::2] = 0
    v0[0, 1::2, 1::2] = 0          # antiferromagnetic checkerboard: every flip lowers E
    ch = chain.make_chains(chain.ISING, np.zeros((1, 2, 2)), np.zeros(1), 0.0, L, 1e-3, (1.0,), 1,
                           np.arange(1), v0=v0)
    metropolis.sweep(ch)
    # even sites flip to 1 (all neighbours 1); then odd sites see all-1 neighbours and stay 1
    assert ch.v.all()
    assert ch.accepts[0] == L * L // 2


@pytest.mark.parametrize("L", [2, 3])
def test_kitaev_local_keeps_target_distribution(L):
    J = (1.0, 0.9, 1.2)
    beta = 4.0
    vs = ising.all_states(L)
    lw = kitaev.log_weight(vs, np.full(len(vs), beta), J)
    p = np.exp(lw - lw.max())
    p /= p.sum()
    g = np.random.default_rng(L + 7)
    C = 8192
    ch = chain.make_chains(chain.KITAEV, np.zeros((1, 2, 2)), np.zeros(1), 0.0, L, 1 / beta, J, 5,
                           np.arange(C), v0=vs[g.choice(len(vs), size=C, p=p)])
    metropolis.run(ch, 2)
    assert 0.02 < ch.accepts.sum() / (2 * L * L * C) < 0.98
    chi2, df, ok = _chi2_ok(_state_index(ch.v), p)
    assert ok, (chi2, df)


def test_tau_ar1_closed_form():
    rng = np.random.default_rng(0)
    for rho in (0.0, 0.5, 0.8):
        n = 200_000
        e = rng.normal(size=n)
        x = np.empty(n)
        x[0] = e[0] / np.sqrt(1 - rho ** 2)
        for t in range(1, n):
            x[t] = rho * x[t - 1] + e[t]
        tau, W = autocorr.tau_int(x)
        exact = (1 + rho) / (2 * (1 - rho))
        assert abs(tau - exact) < 0.1 * exact, (rho, tau, exact, W)
        assert W >= 5 * tau


def test_tau_exact_small_cases():
    n = 10
    x = np.tile([1.0, -1.0], n // 2)
    tau, W = autocorr.tau_int(x)
    assert W == 1
    assert tau == pytest.approx(0.5 - (n - 1) / n, abs=1e-15)
    assert autocorr.tau_int(np.full(7, 3.0)) == (0.5, 0)
    taus, Ws = autocorr.tau_int_columns(np.stack([x, -x], axis=1))
    np.testing.assert_allclose(taus, [tau, tau])
