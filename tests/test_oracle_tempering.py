"""Pins for the oracle's parallel-tempering exchange correction (App. B.2).

Physical chains start in equilibrium at their own temperature and RBM chains in
P_CRBM; after several cycles (Gibbs steps of the RBM chains, Eq. B5 swaps with
the physical chains, neighbour temperature exchanges) every temperature must
still hold its Boltzmann distribution (chi^2 on energy levels, Ising L = 4,
enumerated exactly).  Two planted mistakes -- the swap without its F term, and
temperature exchanges accepted unconditionally -- each fail the same test by
thousands of chi^2 units.
"""
import numpy as np
import pytest

from oracle import chain, crbm, ising, tempering
from test_oracle_chain import _chi2_ok, _perturbed_analytic

BETAS = np.array([0.25, 0.32, 0.4, 0.48])


def _pt_chi2(k, ladders=3000, cycles=6):
    L = 4
    W, hb, vb = _perturbed_analytic(0.35, 3, seed=7)
    vs = ising.all_states(L)
    E = ising.energy(vs)
    T = np.tile(1 / BETAS, ladders)
    rng = np.random.default_rng(5)

    def draws(lw, size):
        p = np.exp(lw - lw.max())
        return vs[rng.choice(len(vs), size=size, p=p / p.sum())]

    v0 = np.empty((len(T), L, L), dtype=np.uint8)
    for t, b in enumerate(BETAS):
        v0[t::len(BETAS)] = draws(-b * E, ladders)
    y0 = draws(-crbm.free_energy(vs, W, hb, vb), len(T))
    ids = np.arange(len(T))
    phys = chain.make_chains(chain.ISING, W, hb, vb, L, T, (1.0,), 3, ids, v0=v0)
    rbm = chain.make_chains(chain.ISING, W, hb, vb, L, T, (1.0,), 3, ids + len(T), v0=y0)
    n_swap = n_temp = 0
    for c in range(cycles):
        d = tempering.cycle(phys, rbm, k)
        n_swap += d["swap"].sum()
        n_temp += d["temp"].sum()
    levels, inv = np.unique(E, return_inverse=True)
    Ec = ising.energy(phys.v)
    out = []
    for t, b in enumerate(BETAS):
        p = np.exp(-b * E - (-b * E).max())
        pe = np.bincount(inv, weights=p / p.sum())
        out.append(_chi2_ok(np.searchsorted(levels, Ec[t::len(BETAS)]), pe))
    return out, n_swap, n_temp


@pytest.mark.parametrize("k", [1, 3])
def test_pt_cycles_keep_every_temperature_exact(k):
    res, n_swap, n_temp = _pt_chi2(k)
    assert n_swap > 1000 and n_temp > 1000
    for t, (chi2, df, ok) in enumerate(res):
        assert ok, (t, chi2, df)


def test_planted_swap_without_F_term_fails(monkeypatch):
    # the F(y) - F(x) term replaced by zero: log a = log pi(y) - log pi(x)
    monkeypatch.setattr(chain.Chains, "free", lambda self, v: np.zeros(len(v)))
    res, _, _ = _pt_chi2(1)
    assert sum(chi2 for chi2, _, _ in res) > 1000


def test_planted_unconditional_temperature_exchange_fails(monkeypatch):
    monkeypatch.setattr(tempering, "_log_weight_at", lambda ch, v, b: np.full(len(v), 1e300))
    res, _, _ = _pt_chi2(1)
    assert sum(chi2 for chi2, _, _ in res) > 1000


def test_kitaev_cycle_keeps_chain_state_consistent():
    """After swaps and temperature exchanges the bookkept log pi, e and F of
    every chain equal a fresh evaluation of its (state, temperature)."""
    L = 3
    J = (1.0, 1.0, 1.0)
    g = np.random.default_rng(2)
    W, hb, vb = g.normal(0, 0.3, (4, 3, 3)), g.normal(0, 0.3, 4), 0.1
    T = np.tile([0.3, 0.5, 0.8, 1.2], 8)
    ids = np.arange(len(T))
    phys = chain.make_chains(chain.KITAEV, W, hb, vb, L, T, J, 9, ids)
    rbm = chain.make_chains(chain.KITAEV, W, hb, vb, L, T, J, 9, ids + 100)
    swaps = temps = 0
    for c in range(5):
        d = tempering.cycle(phys, rbm, 2)
        swaps += d["swap"].sum()
        temps += d["temp"].sum()
    assert swaps > 0 and temps > 0
    for ch in (phys, rbm):
        lp, e, ot = chain.target(chain.KITAEV, ch.v, ch.beta, J)
        np.testing.assert_allclose(ch.logpi, lp, rtol=1e-12)
        np.testing.assert_allclose(ch.E_phys, e, rtol=1e-12)
        np.testing.assert_allclose(ch.obs_terms, ot, rtol=1e-12)
        np.testing.assert_allclose(ch.F, crbm.free_energy(ch.v, W, hb, vb), rtol=1e-12)
