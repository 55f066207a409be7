"""Pins for the oracle's open-boundary Kitaev model and locally connected CRBM
(Sec. IV, open boundary conditions).

Kitaev, open along j: with only y-bonds the spectrum is 2|Jy| (L(L-1) times,
one per bond) and 0 (L times); the Frobenius sum rule counts L(L-1) y-bonds;
rows stay translation invariant; Jy = 0 makes open and periodic identical.
LCRBM: brute-force marginalisation of its joint energy gives e^{-F}; flipping
one hidden or visible unit changes the joint energy by its pre-activation
(so the visible conditional is the exact transpose of the hidden one); with
1x1 kernels it is the periodic CRBM; the MH chain with an LCRBM proposal keeps
the exact open-boundary Kitaev distribution.
"""
import itertools

import numpy as np
import pytest

from oracle import chain, crbm, ising, kitaev, lcrbm
from test_oracle_chain import _chi2_ok, _state_index


def test_open_kitaev_y_bonds_only():
    L = 4
    v = np.random.default_rng(0).integers(0, 2, (3, L, L)).astype(np.uint8)
    eps = np.sort(kitaev.energies(v, (0.0, 1.3, 0.0), open_cols=True), axis=1)
    expect = np.sort(np.concatenate([np.zeros(L), np.full(L * (L - 1), 2.6)]))
    np.testing.assert_allclose(eps, np.broadcast_to(expect, eps.shape), atol=1e-12)
    eps_p = kitaev.energies(v, (0.0, 1.3, 0.0), open_cols=False)
    np.testing.assert_allclose(eps_p, 2.6, atol=1e-12)


def test_open_kitaev_sum_rule_and_symmetries():
    L = 5
    J = (0.7, 1.1, 1.3)
    v = np.random.default_rng(1).integers(0, 2, (4, L, L)).astype(np.uint8)
    eps = kitaev.energies(v, J, open_cols=True)
    N = L * L
    np.testing.assert_allclose((eps ** 2).sum(axis=1),
                               4 * (N * J[0] ** 2 + N * J[2] ** 2 + L * (L - 1) * J[1] ** 2), rtol=1e-12)
    # rows (i) stay periodic: translation along i keeps the spectrum
    np.testing.assert_allclose(np.sort(kitaev.energies(np.roll(v, 2, axis=1), J, True), axis=1),
                               np.sort(eps, axis=1), atol=1e-11)
    # columns do not: a shift along j changes it for some lattice
    diff = np.abs(np.sort(kitaev.energies(np.roll(v, 1, axis=2), J, True), axis=1) - np.sort(eps, axis=1))
    assert diff.max() > 1e-6
    # the 2N x 2N Majorana spectrum is +-eps
    ms = kitaev.majorana_spectrum(v[:1], J, open_cols=True)[0]
    np.testing.assert_allclose(np.sort(np.abs(ms))[::2], np.sort(eps[0]), atol=1e-10)
    # without y-bonds open and periodic coincide
    J0 = (0.7, 0.0, 1.3)
    np.testing.assert_allclose(kitaev.energies(v, J0, True), kitaev.energies(v, J0, False), atol=1e-12)


def test_open_vison_density():
    L = 4
    assert kitaev.vison_density(np.ones((1, L, L), dtype=np.uint8), open_cols=True)[0] == 0.0
    v = np.zeros((1, L, L), dtype=np.uint8)
    v[0, :, ::2] = 1          # alternating columns: every hexagon between columns j, j+1 has flux -1
    assert kitaev.vison_density(v, open_cols=True)[0] == 1.0
    assert kitaev.vison_density(v, open_cols=False)[0] == 1.0


def _lc_params(edge, K, k, seed, scale=0.5):
    g = np.random.default_rng(seed)
    return g.normal(0, scale, (2 * edge + 1, K, k, k)), g.normal(0, scale, K), g.normal(0, scale)


def test_lcrbm_free_energy_marginalises_joint_energy():
    L, K, k, edge = 3, 1, 2, 1
    W, hb, vb = _lc_params(edge, K, k, 3)
    vs = ising.all_states(L)
    hs = np.array(list(itertools.product([0, 1], repeat=K * L * L)), dtype=np.uint8).reshape(-1, K, L, L)
    F = lcrbm.free_energy(vs, W, hb, vb, edge)
    for n in range(0, len(vs), 97):
        E = lcrbm.joint_energy(np.repeat(vs[n:n + 1], len(hs), axis=0), hs, W, hb, vb, edge)
        np.testing.assert_allclose(-np.log(np.exp(-E).sum()), F[n], rtol=1e-12, atol=1e-12)


def test_lcrbm_conditionals_from_joint_energy():
    L, K, k, edge = 5, 2, 3, 2
    W, hb, vb = _lc_params(edge, K, k, 4)
    g = np.random.default_rng(5)
    v = g.integers(0, 2, (1, L, L)).astype(np.uint8)
    h = g.integers(0, 2, (1, K, L, L)).astype(np.uint8)
    a = lcrbm.hidden_preact(v, W, hb, edge)
    b = lcrbm.visible_preact(h, W, vb, edge)
    for f, i, j in [(0, 0, 0), (1, 2, 4), (0, 4, 3), (1, 1, 1)]:
        h0, h1 = h.copy(), h.copy()
        h0[0, f, i, j], h1[0, f, i, j] = 0, 1
        dE = lcrbm.joint_energy(v, h0, W, hb, vb, edge) - lcrbm.joint_energy(v, h1, W, hb, vb, edge)
        assert dE[0] == pytest.approx(a[0, f, i, j], abs=1e-12)
    for i, j in [(0, 0), (3, 4), (2, 1), (4, 2)]:
        v0, v1 = v.copy(), v.copy()
        v0[0, i, j], v1[0, i, j] = 0, 1
        dE = lcrbm.joint_energy(v0, h, W, hb, vb, edge) - lcrbm.joint_energy(v1, h, W, hb, vb, edge)
        assert dE[0] == pytest.approx(b[0, i, j], abs=1e-12)


def test_lcrbm_with_1x1_kernels_is_the_crbm():
    L, K, edge = 6, 2, 2
    g = np.random.default_rng(6)
    w = g.normal(0, 1, (K, 1, 1))
    W = np.broadcast_to(w, (2 * edge + 1, K, 1, 1)).copy()
    hb, vb = g.normal(0, 1, K), 0.3
    v = g.integers(0, 2, (3, L, L)).astype(np.uint8)
    np.testing.assert_allclose(lcrbm.free_energy(v, W, hb, vb, edge), crbm.free_energy(v, w, hb, vb), rtol=1e-13)


@pytest.mark.parametrize("L", [2, 3])
def test_open_kitaev_chain_with_lcrbm_keeps_target(L):
    J, beta, edge = (1.0, 0.9, 1.2), 4.0, 1
    vs = ising.all_states(L)
    lw = kitaev.log_weight(vs, np.full(len(vs), beta), J, open_cols=True)
    p = np.exp(lw - lw.max())
    p /= p.sum()
    W, hb, vb = _lc_params(edge, 2, 2, L, scale=0.3)
    g = np.random.default_rng(L + 11)
    C = 8192
    ch = chain.make_chains(chain.KITAEV, W, hb, vb, L, 1 / beta, J, 13, np.arange(C),
                           v0=vs[g.choice(len(vs), size=C, p=p)], edge=edge)
    chain.run(ch, 5)
    assert 0.02 < ch.accepts.mean() / ch.step < 0.99
    chi2, df, ok = _chi2_ok(_state_index(ch.v), p)
    assert ok, (chi2, df)
