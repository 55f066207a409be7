"""Pins for the oracle's target models: Ising (Eq. 14) and Kitaev (Eqs. 15-16)."""
import numpy as np
import pytest

import crbm_workloads as wl
from oracle import ising, kitaev


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("beta", [0.2, 1 / 2.269, 0.7])
def test_ising_enumeration_matches_kaufman(L, beta):
    """Brute-force sums over every lattice vs Kaufman's closed-form torus Z."""
    ex = ising.enumerate_exact(L, beta)
    km = ising.kaufman_moments(L, beta)
    assert ex["logZ"] == pytest.approx(km["logZ"], rel=1e-13)
    assert ex["E"] == pytest.approx(km["E"], rel=1e-11, abs=1e-11)
    assert ex["E2"] - ex["E"] ** 2 == pytest.approx(km["varE"], rel=1e-10)


def test_ising_energy_special_states():
    for L in (2, 4, 6):
        N = L * L
        up = np.ones((1, L, L), dtype=np.uint8)
        assert ising.energy(up)[0] == -2 * N
        assert ising.energy(1 - up)[0] == -2 * N
        chk = (np.add.outer(np.arange(L), np.arange(L)) % 2).astype(np.uint8)[None]
        assert ising.energy(chk)[0] == 2 * N
        assert ising.magnetisation(up)[0] == N
    # one flipped spin in a ferromagnet costs 2 J per bond, 4 bonds
    v = np.ones((1, 5, 5), dtype=np.uint8)
    v[0, 2, 3] = 0
    assert ising.energy(v)[0] == -2 * 25 + 8


@pytest.mark.parametrize("L", [2, 3, 4, 5, 6, 8])
@pytest.mark.parametrize("J", [(1.0, 1.0, 1.0), (0.3, 1.2, 0.7)])
def test_kitaev_uniform_eta_matches_bloch_closed_form(L, J):
    for eta in (1.0, -1.0):
        v = np.full((1, L, L), 1 if eta > 0 else 0, dtype=np.uint8)
        np.testing.assert_allclose(np.sort(kitaev.energies(v, J)[0]), kitaev.bloch_energies(L, J, eta),
                                   atol=1e-12)


@pytest.mark.parametrize("L", [2, 3, 4, 6])
def test_kitaev_sum_rule_and_majorana_spectrum(L):
    J = (0.9, 1.1, 1.3)
    v = wl.random_lattices(5, L, seed=L)
    eps = kitaev.energies(v, J)
    N = L * L
    np.testing.assert_allclose((eps ** 2).sum(1), 4 * N * (J[0] ** 2 + J[1] ** 2 + J[2] ** 2), rtol=1e-12)
    spec = kitaev.majorana_spectrum(v, J)                        # 2N eigenvalues of iA, +-eps
    np.testing.assert_allclose(np.sort(eps, 1), spec[:, N:], atol=1e-11)
    np.testing.assert_allclose(spec[:, :N], -spec[:, N:][:, ::-1], atol=1e-11)


@pytest.mark.parametrize("L", [4, 6])
def test_kitaev_symmetries(L):
    J = (1.0, 1.0, 1.0)
    v = wl.random_lattices(4, L, seed=3)
    beta = np.array([0.5, 2.0, 10.0, 200.0])
    lp = kitaev.log_weight(v, beta, J)
    np.testing.assert_allclose(kitaev.log_weight(np.roll(v, (1, 3), axis=(1, 2)), beta, J), lp, rtol=1e-12)
    # even L: flipping every eta is a signed-diagonal similarity of M
    np.testing.assert_allclose(kitaev.log_weight(1 - v, beta, J), lp, rtol=1e-12)
    # isotropic J: exchanging the two in-plane axes (transpose) leaves the spectrum
    np.testing.assert_allclose(kitaev.log_weight(np.transpose(v, (0, 2, 1)), beta, J), lp, rtol=1e-12)


@pytest.mark.parametrize("L", [4, 6])
def test_kitaev_flux_free_is_lowest(L):
    """Ground-state energy -1/2 sum eps of uniform eta lies below every single flip."""
    J = (1.0, 1.0, 1.0)
    v0 = np.ones((1, L, L), dtype=np.uint8)
    E0 = -0.5 * kitaev.energies(v0, J).sum()
    flips = np.repeat(v0, L * L, axis=0)
    flips.reshape(L * L, -1)[np.arange(L * L), np.arange(L * L)] = 0
    E1 = -0.5 * kitaev.energies(flips, J).sum(1)
    assert np.all(E1 > E0 + 1e-6)
    assert kitaev.vison_density(v0)[0] == 0.0
    np.testing.assert_allclose(kitaev.vison_density(flips), 2.0 / (L * L))


def test_kitaev_thermal_terms_are_beta_derivatives():
    """e = -d log pi / d beta and c_f = beta^2 d^2 log pi / d beta^2 per configuration."""
    J = (1.0, 1.0, 1.0)
    v = wl.random_lattices(3, 4, seed=9)
    eps = kitaev.energies(v, J)
    for beta in (0.3, 2.0, 20.0):
        h = 2e-3 * beta
        f = lambda b: kitaev.log_weight_from_eps(eps, np.full(3, b))
        fm2, fm1, f0, fp1, fp2 = (f(beta + m * h) for m in (-2, -1, 0, 1, 2))
        d1 = (fm2 - 8 * fm1 + 8 * fp1 - fp2) / (12 * h)               # 5-point stencils
        d2 = (-fm2 + 16 * fm1 - 30 * f0 + 16 * fp1 - fp2) / (12 * h * h)
        e, cf = kitaev.thermal_terms(eps, np.full(3, beta))
        np.testing.assert_allclose(e, -d1, rtol=1e-8)
        np.testing.assert_allclose(cf, beta ** 2 * d2, rtol=2e-5, atol=1e-8 * (1 + np.abs(f0).max()))
