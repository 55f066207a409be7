"""Pins for the oracle's CRBM (Eqs. 12-13, B1-B4, App. C), CPU only."""
import itertools

import numpy as np
import pytest

from oracle import crbm, ising


def _params(K, k, seed, std=0.7):
    g = np.random.default_rng(seed)
    return g.normal(0, std, (K, k, k)), g.normal(0, std, K), float(g.normal(0, std))


def _all(nbits):
    n = np.arange(2 ** nbits)
    return ((n[:, None] >> np.arange(nbits)) & 1).astype(np.uint8)


@pytest.mark.parametrize("L,K,k", [(2, 2, 2), (3, 1, 3), (2, 3, 2)])
def test_free_energy_is_marginal_of_joint_energy(L, K, k):
    """sum_h exp(-E(v,h)) == exp(-F(v)) for every v (Eqs. 12-13, Eq. 3)."""
    W, hb, vb = _params(K, k, seed=L * 10 + K)
    N = L * L
    hs = _all(K * N).reshape(-1, K, L, L)
    for vbits in _all(N):
        v = vbits.reshape(1, L, L)
        E = crbm.joint_energy(np.repeat(v, len(hs), axis=0), hs, W, hb, vb)
        lhs = np.log(np.exp(-E - (-E).max()).sum()) + (-E).max()
        assert lhs == pytest.approx(-crbm.free_energy(v, W, hb, vb)[0], rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("L,K,k", [(2, 2, 2), (3, 1, 3)])
def test_conditionals_match_joint_distribution(L, K, k):
    """P(h_unit=1|v) = sigma(a) and P(v_site=1|h) = sigma(b), both read off the
    exact joint distribution exp(-E(v,h)) (Eqs. B1-B3)."""
    W, hb, vb = _params(K, k, seed=5 + L)
    N = L * L
    vs = _all(N).reshape(-1, L, L)
    hs = _all(K * N).reshape(-1, K, L, L)
    g = np.random.default_rng(1)
    for v in vs[g.choice(len(vs), 4, replace=False)]:
        E = crbm.joint_energy(np.repeat(v[None], len(hs), 0), hs, W, hb, vb)
        p = np.exp(-(E - E.min()))
        p /= p.sum()
        marg = (p[:, None] * hs.reshape(len(hs), -1)).sum(0)
        np.testing.assert_allclose(marg, crbm.sigmoid(crbm.hidden_preact(v[None], W, hb)).ravel(),
                                   rtol=1e-11, atol=1e-13)
    for h in hs[g.choice(len(hs), 4, replace=False)]:
        E = crbm.joint_energy(vs, np.repeat(h[None], len(vs), 0), W, hb, vb)
        p = np.exp(-(E - E.min()))
        p /= p.sum()
        marg = (p[:, None] * vs.reshape(len(vs), -1)).sum(0)
        np.testing.assert_allclose(marg, crbm.sigmoid(crbm.visible_preact(h[None], W, vb)).ravel(),
                                   rtol=1e-11, atol=1e-13)


def test_gibbs_kernel_detailed_balance():
    """P(v) T(v->v') = P(v') T(v'->v) with T = sum_h P(v'|h) P(h|v) (Eq. B4, App. B.1)."""
    L, K, k = 2, 2, 2
    W, hb, vb = _params(K, k, seed=11)
    N = L * L
    vs = _all(N).reshape(-1, L, L)
    hs = _all(K * N).reshape(-1, K, L, L)
    ph = crbm.sigmoid(crbm.hidden_preact(vs, W, hb)).reshape(len(vs), -1)      # (V, KN)
    Hf = hs.reshape(len(hs), -1)
    P_h_given_v = np.prod(np.where(Hf[None] == 1, ph[:, None], 1 - ph[:, None]), axis=2)  # (V, H)
    pv = crbm.sigmoid(crbm.visible_preact(hs, W, vb)).reshape(len(hs), -1)      # (H, N)
    Vf = vs.reshape(len(vs), -1)
    P_v_given_h = np.prod(np.where(Vf[None] == 1, pv[:, None], 1 - pv[:, None]), axis=2)  # (H, V)
    T = P_h_given_v @ P_v_given_h
    np.testing.assert_allclose(T.sum(1), 1.0, rtol=1e-13)
    F = crbm.free_energy(vs, W, hb, vb)
    P = np.exp(-(F - F.min()))
    P /= P.sum()
    flow = P[:, None] * T
    np.testing.assert_allclose(flow, flow.T, rtol=1e-11, atol=1e-16)
    # and P is stationary
    np.testing.assert_allclose(P @ T, P, rtol=1e-11)


@pytest.mark.parametrize("L,k,K", [(3, 3, 2), (5, 2, 3), (6, 4, 1), (8, 5, 4)])
def test_transposed_conv_is_adjoint(L, k, K):
    """<h, W*v> == <W^T (*) h, v> for real-valued fields (periodic conv adjoint)."""
    g = np.random.default_rng(L + k)
    W = g.normal(size=(K, k, k))
    v = g.normal(size=(2, L, L))
    h = g.normal(size=(2, K, L, L))
    lhs = (h * crbm.hidden_preact(v, W, np.zeros(K))).sum(axis=(1, 2, 3))
    rhs = (v * crbm.visible_preact(h, W, 0.0)).sum(axis=(1, 2))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


def test_free_energy_translation_invariant():
    W, hb, vb = _params(3, 3, seed=3)
    v = np.random.default_rng(2).integers(0, 2, (4, 7, 7))
    F = crbm.free_energy(v, W, hb, vb)
    np.testing.assert_allclose(crbm.free_energy(np.roll(v, (2, 5), axis=(1, 2)), W, hb, vb), F, rtol=1e-13)


@pytest.mark.parametrize("L,k", [(3, 2), (4, 2), (4, 3), (5, 4)])
def test_analytic_ising_crbm(L, k):
    """App. C: with W = W_min (Eq. C7), h_bias = -W, v_bias = -2W (Eq. C8) the
    CRBM free energy equals beta E(s) up to one constant for every lattice."""
    for beta in (0.25, 1 / 2.269, 0.8):
        W, hb, vb = ising.analytic_crbm(beta, k)
        # Eq. (C5): 2 beta = log sqrt((1+e^h)(1+e^{h+2W})) / (1+e^{h+W}) with h = hb
        h, w = hb[0], W[0, 0, 0]
        assert np.log(np.sqrt((1 + np.exp(h)) * (1 + np.exp(h + 2 * w))) / (1 + np.exp(h + w))) == \
            pytest.approx(2 * beta, rel=1e-12)
        vs = ising.all_states(L) if L * L <= 16 else np.random.default_rng(0).integers(0, 2, (512, L, L))
        d = crbm.free_energy(vs, W, hb, vb) - beta * ising.energy(vs)
        assert np.ptp(d) < 1e-9 * (1 + np.abs(d).max())
