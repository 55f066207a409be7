"""Pins for the oracle's trainer (Sec. II, App. A, Algorithm 1).

* dF/dtheta and d loss/d theta against central finite differences of F and
  of the loss (which use no gradient code);
* App. C: the analytic Ising CRBM reproduces beta E up to a constant, so its
  loss is zero and its gradient vanishes;
* ADAM: the first step moves every parameter by lr against the sign of its
  gradient, updates do not depend on the scale of the gradient, and ADAM
  drives a quadratic to its minimum;
* the paper's Ising protocol (App. D): training on all 512 states of L = 3
  lowers the loss by orders of magnitude and brings P_CRBM close to P_Ising.
"""
import numpy as np
import pytest

import crbm_workloads as wl
from oracle import chain, crbm, ising, train


def _theta(K, k, seed, scale=0.3):
    g = np.random.default_rng(seed)
    return g.normal(0, scale, K * k * k + 1 + K)


def test_free_energy_gradient_matches_finite_differences():
    K, k, L = 2, 3, 4
    th = _theta(K, k, 1)
    v = wl.random_lattices(5, L, seed=2)
    F, G = train.free_energy_grad(v, th, K, k)
    W, hb, vb = train.split(th, K, k)
    np.testing.assert_allclose(F, crbm.free_energy(v, W, hb, vb), rtol=1e-14)
    h = 1e-5
    for p in range(len(th)):
        e = np.zeros_like(th)
        e[p] = h
        Fp = crbm.free_energy(v, *train.split(th + e, K, k))
        Fm = crbm.free_energy(v, *train.split(th - e, K, k))
        np.testing.assert_allclose(G[:, p], (Fp - Fm) / (2 * h), rtol=1e-6, atol=1e-7)


def test_loss_gradient_matches_finite_differences():
    K, k, L = 2, 2, 3
    th = _theta(K, k, 3)
    v = wl.random_lattices(20, L, seed=4)
    t = ising.energy(v) / 2.2
    loss, g = train.loss_and_grad(v, t, th, K, k)
    h = 1e-6
    for p in range(len(th)):
        e = np.zeros_like(th)
        e[p] = h
        lp, _ = train.loss_and_grad(v, t, th + e, K, k)
        lm, _ = train.loss_and_grad(v, t, th - e, K, k)
        assert g[p] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-8)


def test_analytic_crbm_has_zero_loss():
    beta = 1 / 2.2
    W, hb, vb = ising.analytic_crbm(beta, 2)
    K, k = W.shape[0], W.shape[1]
    th = np.concatenate([W.ravel(), [vb], hb])
    v = ising.all_states(3)
    loss, g = train.loss_and_grad(v, beta * ising.energy(v), th, K, k)
    assert loss < 1e-24
    assert np.abs(g).max() < 1e-11
    # a sign error in the target (or in F) leaves a large loss
    bad, _ = train.loss_and_grad(v, -beta * ising.energy(v), th, K, k)
    assert bad > 1.0


def test_adam_first_step_and_scale_invariance():
    th = np.array([0.5, -0.2, 0.0])
    g = np.array([3.0, -1e-3, 0.0])
    st = train.Adam.zeros(3)
    new = train.adam_step(th, g, st, lr=1e-3)
    np.testing.assert_allclose(new - th, [-1e-3, 1e-3, 0.0], rtol=1e-4, atol=1e-12)
    st1, st2 = train.Adam.zeros(3), train.Adam.zeros(3)
    a, b = th.copy(), th.copy()
    rng = np.random.default_rng(0)
    for _ in range(20):
        gg = rng.normal(size=3)
        a = train.adam_step(a, gg, st1)
        b = train.adam_step(b, 1000.0 * gg, st2)
    np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-9)


def test_adam_minimises_a_quadratic():
    target = np.array([1.0, -2.0, 0.5])
    th = np.zeros(3)
    st = train.Adam.zeros(3)
    for _ in range(3000):
        th = train.adam_step(th, th - target, st, lr=1e-2)
    np.testing.assert_allclose(th, target, atol=1e-3)


def test_ising_L3_training_learns_the_distribution():
    """App. D: K = 2 kernels 2x2 trained on all 512 states of L = 3 at T = 2.2."""
    K, k, L, beta = 2, 2, 3, 1 / 2.2
    v = ising.all_states(L)
    t = beta * ising.energy(v)
    th = wl.init_train_params(K, k, seed=5)
    st = train.Adam.zeros(len(th))
    l0, _ = train.loss_and_grad(v, t, th, K, k)
    for e in range(400):
        th, ls = train.epoch(th, st, v, t, wl.epoch_order(len(v), 9, e), K, k, M=20, lr=1e-2)
    l1, _ = train.loss_and_grad(v, t, th, K, k)
    assert l1 < 1e-3 * l0, (l0, l1)
    # P_CRBM ~ e^{-F} against P_Ising ~ e^{-beta E}: KL divergence small
    W, hb, vb = train.split(th, K, k)
    lq = -crbm.free_energy(v, W, hb, vb)
    lp = -t
    q = np.exp(lq - lq.max()); q /= q.sum()
    p = np.exp(lp - lp.max()); p /= p.sum()
    assert (q * np.log(q / p)).sum() < 1e-3


def test_algorithm1_reduces_the_loss():
    K, k, L = 2, 3, 4
    th0 = wl.init_train_params(K, k, seed=1)
    th, st, losses = train.algorithm1(chain.ISING, L, 2.5, (1.0,), K, k, th0, n_phys=64, phys_sweeps=20,
                                      phys_seed=3, n_train=64, ub=16, g=2, rbm_seed=4, epochs=30,
                                      order_seed=5, M=20, lr=1e-2)
    assert st.t == 30 * ((64 + 64 + 19) // 20)
    assert losses[-1] < 0.5 * losses[0]
