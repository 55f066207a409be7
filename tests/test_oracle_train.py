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


def _metropolis_states(L, T, n, seed, sweeps=200):
    from oracle import metropolis
    K = 1
    ph = chain.make_chains(chain.ISING, np.zeros((K, 1, 1)), np.zeros(K), 0.0, L, T, (1.0,), seed, np.arange(n))
    metropolis.run(ph, sweeps)
    return ph.v.copy()


def test_pretraining_fits_random_states_and_helps_on_physical_states():
    """Pre-training (App. A; Sec. IV): epochs on 10^4 uniformly random lattices
    lower their loss tenfold, and the pre-trained CRBM fits physical
    (Metropolis) states far better than the initial one -- a target with the
    wrong sign would fit the random states just as well, but not these."""
    K, k, L, T = 2, 3, 6, 2.5
    th0 = wl.init_train_params(K, k, seed=1)
    th, st, losses, n = train.pretrain(chain.ISING, L, T, (1.0,), K, k, th0, n_random=10_000, seed=7,
                                       max_epochs=12, order_seed=3, M=20)
    assert n == len(losses) <= 12
    assert losses.min() < 0.1 * losses[0], losses
    x = _metropolis_states(L, T, 1000, 11)
    t = train.targets_of(chain.ISING, x, 1 / T, (1.0,))
    before, _ = train.loss_and_grad(x, t, th0, K, k)
    after, _ = train.loss_and_grad(x, t, th, K, k)
    assert after < 0.1 * before, (before, after)


def test_pretraining_keeps_the_analytic_crbm():
    """App. C's CRBM already has zero loss on every lattice: pre-training on
    random states leaves it (up to ADAM's steps on rounding-level gradients)."""
    T = 2.5
    W, hb, vb = ising.analytic_crbm(1 / T, 2)
    th0 = np.concatenate([W.ravel(), [vb], hb])
    th, _, losses, n = train.pretrain(chain.ISING, 4, T, (1.0,), 2, 2, th0, n_random=10_000, seed=7,
                                      max_epochs=6, order_seed=3)
    assert losses.max() < 1e-4, losses
    assert n < 6                                        # stops once the loss no longer falls
    np.testing.assert_allclose(th, th0, atol=1e-4)


def test_pretraining_stopping_rule_and_kept_parameters():
    """With patience p the run stops p epochs after the last epoch that
    lowered the loss by more than rel_tol (none of them below (1 - rel_tol)
    times it) and returns the parameters of the lowest-loss epoch, which a
    manual replay of the epochs reproduces."""
    K, k, L, T = 1, 2, 4, 3.0
    th0 = wl.init_train_params(K, k, seed=2)
    p, tol = 2, 0.2
    th, st, losses, n = train.pretrain(chain.ISING, L, T, (1.0,), K, k, th0, n_random=400, seed=5,
                                       max_epochs=40, order_seed=8, M=20, patience=p, rel_tol=tol)
    assert n < 40
    j = n - p - 1                                   # the last epoch that lowered the loss by more than tol
    assert losses[j] == losses[:j + 1].min()
    assert all(l >= losses[j] * (1 - tol) for l in losses[j + 1:])
    best = int(np.argmin(losses))
    x = chain.random_init(5, np.arange(400), L)
    t = train.targets_of(chain.ISING, x, 1 / T, (1.0,))
    thr, s = th0.copy(), train.Adam.zeros(len(th0))
    for e in range(best + 1):
        thr, _ = train.epoch(thr, s, x, t, wl.epoch_order(400, 8, e), K, k, 20)
    np.testing.assert_array_equal(th, thr)


def test_algorithm1_starts_lower_after_pretraining():
    """Algorithm 1 from pre-trained parameters starts (and ends) its epochs at
    a lower loss than from the initial parameters (Sec. IV: pre-training
    shortens the training)."""
    K, k, L = 2, 3, 4
    th0 = wl.init_train_params(K, k, seed=1)
    args = dict(n_phys=64, phys_sweeps=20, phys_seed=3, n_train=64, ub=16, g=2, rbm_seed=4, epochs=5,
                order_seed=5, M=20, lr=1e-2)
    _, _, plain = train.algorithm1(chain.ISING, L, 2.5, (1.0,), K, k, th0, **args)
    _, _, pre = train.algorithm1(chain.ISING, L, 2.5, (1.0,), K, k, th0,
                                 pre=dict(n_random=2000, seed=9, max_epochs=20, order_seed=6), **args)
    assert pre[0] < 0.5 * plain[0], (pre, plain)
    assert pre[-1] < plain[-1], (pre, plain)
