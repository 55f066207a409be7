"""Parity of the CUDA trainer (crbm_train_epochs, trainer.algorithm1) with the
oracle's (Sec. II, App. A, Algorithm 1).

FP64 on both sides with different summation orders: parameters, ADAM moments
and minibatch losses agree to 1e-9 relative after whole epochs; the ADAM step
counter exactly.  Algorithm 1 adds sampling (Metropolis physical samples,
Gibbs buffer) whose lattices are bit-exact between the two sides.
"""
import numpy as np
import pytest

import crbm_workloads as wl
from _common import gpu_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


PROBLEMS = [
    # K, k, L, n_samples
    (2, 2, 3, 512),      # the paper's Ising protocol size (all states of L = 3)
    (2, 5, 8, 97),       # the paper's Kitaev kernel shape 2x5x5 at L = 8, ragged last batch
    (4, 3, 16, 45),
]


def test_epochs_match_oracle(ctx):
    import torch
    from oracle import ising, train
    from paper_2008_05401_gb300 import trainer
    batch, epochs = 20, 2
    probs, ref, data = [], [], []
    for j, (K, k, L, n) in enumerate(PROBLEMS):
        v = ising.all_states(L) if n == 2 ** (L * L) else wl.random_lattices(n, L, seed=j + 1)
        t = ising.energy(v) / 2.2
        th0 = wl.init_train_params(K, k, seed=j + 7)
        probs.append(trainer.Problem.new(ctx, K, k, L, th0))
        ref.append([th0.copy(), train.Adam.zeros(len(th0)), []])
        data.append((v, t))
    for e in range(epochs):
        xs, ts, os_ = [], [], []
        for j, (v, t) in enumerate(data):
            order = wl.epoch_order(len(t), 3, e)
            xs.append(torch.tensor(wl.pack_bits(v).view(np.int32), device="cuda:0"))
            ts.append(torch.tensor(t, device="cuda:0"))
            os_.append(torch.tensor(order, device="cuda:0"))
            K, k, _, _ = PROBLEMS[j]
            th, ls = train.epoch(ref[j][0], ref[j][1], v, t, order, K, k, M=batch)
            ref[j][0] = th
            ref[j][2].append(ls)
        losses = trainer.train_epochs(ctx, probs, xs, ts, os_, batch)
        for j in range(len(PROBLEMS)):
            np.testing.assert_allclose(losses[j].cpu().numpy(), ref[j][2][-1], rtol=1e-9, atol=1e-12)
    for j, pr in enumerate(probs):
        np.testing.assert_allclose(pr.theta.cpu().numpy(), ref[j][0], rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(pr.m.cpu().numpy(), ref[j][1].m, rtol=1e-9, atol=1e-14)
        np.testing.assert_allclose(pr.v.cpu().numpy(), ref[j][1].v, rtol=1e-9, atol=1e-18)
        assert int(pr.t.item()) == ref[j][1].t


@pytest.mark.parametrize("model", ["ising", "kitaev"])
def test_algorithm1_matches_oracle(ctx, model):
    from oracle import chain, train
    from paper_2008_05401_gb300 import ISING, KITAEV, trainer
    if model == "ising":
        kind, okind, L, Ts, J, K, k = ISING, chain.ISING, 4, [2.2, 3.0], (1.0,), 2, 3
    else:
        kind, okind, L, Ts, J, K, k = KITAEV, chain.KITAEV, 3, [0.3], (1.0, 1.0, 1.0), 2, 2
    th0 = wl.init_train_params(K, k, seed=11)
    kw = dict(n_phys=24, phys_sweeps=6, phys_seed=5, n_train=30, ub=10, g=2, rbm_seed=6, epochs=3, M=8, lr=1e-2)
    probs, hist = trainer.algorithm1(ctx, kind, L, Ts, J, K, k, th0, order_fn=lambda n, e: wl.epoch_order(n, 4, e),
                                     **kw)
    for i, T in enumerate(Ts):
        th, st, losses = train.algorithm1(okind, L, T, J, K, k, th0, order_seed=4, **kw)
        np.testing.assert_allclose(probs[i].theta.cpu().numpy(), th, rtol=1e-8, atol=1e-11)
        np.testing.assert_allclose(hist[:, i], losses, rtol=1e-8, atol=1e-11)
        assert int(probs[i].t.item()) == st.t


@pytest.mark.parametrize("model", ["ising", "kitaev"])
def test_pretraining_matches_oracle(ctx, model):
    """Pre-training on random states (App. A; Sec. IV; App. D): the random
    lattices drawn on the device, their targets, the epochs and the stopping
    rule give the oracle's epoch losses, stopping epoch and kept parameters at
    every temperature."""
    from oracle import chain, train
    from paper_2008_05401_gb300 import ISING, KITAEV, trainer
    if model == "ising":
        kind, okind, L, Ts, J, K, k = ISING, chain.ISING, 6, [2.0, 2.5, 3.2], (1.0,), 2, 3
    else:
        kind, okind, L, Ts, J, K, k = KITAEV, chain.KITAEV, 4, [0.1, 0.5], (1.0, 1.0, 1.0), 2, 3
    th0 = wl.init_train_params(K, k, seed=13)
    kw = dict(n_random=1500, seed=21, max_epochs=12, M=20, patience=2, rel_tol=0.02)
    probs, hist = trainer.pretrain(ctx, kind, L, Ts, J, K, k, th0, order_fn=lambda n, e: wl.epoch_order(n, 6, e),
                                   **kw)
    stopped_early = 0
    for i, T in enumerate(Ts):
        th, st, losses, n = train.pretrain(okind, L, T, J, K, k, th0, order_seed=6, **kw)
        assert len(hist[i]) == n
        stopped_early += n < kw["max_epochs"]
        np.testing.assert_allclose(hist[i], losses, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(probs[i].theta.cpu().numpy(), th, rtol=1e-9, atol=1e-12)
        assert losses.min() < losses[0]
    if model == "ising":
        assert stopped_early >= 1                    # the stopping rule itself is exercised


def test_algorithm1_with_pretraining_matches_oracle(ctx):
    from oracle import chain, train
    from paper_2008_05401_gb300 import ISING, trainer
    L, Ts, J, K, k = 4, [2.2, 3.0], (1.0,), 2, 3
    th0 = wl.init_train_params(K, k, seed=11)
    kw = dict(n_phys=24, phys_sweeps=6, phys_seed=5, n_train=30, ub=10, g=2, rbm_seed=6, epochs=3, M=8, lr=1e-2)
    probs, hist = trainer.algorithm1(ctx, ISING, L, Ts, J, K, k, th0, order_fn=lambda n, e: wl.epoch_order(n, 4, e),
                                     pre=dict(n_random=400, seed=31, max_epochs=6,
                                              order_fn=lambda n, e: wl.epoch_order(n, 8, e)), **kw)
    for i, T in enumerate(Ts):
        th, st, losses = train.algorithm1(chain.ISING, L, T, J, K, k, th0, order_seed=4,
                                          pre=dict(n_random=400, seed=31, max_epochs=6, order_seed=8), **kw)
        np.testing.assert_allclose(probs[i].theta.cpu().numpy(), th, rtol=1e-8, atol=1e-11)
        np.testing.assert_allclose(hist[:, i], losses, rtol=1e-8, atol=1e-11)


def test_train_rejects_bad_shapes(ctx):
    import torch
    from paper_2008_05401_gb300 import CrbmError, trainer
    pr = trainer.Problem.new(ctx, 2, 3, 40, wl.init_train_params(2, 3))      # L = 40 > 32
    x = torch.zeros((4, 50), dtype=torch.int32, device="cuda:0")
    t = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    o = torch.arange(4, dtype=torch.int32, device="cuda:0")
    with pytest.raises(CrbmError):
        trainer.train_epochs(ctx, [pr], [x], [t], [o])
