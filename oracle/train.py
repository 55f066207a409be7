"""The paper's CRBM trainer (Sec. II, App. A, Algorithm 1) -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  FP64.

Parameters theta = [W (K*k*k, row-major W[f][a][b]), v_bias, h_bias (K)]
(the order of Algorithm 1's ``param``).  For samples x_i with targets
t_i = beta E_phys(x_i) (for the Kitaev model -log pi(x_i), the log-weight of
the gauge configuration) the loss of a minibatch of M samples is

    diff_i = t_i - F(x_i; theta),   C = (1/M) sum_i diff_i,
    loss = (1/M) sum_i (diff_i - C)^2                    (Sec. II; App. A)

with F the CRBM free energy of Eq. (13).  Since sum_i (diff_i - C) = 0 the
dependence of C on theta drops out of the gradient:

    d loss / d theta = -(2/M) sum_i (diff_i - C) dF(x_i)/d theta,
    dF/dv_bias = -sum_ij v_ij,   dF/dh_bias^f = -sum_ij sigma(a^f_ij),
    dF/dW^f_ab = -sum_ij sigma(a^f_ij) v_(i+a)(j+b),

a^f the hidden pre-activations of Eq. (12).  ADAM (Kingma & Ba 2014):
m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2, theta <- theta - lr m^ / (sqrt(v^) + eps),
m^ = m / (1 - b1^t), v^ = v / (1 - b2^t), t the number of steps taken.
An epoch visits its samples in a given order, in consecutive minibatches of M
(the last one holds the remainder), one ADAM step per minibatch.

``algorithm1`` is the outer loop of Algorithm 1: physical samples from local
Metropolis chains, a buffer of RBM samples refreshed by g uncorrected Gibbs
steps of ub chains per epoch (new samples in front, the buffer cut to n_train),
and one epoch over buffer + physical samples after each refresh.

``pretrain`` is the pre-training step (App. A; Sec. IV; App. D): the same
loss and ADAM epochs on uniformly random lattices, whose targets are computed
once, until the epoch loss no longer decreases.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import crbm_workloads as wl

from . import chain, crbm, metropolis


def split(theta, K, k):
    W = np.asarray(theta[:K * k * k], dtype=np.float64).reshape(K, k, k)
    return W, np.asarray(theta[K * k * k + 1:], dtype=np.float64), float(theta[K * k * k])


def free_energy_grad(v, theta, K, k):
    """F(v) (Eq. 13) and dF/dtheta for every lattice of v (C, L, L)."""
    W, hb, vb = split(theta, K, k)
    v = np.asarray(v)
    C = v.shape[0]
    a = crbm.hidden_preact(v, W, hb)                 # (C, K, L, L)
    s = crbm.sigmoid(a)
    F = crbm.free_energy(v, W, hb, vb)
    vf = v.astype(np.float64)
    dW = np.empty((C, K, k, k))
    for p in range(k):
        for q in range(k):
            shifted = np.roll(vf, (-p, -q), axis=(1, 2))    # shifted[i, j] = v[(i+p)%L, (j+q)%L]
            dW[:, :, p, q] = -(s * shifted[:, None]).sum(axis=(2, 3))
    dvb = -vf.sum(axis=(1, 2))
    dhb = -s.sum(axis=(2, 3))
    return F, np.concatenate([dW.reshape(C, -1), dvb[:, None], dhb], axis=1)


def loss_and_grad(v, targets, theta, K, k):
    F, G = free_energy_grad(v, theta, K, k)
    diff = np.asarray(targets, dtype=np.float64) - F
    C = diff.mean()
    loss = ((diff - C) ** 2).mean()
    grad = -(2.0 / len(diff)) * ((diff - C)[:, None] * G).sum(axis=0)
    return loss, grad


@dataclass
class Adam:
    m: np.ndarray
    v: np.ndarray
    t: int = 0

    @classmethod
    def zeros(cls, P):
        return cls(np.zeros(P), np.zeros(P), 0)


def adam_step(theta, g, st: Adam, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    st.t += 1
    st.m = b1 * st.m + (1.0 - b1) * g
    st.v = b2 * st.v + (1.0 - b2) * g * g
    mh = st.m / (1.0 - b1 ** st.t)
    vh = st.v / (1.0 - b2 ** st.t)
    return theta - lr * mh / (np.sqrt(vh) + eps)


def epoch(theta, st: Adam, samples, targets, order, K, k, M=20, **adam):
    """One epoch; returns (theta, losses of its minibatches)."""
    theta = np.asarray(theta, dtype=np.float64).copy()
    losses = []
    for b in range(0, len(order), M):
        idx = order[b:b + M]
        loss, g = loss_and_grad(samples[idx], targets[idx], theta, K, k)
        losses.append(loss)
        theta = adam_step(theta, g, st, **adam)
    return theta, np.array(losses)


def targets_of(model, v, beta, J):
    """t = -log pi(v): beta E for the Ising model, the negative Majorana
    log-weight for the Kitaev model."""
    return -chain.target(model, v, np.broadcast_to(beta, (len(v),)), J)[0]


def algorithm1(model, L, T, J, K, k, theta0, n_phys, phys_sweeps, phys_seed, n_train, ub, g,
               rbm_seed, epochs, order_seed, M=20, pre=None, **adam):
    """Algorithm 1 at one temperature; returns (theta, adam state, per-epoch losses).

    Physical samples: the final lattices of n_phys local-Metropolis chains
    (``oracle.metropolis``, seed phys_seed, chain ids 0..n_phys-1) after
    phys_sweeps sweeps from random lattices.  Buffer chains: ub chains (seed
    rbm_seed, ids 0..ub-1) from random lattices; each refresh is one
    uncorrected proposal of g Gibbs steps with the current parameters.
    pre: keyword arguments of ``pretrain`` (n_random, seed, max_epochs,
    order_seed and optionally patience, rel_tol): the pre-training step runs
    first, from theta0, and the main loop starts from its parameters with a
    fresh ADAM state (reading: the paper treats the two as separate steps).
    """
    if pre is not None:
        theta0 = pretrain(model, L, T, J, K, k, theta0, M=M, **pre, **adam)[0]
    beta = 1.0 / T
    zeroW, zh = np.zeros((K, k, k)), np.zeros(K)
    phys = chain.make_chains(model, zeroW, zh, 0.0, L, T, J, phys_seed, np.arange(n_phys))
    metropolis.run(phys, phys_sweeps)
    x_phys = phys.v.copy()
    t_phys = targets_of(model, x_phys, beta, J)
    theta = np.asarray(theta0, dtype=np.float64).copy()
    W, hb, vb = split(theta, K, k)
    buf = chain.make_chains(model, W, hb, vb, L, T, J, rbm_seed, np.arange(ub))
    x_rbm = np.zeros((0, L, L), dtype=np.uint8)

    def refresh():
        nonlocal x_rbm
        buf.W, buf.hb, buf.vb = split(theta, K, k)
        y, _ = chain.propose(buf, g)
        buf.v = y
        buf.step += 1
        x_rbm = np.concatenate([y, x_rbm])[:n_train]

    while len(x_rbm) < n_train:
        refresh()
    st = Adam.zeros(len(theta))
    losses = []
    for e in range(epochs):
        refresh()
        x_tot = np.concatenate([x_rbm, x_phys])
        t_tot = np.concatenate([targets_of(model, x_rbm, beta, J), t_phys])
        theta, ls = epoch(theta, st, x_tot, t_tot, wl.epoch_order(len(x_tot), order_seed, e), K, k, M, **adam)
        losses.append(ls.mean())
    return theta, st, np.array(losses)


def pretrain(model, L, T, J, K, k, theta0, n_random, seed, max_epochs, order_seed, M=20, patience=1,
             rel_tol=1e-4, **adam):
    """Pre-training on random states (App. A; Sec. IV; App. D), at one temperature.

    The n_random lattices are uniform: v_ij = [u < 1/2] from the init tag of
    chains 0 .. n_random-1 of `seed` (``chain.random_init``); their targets
    t = -log pi at T are computed once.  Epochs of minibatch ADAM steps
    (``epoch``, visiting order ``wl.epoch_order(n_random, order_seed, e)``)
    run until for `patience` consecutive epochs the epoch's loss -- the mean
    of its minibatch losses -- has not fallen below (1 - rel_tol) times the
    loss of the last epoch that did, or max_epochs have run.  Reading: the paper ends the
    step once the loss stops falling, without a tolerance; the parameters kept
    are those of the epoch with the lowest loss, the ADAM state the one after
    the last epoch.
    Returns (theta, adam state, epoch losses, epochs run).
    """
    x = chain.random_init(seed, np.arange(n_random), L)
    t = targets_of(model, x, 1.0 / T, J)
    theta = np.asarray(theta0, dtype=np.float64).copy()
    st = Adam.zeros(len(theta))
    best, best_theta = np.inf, theta.copy()       # lowest epoch loss and its parameters
    level, stale, losses = np.inf, 0, []          # loss at the last decrease by more than rel_tol
    for e in range(max_epochs):
        theta, ls = epoch(theta, st, x, t, wl.epoch_order(n_random, order_seed, e), K, k, M, **adam)
        loss = float(ls.mean())
        losses.append(loss)
        if loss < best:
            best, best_theta = loss, theta.copy()
        if loss < level * (1.0 - rel_tol):
            level, stale = loss, 0
        else:
            stale += 1
            if stale >= patience:
                break
    return best_theta, st, np.array(losses), len(losses)
