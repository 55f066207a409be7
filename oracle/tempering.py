"""Parallel-tempering exchange correction (App. B.2, Fig. 8b) -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  FP64.

Every temperature T_i of a ladder (chains sorted by T) has a physical chain
x_i (target pi_i) and an RBM chain y_i (target P_CRBM ~ e^{-F}).  One cycle:
 1. every RBM chain makes k block-Gibbs steps (uncorrected, Eq. B4);
 2. at every temperature x_i and y_i are exchanged with the probability of
    Eq. (B5) for the pair of distributions (pi_i, P_CRBM):
        log a = [log pi_i(y) - log pi_i(x)] + [F(y) - F(x)];
 3. neighbouring physical chains exchange states with Eq. (B5) for the pair
    (pi_i, pi_j):  log b = log pi_i(x_j) + log pi_j(x_i) - log pi_i(x_i) - log pi_j(x_j),
    pairing (0,1), (2,3), ... on even cycles and (1,2), (3,4), ... on odd ones;
 4. the observables of the physical chains are accumulated.
Uniforms: acceptance of step 2 from tag TAG_SWAP of the physical chain (step =
cycle counter = the physical chains' step); of step 3 from tag TAG_TEMP of the lower chain of the pair.  The
oracle evaluates the log-weight of a state at another temperature afresh; it
depends on the state only through its single-fermion energies eps (Kitaev) or
its energy E (Ising), so a fast path may reuse those.
"""
from __future__ import annotations

import numpy as np

from . import chain, philox

TAG_SWAP = 0xFFFFFFFD
TAG_TEMP = 0xFFFFFFFC


def _log_weight_at(ch, v, beta):
    """log pi_beta of lattices v (one beta per lattice) under ch's physics."""
    return ch.targ(v, beta)[0]


def exchange_temperatures(phys: chain.Chains, c: int):
    """Neighbouring chains (i, i+1), i = c % 2, c % 2 + 2, ... exchange their
    lattices with the Eq. (B5) probability for the pair (pi_i, pi_{i+1});
    uniform from tag TAG_TEMP of chain i at step c.  Returns the per-chain
    decision (set at the lower chain of an accepted pair) and margin."""
    n = len(phys.chain_ids)
    i = np.arange(c % 2, n - 1, 2)
    j = i + 1
    temp = np.zeros(n, dtype=bool)
    temp_margin = np.full(n, np.inf)
    if len(i):
        beta = phys.beta
        lp_ij = _log_weight_at(phys, phys.v[j], beta[i])   # log pi_i(x_j)
        lp_ji = _log_weight_at(phys, phys.v[i], beta[j])   # log pi_j(x_i)
        log_b = lp_ij + lp_ji - phys.logpi[i] - phys.logpi[j]
        ub = philox.uniforms(phys.seed, phys.chain_ids[i], c, TAG_TEMP, 1)[:, 0]
        acc = np.log(ub) < log_b
        temp_margin[i] = np.abs(np.log(ub) - log_b) / (
            np.abs(lp_ij) + np.abs(lp_ji) + np.abs(phys.logpi[i]) + np.abs(phys.logpi[j]) + 1.0)
        temp[i[acc]] = True
        ii, jj = i[acc], j[acc]
        v_i, v_j = phys.v[ii].copy(), phys.v[jj].copy()
        F_i, F_j = phys.F[ii].copy(), phys.F[jj].copy()
        phys.v[ii], phys.v[jj] = v_j, v_i
        phys.F[ii], phys.F[jj] = F_j, F_i
        # log pi, E and observables of the moved states at their new temperatures
        for idx in (ii, jj):
            if len(idx):
                lp, E, ot = phys.targ(phys.v[idx], phys.beta[idx])
                phys.logpi[idx], phys.E_phys[idx], phys.obs_terms[idx] = lp, E, ot
    return temp, temp_margin


def cycle(phys: chain.Chains, rbm: chain.Chains, k: int):
    """One PT-exchange-correction cycle; mutates both chain sets.  The cycle
    counter is the physical chains' step counter.  Returns the swap and
    temperature-exchange decisions and how close each came to its threshold."""
    c = int(phys.step)
    # 1. RBM chains: k Gibbs steps from their own states, then the FP64 values
    #    the exchange needs (no correction, no observables of their own)
    y, bmargin = chain.propose(rbm, k)
    rbm.v = y
    rbm.F = rbm.free(y)
    rbm.logpi, rbm.E_phys, rbm.obs_terms = rbm.targ(y)
    rbm.step += 1
    # 2. physical <-> RBM exchange at every temperature
    log_a = (rbm.logpi - phys.logpi) + (rbm.F - phys.F)
    u = philox.uniforms(phys.seed, phys.chain_ids, c, TAG_SWAP, 1)[:, 0]
    swap = np.log(u) < log_a
    swap_margin = np.abs(np.log(u) - log_a) / (
        np.abs(rbm.logpi) + np.abs(phys.logpi) + np.abs(rbm.F) + np.abs(phys.F) + 1.0)
    for name in ("v", "F", "logpi", "E_phys", "obs_terms"):
        a, b = getattr(phys, name), getattr(rbm, name)
        m = swap.reshape((-1,) + (1,) * (a.ndim - 1))
        a_new, b_new = np.where(m, b, a), np.where(m, a, b)
        setattr(phys, name, a_new)
        setattr(rbm, name, b_new)
    # 3. temperature exchange between neighbours
    temp, temp_margin = exchange_temperatures(phys, c)
    # 4. observables of the physical chains
    phys.obs += phys.obs_terms
    phys.accepts += swap
    phys.step += 1
    return {"swap": swap, "temp": temp, "bernoulli_margin": bmargin,
            "swap_margin": swap_margin, "temp_margin": temp_margin}


def run(phys, rbm, k, cycles, record=None):
    """``cycles`` PT cycles; ``record`` (optional) sees the diagnostics of each."""
    for _ in range(cycles):
        d = cycle(phys, rbm, k)
        if record is not None:
            record(d)
    return phys, rbm
