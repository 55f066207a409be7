"""Local-update Metropolis baselines (Sec. III and Sec. IV) -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  FP64.

The paper compares the CRBM sampler with local-update Metropolis: single
spin flips for the Ising model (Sec. III) and single gauge-field (eta) flips
for the Kitaev model, run with parallel tempering (Sec. IV).  One *sweep* of
chain c at step t:

* Ising, checkerboard order: the sites with (i + j) even, then those with
  (i + j) odd (even L: no two sites of one colour are neighbours, so each
  colour is updated at once).  Site (i, j) flips with probability
  min(1, e^{-beta dE}), dE = 2 J s_ij sum_nn s, i.e. iff u < e^{-beta dE}.
* Kitaev, sites n = 0 .. N-1 in order: flip eta_n iff
  log u < log pi(eta with eta_n flipped) - log pi(eta).

The uniform of site n is word n % 4 of Philox block n / 4 of tag TAG_LOCAL
at step t (the same site numbering as the Gibbs planes).  After a sweep the
chain's F, log pi, E and observables are those of its new lattice; the
accept counter counts accepted flips.  With ``exchange`` the sweep is
followed by the neighbour temperature exchange of the tempering correction
at cycle counter t (``tempering.exchange_temperatures``).  Then the
observables are added to the sums and the step counter advances.
"""
from __future__ import annotations

import numpy as np

from . import chain, kitaev, philox, tempering

TAG_LOCAL = 0xFFFFFFFB


def _delta_E(s, J):
    """Energy change of flipping each spin: 2 J s_ij (sum of its 4 neighbours)."""
    nn = (np.roll(s, 1, axis=1) + np.roll(s, -1, axis=1) + np.roll(s, 1, axis=2)
          + np.roll(s, -1, axis=2))
    return 2.0 * J * s * nn


def ising_sweep(ch: chain.Chains):
    """One checkerboard sweep; returns (flips per chain, smallest |u - p|)."""
    L = ch.L
    if L % 2:
        raise ValueError("checkerboard Metropolis needs an even L")
    C = len(ch.chain_ids)
    u = philox.uniforms(ch.seed, ch.chain_ids, ch.step, TAG_LOCAL, L * L).reshape(C, L, L)
    ii, jj = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    s = 2.0 * ch.v.astype(np.float64) - 1.0
    flips = np.zeros(C, dtype=np.int64)
    margin = np.full(C, np.inf)
    for colour in (0, 1):
        mask = ((ii + jj) % 2 == colour)[None]
        with np.errstate(over="ignore"):       # e^{+large} = inf: always accepted
            p = np.exp(-ch.beta[:, None, None] * _delta_E(s, ch.J[0]))
        flip = mask & (u < p)
        margin = np.minimum(margin, np.where(mask, np.abs(u - p), np.inf).reshape(C, -1).min(axis=1))
        flips += flip.reshape(C, -1).sum(axis=1)
        s = np.where(flip, -s, s)
    ch.v = (s > 0).astype(np.uint8)
    return flips, margin


def kitaev_sweep(ch: chain.Chains):
    """One sequential single-eta sweep; returns (flips, smallest relative |log u - log r|)."""
    C, L = len(ch.chain_ids), ch.L
    N = L * L
    u = philox.uniforms(ch.seed, ch.chain_ids, ch.step, TAG_LOCAL, N)
    v = ch.v.reshape(C, N).copy()
    lp = ch.logpi.copy()
    flips = np.zeros(C, dtype=np.int64)
    margin = np.full(C, np.inf)
    for n in range(N):
        w = v.copy()
        w[:, n] ^= 1
        lp_new = kitaev.log_weight(w.reshape(C, L, L), ch.beta, ch.J, ch.open_cols)
        log_r = lp_new - lp
        log_u = np.log(u[:, n])
        acc = log_u < log_r
        margin = np.minimum(margin, np.abs(log_u - log_r) / (np.abs(lp_new) + np.abs(lp) + 1.0))
        v = np.where(acc[:, None], w, v)
        lp = np.where(acc, lp_new, lp)
        flips += acc
    ch.v = v.reshape(C, L, L)
    return flips, margin


def sweep(ch: chain.Chains, exchange: bool = False):
    """One sweep (and, with ``exchange``, one temperature exchange) of every
    chain; mutates ``ch``.  Returns per-chain diagnostics."""
    if ch.model == chain.ISING:
        flips, margin = ising_sweep(ch)
    else:
        flips, margin = kitaev_sweep(ch)
    ch.F = ch.free(ch.v)
    ch.logpi, ch.E_phys, ch.obs_terms = ch.targ(ch.v)
    temp = np.zeros(len(ch.chain_ids), dtype=bool)
    temp_margin = np.full(len(ch.chain_ids), np.inf)
    if exchange:
        temp, temp_margin = tempering.exchange_temperatures(ch, int(ch.step))
    ch.obs += ch.obs_terms
    ch.accepts += flips
    ch.step += 1
    return {"flips": flips, "margin": margin, "temp": temp, "temp_margin": temp_margin}


def run(ch: chain.Chains, sweeps: int, exchange: bool = False, record=None):
    """``sweeps`` sweeps; ``record`` (optional) sees (ch, diag) after each."""
    for _ in range(sweeps):
        d = sweep(ch, exchange)
        if record is not None:
            record(ch, d)
    return ch
