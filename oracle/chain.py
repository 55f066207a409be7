"""CRBM proposal + exact Metropolis-Hastings correction over many chains.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  FP64, vectorised over
chains, no blocking or reordering beyond the definitions below.

One proposal for chain c at step t (the method of App. B, run as an in-place
Metropolis-Hastings chain):
 1. g block-Gibbs steps v -> h -> v' (Eq. B4), every Bernoulli draw taken as
    [u < sigma(x)] with the Philox uniforms of ``oracle.philox``.
 2. F(v') by Eq. (13); log pi(v') by Eq. (14) (Ising: -beta E) or by the
    Kitaev log-weight of Sec. IV.
 3. The Gibbs kernel is reversible with respect to P_CRBM ~ e^{-F} (App. B.1:
    it satisfies detailed balance), so its proposal ratio is
    T(v'->v)/T(v->v') = e^{F(v') - F(v)}.  The acceptance of Eq. (B5) with the
    pair (pi, P_CRBM) in place of two tempered distributions is therefore
    log r = [log pi(v') - log pi(v)] + [F(v') - F(v)],
    accept iff log u_acc < log r.  On rejection v, F(v), log pi(v) are kept.
    ``correct=False`` accepts every proposal (the uncorrected Gibbs sampling
    the paper uses for its Ising runs, Sec. III).
 4. Observables of the state after the decision are added to per-chain sums:
    Ising (E, E^2, |M|, M^2); Kitaev (e, e^2, c_f, vison density).
The step counter advances whether or not the proposal is accepted.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import crbm, ising, kitaev, lcrbm, philox

ISING = 0
KITAEV = 1
NOBS = 4


@dataclass
class Chains:
    model: int
    W: np.ndarray
    hb: np.ndarray
    vb: float
    L: int
    T: np.ndarray                 # (C,)
    J: tuple                      # Ising: (J,), Kitaev: (Jx, Jy, Jz)
    seed: int
    chain_ids: np.ndarray         # (C,) uint64
    v: np.ndarray                 # (C, L, L) uint8
    step: int = 0
    F: np.ndarray = None
    logpi: np.ndarray = None
    E_phys: np.ndarray = None
    obs: np.ndarray = None        # (C, NOBS) running sums
    obs_terms: np.ndarray = None  # (C, NOBS) observables of the current lattices
    accepts: np.ndarray = None    # (C,)
    extras: dict = field(default_factory=dict)
    edge: int = 0                 # > 0: LCRBM with `edge` unshared kernels per side, open columns

    @property
    def beta(self):
        return 1.0 / self.T

    @property
    def open_cols(self):
        return self.edge > 0

    # the model's free energy and conditionals: periodic CRBM or, with edge > 0, LCRBM
    def free(self, v):
        if self.edge:
            return lcrbm.free_energy(v, self.W, self.hb, self.vb, self.edge)
        return crbm.free_energy(v, self.W, self.hb, self.vb)

    def hpre(self, v):
        if self.edge:
            return lcrbm.hidden_preact(v, self.W, self.hb, self.edge)
        return crbm.hidden_preact(v, self.W, self.hb)

    def vpre(self, h):
        if self.edge:
            return lcrbm.visible_preact(h, self.W, self.vb, self.edge)
        return crbm.visible_preact(h, self.W, self.vb)

    def targ(self, v, beta=None):
        return target(self.model, v, self.beta if beta is None else beta, self.J, self.open_cols)

    @property
    def K(self):
        return self.W.shape[-3]


def random_init(seed: int, chain_ids, L: int) -> np.ndarray:
    """v_ij = [u < 1/2] with the TAG_INIT uniforms at step 0."""
    w = philox.words(seed, chain_ids, 0, philox.TAG_INIT, L * L)
    return (w < np.uint32(2 ** 31)).astype(np.uint8).reshape(len(chain_ids), L, L)


def target(model: int, v, beta, J, open_cols=False):
    """(log pi, E_phys, obs-terms) of each chain's lattice (open_cols: the
    Kitaev lattice is open along j, see ``kitaev.hopping_matrix``)."""
    if model == ISING:
        E = ising.energy(v, J[0])
        M = ising.magnetisation(v)
        return -beta * E, E, np.stack([E, E * E, np.abs(M), M * M], axis=1)
    eps = kitaev.energies(v, J, open_cols)
    lp = kitaev.log_weight_from_eps(eps, beta)
    e, cf = kitaev.thermal_terms(eps, beta)
    return lp, e, np.stack([e, e * e, cf, kitaev.vison_density(v, open_cols)], axis=1)


def make_chains(model, W, hb, vb, L, T, J, seed, chain_ids, v0=None, edge=0) -> Chains:
    chain_ids = np.asarray(chain_ids, dtype=np.uint64)
    T = np.broadcast_to(np.asarray(T, dtype=np.float64), (len(chain_ids),)).copy()
    if v0 is None:
        v0 = random_init(seed, chain_ids, L)
    ch = Chains(model, np.asarray(W, dtype=np.float64), np.asarray(hb, dtype=np.float64),
                float(vb), L, T, tuple(float(x) for x in J), seed, chain_ids,
                np.asarray(v0, dtype=np.uint8).copy(), edge=int(edge))
    ch.F = ch.free(ch.v)
    ch.logpi, ch.E_phys, ch.obs_terms = ch.targ(ch.v)
    ch.obs = np.zeros((len(chain_ids), NOBS))
    ch.accepts = np.zeros(len(chain_ids), dtype=np.int64)
    return ch


def propose(ch: Chains, g: int = 1):
    """g Gibbs steps from the current lattices at the current step counter.

    Returns (v', bernoulli_margin) where the margin is, per chain, the smallest
    |u - sigma(x)| over every Bernoulli draw of the proposal (how close any
    draw came to flipping).
    """
    C, L, K, N = len(ch.chain_ids), ch.L, ch.K, ch.L * ch.L
    v = ch.v
    margin = np.full(C, np.inf)
    for s in range(g):
        u_h = np.stack([philox.uniforms(ch.seed, ch.chain_ids, ch.step, philox.hidden_tag(s, K, kk), N)
                        for kk in range(K)], axis=1).reshape(C, K, L, L)
        u_v = philox.uniforms(ch.seed, ch.chain_ids, ch.step, philox.visible_tag(s, K), N).reshape(C, L, L)
        p_h = crbm.sigmoid(ch.hpre(v))
        h = (u_h < p_h).astype(np.uint8)
        p_v = crbm.sigmoid(ch.vpre(h))
        v = (u_v < p_v).astype(np.uint8)
        margin = np.minimum(margin, np.abs(u_h - p_h).reshape(C, -1).min(axis=1))
        margin = np.minimum(margin, np.abs(u_v - p_v).reshape(C, -1).min(axis=1))
    return v, margin


def step(ch: Chains, g: int = 1, correct: bool = True):
    """One proposal + MH decision for every chain; mutates ``ch``.

    Returns a dict of per-chain diagnostics: accepted, log_r, log_u,
    bernoulli_margin and the MH margin |log u - log r|.
    """
    v_new, bmargin = propose(ch, g)
    F_new = ch.free(v_new)
    lp_new, E_new, obs_new = ch.targ(v_new)
    log_r = (lp_new - ch.logpi) + (F_new - ch.F)
    scale = np.abs(lp_new) + np.abs(ch.logpi) + np.abs(F_new) + np.abs(ch.F) + 1.0
    u_acc = philox.uniforms(ch.seed, ch.chain_ids, ch.step, philox.TAG_ACC, 1)[:, 0]
    log_u = np.log(u_acc)
    acc = (log_u < log_r) if correct else np.ones(len(ch.chain_ids), dtype=bool)
    ch.v = np.where(acc[:, None, None], v_new, ch.v)
    ch.F = np.where(acc, F_new, ch.F)
    ch.logpi = np.where(acc, lp_new, ch.logpi)
    ch.E_phys = np.where(acc, E_new, ch.E_phys)
    ch.obs_terms = np.where(acc[:, None], obs_new, ch.obs_terms)
    ch.obs += ch.obs_terms
    ch.accepts += acc
    ch.step += 1
    return {"accepted": acc, "log_r": log_r, "log_u": log_u, "bernoulli_margin": bmargin,
            "mh_margin": np.abs(log_u - log_r), "mh_scale": scale}


def run(ch: Chains, S: int, g: int = 1, correct: bool = True, record=None):
    """S proposals; ``record`` (optional callable) sees (ch, diag) after each step."""
    for _ in range(S):
        d = step(ch, g, correct)
        if record is not None:
            record(ch, d)
    return ch
