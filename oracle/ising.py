"""2D Ising model on an L x L torus: energy, magnetisation, exact references.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Energy (Sec. III, Eq. 14): E(s) = -J sum_<ij> s_i s_j with s = 2v - 1 (App. A:
the RBM's 0/1 units map to spins +-1).  The paper's "ferromagnetic, J < 0"
contradicts its own E = -J sum s s and App. C (aligned pairs carry log-weight
+beta); the reading used here is J = +1 ferromagnetic.  The bond set is the
2 L^2 pairs (i,j)-(i+1,j) and (i,j)-(i,j+1) taken mod L, so at L = 2 each pair
is counted twice.  Target log-weight: log pi(s) = -beta E(s).
"""
from __future__ import annotations

import itertools

import numpy as np


def spins(v):
    return 2.0 * np.asarray(v, dtype=np.float64) - 1.0


def energy(v, J: float = 1.0):
    """E = -J sum_{i,j} s_ij (s_{i+1,j} + s_{i,j+1}) per chain; v is (C, L, L) 0/1."""
    s = spins(v)
    right = np.roll(s, -1, axis=2)
    down = np.roll(s, -1, axis=1)
    return -J * (s * (right + down)).sum(axis=(1, 2))


def magnetisation(v):
    """M = sum_ij s_ij per chain."""
    return spins(v).sum(axis=(1, 2))


def log_weight(v, beta, J: float = 1.0):
    """log pi(v) = -beta E(v)."""
    return -np.asarray(beta, dtype=np.float64) * energy(v, J)


def analytic_crbm(beta: float, k: int = 2):
    """App. C closed-form CRBM whose marginal equals the Ising distribution.

    Kernels W^1 = [[W,0],[W,0]] (vertical bond), W^2 = [[W,W],[0,0]]
    (horizontal bond), zero-padded to k x k; W = W_min of Eq. (C7), h_bias = -W,
    v_bias = -2W (Eq. C8).  Then F(v) - beta E(s) is the same for every v.
    """
    x = np.exp(2.0 * beta)
    W = np.log(2.0 * x * (np.sqrt(x * x - 1.0) + x) - 1.0)   # Eq. (C7)
    K = np.zeros((2, k, k))
    K[0, 0, 0] = K[0, 1, 0] = W
    K[1, 0, 0] = K[1, 0, 1] = W
    return K, np.array([-W, -W]), -2.0 * W


def all_states(L: int) -> np.ndarray:
    """Every lattice of an L x L torus, (2^(L*L), L, L) uint8 (use for L*L <= 20)."""
    N = L * L
    n = np.arange(2 ** N, dtype=np.int64)
    return ((n[:, None] >> np.arange(N)) & 1).astype(np.uint8).reshape(-1, L, L)


def enumerate_exact(L: int, beta: float, J: float = 1.0):
    """Exact <E>, <E^2>, <|M|>, <M^2> and log Z by summing every state (tiny L only)."""
    v = all_states(L)
    E = energy(v, J)
    M = magnetisation(v)
    lw = -beta * E
    m = lw.max()
    w = np.exp(lw - m)
    Z = w.sum()
    p = w / Z
    return {"logZ": m + np.log(Z), "E": (p * E).sum(), "E2": (p * E * E).sum(),
            "absM": (p * np.abs(M)).sum(), "M2": (p * M * M).sum()}


def kaufman_logZ(L: int, beta, J: float = 1.0):
    """Kaufman's (1949) exact partition function of the L x L periodic Ising model.

    Z = 1/2 (2 sinh 2K)^{N/2} (Z1 + Z2 + Z3 + Z4), K = beta J, with
    Z1 = prod_r 2cosh(L g_{2r+1}/2), Z2 = prod_r 2sinh(L g_{2r+1}/2),
    Z3 = prod_r 2cosh(L g_{2r}/2),   Z4 = prod_r 2sinh(L g_{2r}/2),  r = 0..L-1,
    cosh g_l = cosh 2K coth 2K - cos(pi l / L) for l >= 1 and g_0 = 2K + ln tanh K.
    Evaluated with mpmath at the caller's working precision (40 digits from
    ``kaufman_moments``); ``beta`` may be an mpmath number.
    """
    import mpmath as mp
    K = mp.mpf(beta) * J
    c = mp.cosh(2 * K) * mp.coth(2 * K)

    def g(l):
        if l == 0:
            return 2 * K + mp.log(mp.tanh(K))
        return mp.acosh(c - mp.cos(mp.pi * l / L))

    odd = [g(2 * r + 1) for r in range(L)]
    even = [g(2 * r) for r in range(L)]
    Z1 = mp.fprod(2 * mp.cosh(L * x / 2) for x in odd)
    Z2 = mp.fprod(2 * mp.sinh(L * x / 2) for x in odd)
    Z3 = mp.fprod(2 * mp.cosh(L * x / 2) for x in even)
    Z4 = mp.fprod(2 * mp.sinh(L * x / 2) for x in even)
    return mp.log(mp.mpf(1) / 2) + (L * L) * mp.log(2 * mp.sinh(2 * K)) / 2 + mp.log(Z1 + Z2 + Z3 + Z4)


def kaufman_moments(L: int, beta: float, J: float = 1.0):
    """Exact <E> = -d lnZ/d beta and C = beta^2 d^2 lnZ/d beta^2 (= beta^2 Var E)."""
    import mpmath as mp
    with mp.workdps(40):
        f = lambda b: kaufman_logZ(L, b, J)
        d1 = mp.diff(f, mp.mpf(beta), 1)
        d2 = mp.diff(f, mp.mpf(beta), 2)
        return {"logZ": float(f(mp.mpf(beta))), "E": float(-d1), "varE": float(d2),
                "C": float(mp.mpf(beta) ** 2 * d2)}
