"""Convolutional RBM: energy, free energy, conditionals and one block-Gibbs step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  FP64 throughout.

Reading of the paper's "wrap around convolution" (Sec. II, text after Eq. 12):
a periodic cross-correlation anchored at the top-left tap,

    (W^k * v)_{ij} = sum_{a,b=0}^{k-1} W^k_{ab} v_{(i+a) mod L, (j+b) mod L}.

Visible units v_{ij} in {0,1} (App. A), K hidden planes h^k_{ij} in {0,1},
one visible bias and K hidden biases (Sec. II, Eq. 12 and Fig. 2 caption).
All arrays carry a leading chain axis: v is (C, L, L), h is (C, K, L, L).
"""
from __future__ import annotations

import numpy as np


def sigmoid(x):
    """sigma(x) = 1 / (1 + e^-x) (App. B, Eq. B2)."""
    with np.errstate(over="ignore"):
        return 1.0 / (1.0 + np.exp(-x))


def softplus(x):
    """log(1 + e^x), written as max(x,0) + log1p(e^-|x|) so it never overflows."""
    return np.maximum(x, 0.0) + np.log1p(np.exp(-np.abs(x)))


def hidden_preact(v, W, hb):
    """a^k_{ij} = h_bias^k + (W^k * v)_{ij}  -- the argument of Eq. (B2) in CRBM form.

    v: (C, L, L) 0/1; W: (K, k, k); hb: (K,).  Returns (C, K, L, L).
    """
    v = np.asarray(v, dtype=np.float64)
    K, k, _ = W.shape
    C, L, _ = v.shape
    a = np.empty((C, K, L, L))
    a[:] = np.asarray(hb, dtype=np.float64)[None, :, None, None]
    for da in range(k):
        for db in range(k):
            # shifted[c, i, j] = v[c, (i+da) % L, (j+db) % L]
            shifted = np.roll(v, shift=(-da, -db), axis=(1, 2))
            a += W[None, :, da, db, None, None] * shifted[:, None, :, :]
    return a


def visible_preact(h, W, vb):
    """b_{ij} = v_bias + sum_k sum_{a,b} W^k_{ab} h^k_{(i-a) mod L, (j-b) mod L}  (Eq. B3).

    The coefficient of v_{ij} in the joint energy (Eq. 12) collects every hidden
    unit whose receptive field contains (i, j): the transposed periodic conv.
    h: (C, K, L, L) 0/1.  Returns (C, L, L).
    """
    h = np.asarray(h, dtype=np.float64)
    C, K, L, _ = h.shape
    k = W.shape[1]
    b = np.full((C, L, L), float(vb))
    for kk in range(K):
        for da in range(k):
            for db in range(k):
                # shifted[c, i, j] = h[c, kk, (i-da) % L, (j-db) % L]
                shifted = np.roll(h[:, kk], shift=(da, db), axis=(1, 2))
                b += W[kk, da, db] * shifted
    return b


def joint_energy(v, h, W, hb, vb):
    """E(v,h) = -sum h^k (W^k*v) - sum_k h_bias^k sum h^k - v_bias sum v   (Eq. 12)."""
    v = np.asarray(v, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    conv = hidden_preact(v, W, np.zeros(W.shape[0]))
    return (-(h * conv).sum(axis=(1, 2, 3))
            - (np.asarray(hb)[None, :] * h.sum(axis=(2, 3))).sum(axis=1)
            - float(vb) * v.sum(axis=(1, 2)))


def free_energy(v, W, hb, vb):
    """F(v) = -v_bias sum v - sum_{k,i,j} log(1 + exp((v*W^k)_{ij} + h_bias^k))  (Eq. 13)."""
    v = np.asarray(v, dtype=np.float64)
    a = hidden_preact(v, W, hb)
    return -float(vb) * v.sum(axis=(1, 2)) - softplus(a).sum(axis=(1, 2, 3))


def gibbs_step(v, W, hb, vb, u_hidden, u_visible):
    """One block-Gibbs step v -> h -> v' (App. B.1, Eq. B4).

    h^k_{ij} = [u_hidden < sigma(a^k_{ij})], v'_{ij} = [u_visible < sigma(b_{ij})]:
    a Bernoulli draw of probability p taken as [u < p] with u uniform on (0,1).
    u_hidden: (C, K, L, L), u_visible: (C, L, L).  Returns (h, v') as uint8.
    """
    a = hidden_preact(v, W, hb)
    h = (u_hidden < sigmoid(a)).astype(np.uint8)
    b = visible_preact(h, W, vb)
    v_new = (u_visible < sigmoid(b)).astype(np.uint8)
    return h, v_new
