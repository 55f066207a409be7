"""Locally connected CRBM (LCRBM) for open boundaries (Sec. IV, open
boundary conditions) -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  FP64.

Reading (the paper gives the idea, not the layout): the lattice is open along
the column direction j and periodic along the rows i.  A hidden unit (f, i, j)
sees the visible window rows (i + a) mod L (periodic), columns j + b for
b = 0..k-1 (top-left anchor, as in the periodic CRBM), and a column past L-1
contributes nothing (open: no wrap).  Its kernel depends on the column class
of j: the `edge` left columns j < edge have their own kernels (classes
0..edge-1), the `edge` right columns j >= L - edge theirs (classes
edge..2 edge-1), every other column shares the bulk kernel (class 2 edge).
The paper introduces three unshared kernels on each side: edge = 3.
Hidden biases are shared per filter.  W has shape (2 edge + 1, K, k, k).

    a^f_ij = h_bias^f + sum_ab W[c(j), f, a, b] v_(i+a mod L),(j+b)      (j+b < L)
    E(v, h) = -v_bias sum v - sum_f h_bias^f sum h^f - sum_f sum_ij h^f_ij (a^f_ij - h_bias^f)
    F(v)    = -v_bias sum v - sum_fij softplus(a^f_ij)
    b_ij    = v_bias + sum_f sum_ab W[c(j-b), f, a, b] h^f_(i-a mod L),(j-b)  (j-b >= 0)

The same Bernoulli draws and Gibbs step as the periodic CRBM (Eqs. B1-B4).
"""
from __future__ import annotations

import numpy as np

from .crbm import softplus


def col_class(L: int, edge: int) -> np.ndarray:
    c = np.full(L, 2 * edge, dtype=np.int64)
    c[:edge] = np.arange(edge)
    c[L - edge:] = edge + np.arange(edge)
    return c


def hidden_preact(v, W, hb, edge):
    """(C, K, L, L) pre-activations; W: (2 edge + 1, K, k, k)."""
    v = np.asarray(v, dtype=np.float64)
    C, L, _ = v.shape
    _, K, k, _ = W.shape
    cls = col_class(L, edge)
    a = np.empty((C, K, L, L))
    a[:] = np.asarray(hb, dtype=np.float64)[None, :, None, None]
    for da in range(k):
        rows = np.roll(v, -da, axis=1)                     # rows[c, i, :] = v[c, (i+da) % L, :]
        for db in range(k):
            shifted = np.zeros_like(v)
            shifted[:, :, :L - db] = rows[:, :, db:]       # v[(i+da)%L, j+db], 0 past the edge
            w = W[cls, :, da, db].T                        # (K, L): weight of column j's class
            a += w[None, :, None, :] * shifted[:, None, :, :]
    return a


def visible_preact(h, W, vb, edge):
    """(C, L, L): the transpose of hidden_preact's weight part plus v_bias."""
    h = np.asarray(h, dtype=np.float64)
    C, K, L, _ = h.shape
    k = W.shape[2]
    cls = col_class(L, edge)
    b = np.full((C, L, L), float(vb))
    for da in range(k):
        for db in range(k):
            for j in range(db, L):
                jh = j - db                                # hidden column feeding visible column j
                w = W[cls[jh], :, da, db]                  # (K,)
                hs = np.roll(h[:, :, :, jh], da, axis=2)   # h[f, (i-da) % L, jh]
                b[:, :, j] += (w[None, :, None] * hs).sum(axis=1)
    return b


def joint_energy(v, h, W, hb, vb, edge):
    v = np.asarray(v, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    conv = hidden_preact(v, W, np.zeros(W.shape[1]), edge)
    return (-(h * conv).sum(axis=(1, 2, 3))
            - (np.asarray(hb)[None, :] * h.sum(axis=(2, 3))).sum(axis=1)
            - float(vb) * v.sum(axis=(1, 2)))


def free_energy(v, W, hb, vb, edge):
    v = np.asarray(v, dtype=np.float64)
    return -float(vb) * v.sum(axis=(1, 2)) - softplus(hidden_preact(v, W, hb, edge)).sum(axis=(1, 2, 3))
