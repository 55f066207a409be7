"""Seeded CD-1 training of a CRBM on the build's own Metropolis samples.

Produces the filter bank of the batch Ising workload: K = 4 filters 5 x 5,
trained on an L = 16 periodic lattice at T = 2.269 and then applied unchanged
at larger L (the paper's point that a CRBM trained small transfers to large
lattices, Sec. I and Sec. III).  The paper itself trains with an energy-matching
loss and ADAM (Sec. II, Algorithm 1); this workload instead asks for plain
contrastive divergence with one Gibbs step, with the paper's learning rate
1e-3 and batch size 20 (App. D).  Offline input generation on the CPU (numpy),
not part of the sampling path.

    python -m paper_2008_05401_gb300.train_cd1   # writes data/ising_cd1_L16_K4_k5.npz
"""
from __future__ import annotations

import os

import numpy as np

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "ising_cd1_L16_K4_k5.npz")


def metropolis_samples(L=16, T=2.269, n_chains=64, warm=1000, n_samples=10000, spacing=10, seed=1):
    """Checkerboard single-spin Metropolis for E = -sum s_i s_j on the torus;
    returns n_samples lattices as 0/1 arrays (v = (s + 1) / 2)."""
    g = np.random.default_rng(seed)
    s = g.choice(np.array([-1, 1], dtype=np.int8), size=(n_chains, L, L))
    ii, jj = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    masks = [((ii + jj) % 2 == c) for c in (0, 1)]
    beta = 1.0 / T

    def sweep():
        for m in masks:
            nb = (np.roll(s, 1, 1) + np.roll(s, -1, 1) + np.roll(s, 1, 2) + np.roll(s, -1, 2)).astype(np.int16)
            dE = 2 * s * nb                                 # energy change of flipping each spin
            flip = (g.random(s.shape) < np.exp(-beta * dE)) & m
            s[flip] *= -1

    for _ in range(warm):
        sweep()
    out = []
    while len(out) * n_chains < n_samples:
        for _ in range(spacing):
            sweep()
        out.append(((s + 1) // 2).astype(np.uint8).copy())
    return np.concatenate(out)[:n_samples]


def _corr(v, W, hb):
    """a[c,f,i,j] = hb[f] + sum_ab W[f,a,b] v[c,(i+a)%L,(j+b)%L]."""
    K, k, _ = W.shape
    a = np.broadcast_to(hb[None, :, None, None], (v.shape[0], K) + v.shape[1:]).copy()
    for da in range(k):
        for db in range(k):
            a += W[None, :, da, db, None, None] * np.roll(v, (-da, -db), axis=(1, 2))[:, None]
    return a


def _corr_t(h, W, vb):
    """b[c,i,j] = vb + sum_f sum_ab W[f,a,b] h[c,f,(i-a)%L,(j-b)%L]."""
    K, k, _ = W.shape
    b = np.full((h.shape[0],) + h.shape[2:], vb)
    for f in range(K):
        for da in range(k):
            for db in range(k):
                b += W[f, da, db] * np.roll(h[:, f], (da, db), axis=(1, 2))
    return b


def _grad_W(v, p, k):
    """sum over chains and sites of p[c,f,i,j] v[c,i+a,j+b], shape (K, k, k)."""
    K = p.shape[1]
    G = np.empty((K, k, k))
    for da in range(k):
        for db in range(k):
            G[:, da, db] = np.einsum("cfij,cij->f", p, np.roll(v, (-da, -db), axis=(1, 2)))
    return G


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def cd1(data, K=4, k=5, lr=1e-3, batch=20, epochs=20, seed=2):
    g = np.random.default_rng(seed)
    W = g.normal(0.0, 0.01, size=(K, k, k))
    hb = np.zeros(K)
    vb = 0.0
    v_all = data.astype(np.float64)
    n = len(v_all)
    for _ in range(epochs):
        order = g.permutation(n)
        for s in range(0, n - batch + 1, batch):
            v0 = v_all[order[s:s + batch]]
            p0 = sigmoid(_corr(v0, W, hb))
            h0 = (g.random(p0.shape) < p0).astype(np.float64)
            v1 = (g.random(v0.shape) < sigmoid(_corr_t(h0, W, vb))).astype(np.float64)
            p1 = sigmoid(_corr(v1, W, hb))
            W += lr * (_grad_W(v0, p0, k) - _grad_W(v1, p1, k)) / batch
            hb += lr * (p0.sum(axis=(0, 2, 3)) - p1.sum(axis=(0, 2, 3))) / batch
            vb += lr * (v0.sum() - v1.sum()) / batch
    return W, hb, vb


def main():
    data = metropolis_samples()
    W, hb, vb = cd1(data)
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    np.savez(OUT, W=W, hb=hb, vb=np.array(vb), T=np.array(2.269), L=np.array(16))
    print(OUT, "W range", W.min(), W.max(), "hb", hb, "vb", vb)


if __name__ == "__main__":
    main()
