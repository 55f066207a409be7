"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the sampling method itself: it only draws
model parameters, temperature ladders and initial lattices from numpy's seeded
generators, and converts lattices between the unpacked 0/1 form and the packed
bit layout used at the C-ABI boundary.

Packed layout (one chain): site n = i*L + j of the L x L lattice is bit (n % 32)
of uint32 word n // 32; a chain occupies ceil(L*L/32) words.

Workload recipes (the paper has no dataset; its runs are its own Monte Carlo
chains, Sec. III and Sec. IV):
  * Ising, small:  L=8, J=1, T=2.269, 16 chains, K=2 filters 3x3, W, v_bias,
    h_bias ~ N(0, 0.1^2).
  * Ising, batch:  L in {16,32,64,128}, 4096 chains per L, 32 temperatures
    uniform in [1.5, 3.5] (chain c -> T index c mod 32), K=4 filters 5x5.
  * Kitaev, small: L=6 (N=36 cells, 72 sites), J=(1,1,1), 1024 chains, 24
    temperatures log-spaced in [0.005, 1] (chain c -> c mod 24), K=4 filters
    3x3, parameters ~ N(0, 0.05^2).
  * Kitaev, batch: L in {8,10,12}, 2048 chains split over L by c mod 3.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 2008054010


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.uint64(seed))


def gaussian_crbm(K: int, k: int, std: float, seed: int = BASE_SEED):
    """CRBM parameters drawn i.i.d. N(0, std^2): W[K,k,k], h_bias[K], v_bias."""
    g = rng(seed)
    W = g.normal(0.0, std, size=(K, k, k))
    hb = g.normal(0.0, std, size=(K,))
    vb = float(g.normal(0.0, std))
    return W, hb, vb


def ising_ladder(n_chains: int, n_T: int = 32, lo: float = 1.5, hi: float = 3.5):
    """Per-chain temperatures: T_i = lo + (hi-lo) i/(n_T-1), chain c -> i = c mod n_T."""
    Ts = lo + (hi - lo) * np.arange(n_T) / max(n_T - 1, 1)
    return Ts[np.arange(n_chains) % n_T]


def kitaev_ladder(n_chains: int, n_T: int = 24, lo: float = 0.005, hi: float = 1.0):
    """Per-chain temperatures log-spaced in [lo, hi], chain c -> i = c mod n_T."""
    Ts = lo * (hi / lo) ** (np.arange(n_T) / max(n_T - 1, 1))
    return Ts[np.arange(n_chains) % n_T]


def words_per_chain(L: int) -> int:
    return (L * L + 31) // 32


def pack_bits(v: np.ndarray) -> np.ndarray:
    """(C, L, L) 0/1 array -> (C, ceil(L*L/32)) uint32 in the packed layout."""
    v = np.asarray(v)
    C, L, _ = v.shape
    N = L * L
    W = words_per_chain(L)
    flat = np.zeros((C, W * 32), dtype=np.uint64)
    flat[:, :N] = v.reshape(C, N).astype(np.uint64)
    weights = np.uint64(1) << np.arange(32, dtype=np.uint64)
    return (flat.reshape(C, W, 32) * weights).sum(axis=2).astype(np.uint32)


def unpack_bits(words: np.ndarray, L: int) -> np.ndarray:
    """(C, ceil(L*L/32)) uint32 -> (C, L, L) uint8 0/1 array."""
    words = np.asarray(words, dtype=np.uint32)
    C = words.shape[0]
    N = L * L
    bits = (words[:, :, None] >> np.arange(32, dtype=np.uint32)) & np.uint32(1)
    return bits.reshape(C, -1)[:, :N].reshape(C, L, L).astype(np.uint8)


def random_lattices(n_chains: int, L: int, seed: int = BASE_SEED) -> np.ndarray:
    """Bernoulli(1/2) initial lattices, (C, L, L) uint8."""
    return rng(seed).integers(0, 2, size=(n_chains, L, L), dtype=np.uint8)


def init_train_params(K: int, k: int, seed: int = BASE_SEED):
    """Initial CRBM parameters of the trainer (Algorithm 1): W ~ N(0, sigma)
    with sigma = 2 / (K k^2) read as a standard deviation, v_bias = 0,
    h_bias = 0.  Returned as the flat FP64 vector [W (K*k*k), v_bias, h_bias (K)]."""
    g = rng(seed)
    W = g.normal(0.0, 2.0 / (K * k * k), size=K * k * k)
    return np.concatenate([W, [0.0], np.zeros(K)])


def split_params(theta, K: int, k: int):
    """[W, v_bias, h_bias] flat vector -> (W (K, k, k), h_bias (K,), v_bias)."""
    theta = np.asarray(theta, dtype=np.float64)
    return theta[:K * k * k].reshape(K, k, k), theta[K * k * k + 1:].copy(), float(theta[K * k * k])


def epoch_order(n: int, seed: int, epoch: int) -> np.ndarray:
    """Order in which one training epoch visits its n samples (a seeded
    permutation; minibatches are consecutive runs of it)."""
    return rng(seed * 1000003 + epoch).permutation(n).astype(np.int32)
