"""Philox4x32-10 counter-based generator and the uniform streams of the sampler.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper does not say which random numbers its Theano sampler used.  Both
sides of this project draw every uniform from Philox4x32 with 10 rounds
(Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11), written here from that description:

* state: four 32-bit counter words (x0, x1, x2, x3), key (k0, k1);
* one round: multiply x0 by M0 = 0xD2511F53 and x2 by M1 = 0xCD9E8D57 as
  32x32 -> 64-bit products, then
  (x0, x1, x2, x3) <- (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0));
* between rounds the key is bumped by the Weyl constants
  (k0, k1) += (0x9E3779B9, 0xBB67AE85) mod 2^32.

Stream layout (one call = four words = four consecutive sites):
  counter = (q, tag, step, chain_id), key = (seed & 0xffffffff, seed >> 32),
  site n of plane ``tag`` uses word n % 4 of block q = n // 4;
  u = (word + 0.5) * 2^-32, so u lies strictly inside (0, 1).
Tags for Gibbs sub-step s of a model with K filters: hidden plane k -> s*(K+1)+k,
visible plane -> s*(K+1)+K; the acceptance uniform -> TAG_ACC (block 0,
word 0); random initial lattices -> TAG_INIT at step 0.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF

TAG_ACC = 0xFFFFFFFE
TAG_INIT = 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on broadcastable uint32 arrays; returns 4 uint32 arrays."""
    x = [np.asarray(c, dtype=np.uint64) & np.uint64(MASK) for c in (c0, c1, c2, c3)]
    x = np.broadcast_arrays(*x)
    x = [a.copy() for a in x]
    ka = np.asarray(k0, dtype=np.uint64) & np.uint64(MASK)
    kb = np.asarray(k1, dtype=np.uint64) & np.uint64(MASK)
    m0, m1, mask = np.uint64(M0), np.uint64(M1), np.uint64(MASK)
    for _ in range(10):
        p0 = m0 * x[0]          # < 2^64: exact in uint64
        p1 = m1 * x[2]
        x = [(p1 >> np.uint64(32)) ^ x[1] ^ ka,
             p1 & mask,
             (p0 >> np.uint64(32)) ^ x[3] ^ kb,
             p0 & mask]
        ka = (ka + np.uint64(W0)) & mask
        kb = (kb + np.uint64(W1)) & mask
    return [a.astype(np.uint32) for a in x]


def words(seed: int, chain_ids, step: int, tag: int, n_sites: int) -> np.ndarray:
    """Raw 32-bit words for sites 0..n_sites-1 of one tag; shape (len(chain_ids), n_sites)."""
    chain_ids = np.asarray(chain_ids, dtype=np.uint64).reshape(-1, 1)
    n = np.arange(n_sites, dtype=np.uint64).reshape(1, -1)
    q = n >> np.uint64(2)
    out = philox4x32_10(q, np.uint64(tag), np.uint64(step & MASK), chain_ids,
                        np.uint64(seed & MASK), np.uint64((seed >> 32) & MASK))
    out = np.stack(out, axis=-1)                      # (C, n_sites, 4)
    sel = (n & np.uint64(3)).astype(np.int64)
    return np.take_along_axis(out, np.broadcast_to(sel, out.shape[:2])[..., None], axis=-1)[..., 0]


def uniforms(seed: int, chain_ids, step: int, tag: int, n_sites: int) -> np.ndarray:
    """u = (word + 1/2) 2^-32 for sites 0..n_sites-1 of one tag (FP64, exact)."""
    return (words(seed, chain_ids, step, tag, n_sites).astype(np.float64) + 0.5) * 2.0 ** -32


def hidden_tag(sub: int, K: int, k: int) -> int:
    return sub * (K + 1) + k


def visible_tag(sub: int, K: int) -> int:
    return sub * (K + 1) + K
