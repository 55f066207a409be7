"""Shared helpers of the test-suite (no method arithmetic: setup and comparison)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import crbm_workloads as wl  # noqa: E402


def gpu_ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_05401_gb300 import Context, load
    import __graft_entry__
    __graft_entry__.build()
    load()
    return Context(0)


def kind_of(model):
    return 0 if model == "ising" else 1


def oracle_chains(model, W, hb, vb, L, T, J, seed, n, bits0, cid_base=0):
    from oracle import chain
    v0 = wl.unpack_bits(bits0, L)
    return chain.make_chains(chain.ISING if model == "ising" else chain.KITAEV, W, hb, vb, L, T, J, seed,
                             np.arange(cid_base, cid_base + n), v0=v0)


def run_oracle(ch, S, g=1, correct=True):
    """Run the oracle S steps; return (max-margin info) to judge exact comparisons."""
    from oracle import chain
    worst = {"bern": np.inf, "mh": np.inf}

    def rec(c, d):
        worst["bern"] = min(worst["bern"], float(np.min(d["bernoulli_margin"])))
        rel = d["mh_margin"] / d["mh_scale"]
        if correct:
            worst["mh"] = min(worst["mh"], float(np.min(rel)))

    chain.run(ch, S, g=g, correct=correct, record=rec)
    return worst


def decisions_are_clear(worst, bern_tol=1e-12, mh_tol=1e-10):
    """True when no Bernoulli draw came within bern_tol of its threshold and no
    MH decision within mh_tol (relative) -- then both sides must agree exactly."""
    return worst["bern"] > bern_tol and worst["mh"] > mh_tol
