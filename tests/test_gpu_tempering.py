"""Parity of the CUDA parallel-tempering exchange correction (crbm_pt_run)
with the oracle's (App. B.2, Fig. 8b).

Both sides start from the same lattices and Philox streams.  Lattices,
exchange counts and the step counters must match bit for bit unless the oracle
reports a Bernoulli draw within 1e-12 of its threshold or an exchange decision
within 1e-10 (relative) of it; log pi, F, E and observable sums to 1e-9
relative (FP64 with other exp/log implementations and summation orders).
"""
import numpy as np
import pytest

import crbm_workloads as wl
from _common import gpu_ctx, oracle_chains

pytestmark = pytest.mark.gpu

SEED_X, SEED_Y = 2008054010, 77


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


def _run_oracle_pt(px, py, k, cycles):
    from oracle import tempering
    worst = {"bern": np.inf, "dec": np.inf}

    def rec(d):
        worst["bern"] = min(worst["bern"], float(np.min(d["bernoulli_margin"])))
        worst["dec"] = min(worst["dec"], float(np.min(d["swap_margin"])), float(np.min(d["temp_margin"])))

    tempering.run(px, py, k, cycles, record=rec)
    return worst


def _clear(worst):
    return worst["bern"] > 1e-12 and worst["dec"] > 1e-10


def _setup(ctx, kind, L, K, k, n, J, prec, pre_steps=0, std=0.3):
    from paper_2008_05401_gb300 import ISING
    W, hb, vb = wl.gaussian_crbm(K, k, std, seed=L * 7 + K)
    if kind == ISING:
        T = wl.ising_ladder(n, n, 1.8, 3.2)
    else:
        T = wl.kitaev_ladder(n, n, 0.05, 1.0)
    bx = wl.pack_bits(wl.random_lattices(n, L, seed=L + 1))
    by = wl.pack_bits(wl.random_lattices(n, L, seed=L + 2))
    name = "ising" if kind == ISING else "kitaev"
    px = oracle_chains(name, W, hb, vb, L, T, J, SEED_X, n, bx)
    py = oracle_chains(name, W, hb, vb, L, T, J, SEED_Y, n, by, cid_base=1000)
    mid = ctx.load_model(kind, W, vb, hb)
    jx = ctx.new_job(mid, kind, L, T, J, SEED_X, 0, bx, prec)
    jy = ctx.new_job(mid, kind, L, T, J, SEED_Y, 1000, by, prec)
    return px, py, jx, jy


def _compare(jx, jy, px, py, worst):
    if not _clear(worst):
        pytest.skip(f"oracle reports a decision inside the FP64 margin: {worst}")
    bits, step = jx.state()
    assert step == px.step
    np.testing.assert_array_equal(bits, wl.pack_bits(px.v))
    np.testing.assert_array_equal(jy.state()[0], wl.pack_bits(py.v))
    sums, acc, _ = jx.observables()
    np.testing.assert_array_equal(acc, px.accepts)
    np.testing.assert_allclose(sums, px.obs, rtol=1e-9, atol=1e-9)
    lp, F, E = jx.energies()
    np.testing.assert_allclose(lp, px.logpi, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(E, px.E_phys, rtol=1e-9, atol=1e-9)
    # the mixed path carries F as its FP32 value (within the certified bound
    # its decisions used); the read-back re-evaluates it in FP64 either way
    tol = dict(rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(F, px.F, **tol)
    lpy, Fy, _ = jy.energies()
    np.testing.assert_allclose(lpy, py.logpi, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(Fy, py.F, **tol)


ISING_PT = [
    # L, K, k, n, g, cycles
    (4, 2, 3, 12, 1, 8),
    (8, 4, 5, 9, 2, 6),      # odd ladder: a lone end chain on every cycle
    (16, 4, 3, 16, 1, 5),
    (64, 2, 5, 4, 1, 3),     # multi-word rows
]


@pytest.mark.parametrize("L,K,k,n,g,cycles", ISING_PT)
@pytest.mark.parametrize("prec_name", ["FP64", "MIXED"])
def test_ising_pt_matches_oracle(ctx, L, K, k, n, g, cycles, prec_name):
    import paper_2008_05401_gb300 as P
    prec = getattr(P, prec_name)
    px, py, jx, jy = _setup(ctx, P.ISING, L, K, k, n, (1.0,), prec)
    worst = _run_oracle_pt(px, py, g, cycles)
    ctx.pt_run(jx, jy, cycles, g=g, precision=prec)
    _compare(jx, jy, px, py, worst)
    if L <= 16:     # random filters: swaps become rare on large lattices
        assert px.accepts.sum() > 0
    jx.release()
    jy.release()


KITAEV_PT = [
    # L, K, k, n, cycles, J
    (3, 4, 3, 8, 5, (0.8, 1.1, 1.3)),
    (4, 4, 3, 7, 4, (1.0, 1.0, 1.0)),
    (6, 2, 3, 4, 3, (1.0, 1.0, 1.0)),
]


@pytest.mark.parametrize("L,K,k,n,cycles,J", KITAEV_PT)
@pytest.mark.parametrize("prec_name", ["FP64", "MIXED"])
def test_kitaev_pt_matches_oracle(ctx, L, K, k, n, cycles, J, prec_name):
    import paper_2008_05401_gb300 as P
    prec = getattr(P, prec_name)
    px, py, jx, jy = _setup(ctx, P.KITAEV, L, K, k, n, J, prec, std=0.05)
    worst = _run_oracle_pt(px, py, 1, cycles)
    ctx.pt_run(jx, jy, cycles, precision=prec)
    _compare(jx, jy, px, py, worst)
    jx.release()
    jy.release()


def test_pt_split_calls_equal_one_call(ctx):
    """Cycles split over calls continue exactly (device step counters, cached
    spectra): 2 + 3 cycles == 5 cycles, bit for bit."""
    import paper_2008_05401_gb300 as P
    out = []
    for parts in ((5,), (2, 3)):
        _, _, jx, jy = _setup(ctx, P.KITAEV, 4, 4, 3, 6, (1.0, 1.0, 1.0), P.FP64, std=0.05)
        for c in parts:
            ctx.pt_run(jx, jy, c)
        out.append((jx.state()[0], jx.energies(), jx.observables()[:2], jy.state()[0]))
        jx.release()
        jy.release()
    a, b = out
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[3], b[3])
    for x, y in zip(a[1] + a[2], b[1] + b[2]):
        np.testing.assert_array_equal(x, y)


def test_pt_after_proposals_reevaluates(ctx):
    """Proposals on the physical job (mixed precision: F within a bound) then
    tempering: the physical chains are re-evaluated in FP64 first, matching
    the oracle's run of the same sequence."""
    import paper_2008_05401_gb300 as P
    from oracle import chain
    px, py, jx, jy = _setup(ctx, P.ISING, 8, 4, 5, 8, (1.0,), P.MIXED)
    chain.run(px, 3)
    jx.run(3, precision=P.MIXED)
    worst = _run_oracle_pt(px, py, 1, 4)
    ctx.pt_run(jx, jy, 4, precision=P.MIXED)
    # sums and accepts continue from the 3 proposals
    _compare(jx, jy, px, py, worst)
    jx.release()
    jy.release()


def test_pt_rejects_mismatched_jobs(ctx):
    import paper_2008_05401_gb300 as P
    from paper_2008_05401_gb300 import CrbmError
    W, hb, vb = wl.gaussian_crbm(2, 3, 0.2)
    mid = ctx.load_model(P.ISING, W, vb, hb)
    a = ctx.new_job(mid, P.ISING, 8, np.array([2.0, 2.5]), (1.0,), 1)
    b = ctx.new_job(mid, P.ISING, 8, np.array([2.0, 2.6]), (1.0,), 2)
    c = ctx.new_job(mid, P.ISING, 16, np.array([2.0, 2.5]), (1.0,), 3)
    for x, y in ((a, b), (a, c), (a, a)):
        with pytest.raises(CrbmError):
            ctx.pt_run(x, y, 1)
    with pytest.raises(CrbmError):
        ctx.pt_run(a, b, 1, g=0)
    for j in (a, b, c):
        j.release()


def _cd1_bank():
    import os
    from _common import ROOT
    d = np.load(os.path.join(ROOT, "paper_2008_05401_gb300", "data", "ising_cd1_L16_K4_k5.npz"))
    return d["W"], d["hb"], float(d["vb"])


FULL_PT = [
    # model, L, chains per side, g, warm-up cycles, compared cycles
    ("ising", 16, 4096, 1, 2, 3),
    ("kitaev", 6, 1024, 1, 2, 4),
    ("kitaev", 8, 1024, 4, 2, 2),     # k = 4 Gibbs steps per correction (Table II)
]


@pytest.mark.parametrize("model,L,n,g,warm,cycles", FULL_PT)
def test_full_size_pt_matches_oracle(ctx, model, L, n, g, warm, cycles):
    """The tempering configurations the bench times, at their full size and in
    their launch configuration: the Ising L = 16 ladder of 4096 physical plus
    4096 RBM chains on the CD-1 filter bank (32 temperatures in [1.5, 3.5]),
    and the Kitaev L = 6 and L = 8 (g = 4) ladders of 1024 + 1024 chains over
    24 temperatures in [0.005, 1], mixed precision.  Job x (seed s, chain ids
    0..n-1) and job y (seed s + 1, ids n..2n-1) run warm-up cycles and then
    more in a second call; the oracle runs the same cycles from the same
    lattices.  Both lattices, swap counts, step counters, observable sums and
    FP64 energies must match as in the small cases."""
    import paper_2008_05401_gb300 as P
    if model == "ising":
        W, hb, vb = _cd1_bank()
        T, J, kind = wl.ising_ladder(n, 32), (1.0,), P.ISING
    else:
        W, hb, vb = wl.gaussian_crbm(4, 3, 0.05)
        T, J, kind = wl.kitaev_ladder(n, 24), (1.0, 1.0, 1.0), P.KITAEV
    bx = wl.pack_bits(wl.random_lattices(n, L, seed=SEED_X + L))
    by = wl.pack_bits(wl.random_lattices(n, L, seed=SEED_X + L + 1))
    px = oracle_chains(model, W, hb, vb, L, T, J, SEED_X, n, bx)
    py = oracle_chains(model, W, hb, vb, L, T, J, SEED_X + 1, n, by, cid_base=n)
    mid = ctx.load_model(kind, W, vb, hb)
    jx = ctx.new_job(mid, kind, L, T, J, SEED_X, 0, bx, P.MIXED)
    jy = ctx.new_job(mid, kind, L, T, J, SEED_X + 1, n, by, P.MIXED)
    worst = _run_oracle_pt(px, py, g, warm + cycles)
    ctx.pt_run(jx, jy, warm, g=g, precision=P.MIXED)
    ctx.pt_run(jx, jy, cycles, g=g, precision=P.MIXED)
    _compare(jx, jy, px, py, worst)
    assert px.accepts.sum() > 0
    jx.release()
    jy.release()
