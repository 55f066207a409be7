"""Parity of the CUDA path with the oracle for the open-boundary Kitaev model
and the locally connected CRBM (Sec. IV, open boundary conditions): MH
proposals, uncorrected Gibbs, local sweeps and the tempering correction.

Lattices and accept counts bit-exact unless the oracle reports a decision
within its FP64 margin; log pi, F, E and sums to 1e-9 relative.
"""
import numpy as np
import pytest

import crbm_workloads as wl
from _common import decisions_are_clear, gpu_ctx, run_oracle

pytestmark = pytest.mark.gpu

SEED = 2008054010


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


def _params(edge, K, k, seed, std=0.1):
    g = np.random.default_rng(seed)
    return g.normal(0, std, (2 * edge + 1, K, k, k)), g.normal(0, std, K), float(g.normal(0, std))


def _oracle(W, hb, vb, L, T, J, seed, bits0, edge, cid_base=0):
    from oracle import chain
    return chain.make_chains(chain.KITAEV, W, hb, vb, L, T, J, seed, np.arange(cid_base, cid_base + len(T)),
                             v0=wl.unpack_bits(bits0, L), edge=edge)


def _compare(job, ref):
    bits, step = job.state()
    assert step == ref.step
    np.testing.assert_array_equal(bits, wl.pack_bits(ref.v))
    sums, acc, _ = job.observables()
    np.testing.assert_array_equal(acc, ref.accepts)
    np.testing.assert_allclose(sums, ref.obs, rtol=1e-9, atol=1e-9)
    lp, F, E = job.energies()
    np.testing.assert_allclose(lp, ref.logpi, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(F, ref.F, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(E, ref.E_phys, rtol=1e-9, atol=1e-9)


CASES = [
    # L, edge, K, k, n, correct, J
    (3, 1, 2, 2, 6, True, (0.8, 1.1, 1.3)),
    (6, 2, 2, 3, 6, True, (1.0, 1.0, 1.0)),
    (6, 1, 4, 3, 4, False, (1.0, 1.0, 1.0)),     # a specialised shape: runs the generic variant
    (8, 3, 2, 5, 3, True, (1.0, 1.0, 1.0)),      # the paper's three edge kernels, 2x5x5 kernels
]


@pytest.mark.parametrize("L,edge,K,k,n,correct,J", CASES)
def test_lcrbm_open_kitaev_matches_oracle(ctx, L, edge, K, k, n, correct, J):
    from paper_2008_05401_gb300 import FP64, KITAEV
    W, hb, vb = _params(edge, K, k, L * 10 + edge)
    T = wl.kitaev_ladder(n, n, 0.05, 1.0)
    bits0 = wl.pack_bits(wl.random_lattices(n, L, seed=L + 21))
    ref = _oracle(W, hb, vb, L, T, J, SEED, bits0, edge)
    worst = run_oracle(ref, 4, correct=correct)
    mid = ctx.load_lcrbm(KITAEV, W, vb, hb)
    job = ctx.new_job(mid, KITAEV, L, T, J, SEED, 0, bits0, FP64)
    job.run(4, correct=correct, precision=FP64)
    if not decisions_are_clear(worst):
        pytest.skip(f"oracle reports a decision inside the FP64 margin: {worst}")
    _compare(job, ref)
    job.release()


def test_open_kitaev_local_sweeps_match_oracle(ctx):
    from oracle import metropolis
    from paper_2008_05401_gb300 import FP64, KITAEV
    L, edge, n = 4, 1, 5
    W, hb, vb = _params(edge, 2, 2, 3)
    T = wl.kitaev_ladder(n, n, 0.05, 1.0)
    bits0 = wl.pack_bits(wl.random_lattices(n, L, seed=8))
    ref = _oracle(W, hb, vb, L, T, (1.0, 1.0, 1.0), SEED, bits0, edge)
    worst = np.inf
    for _ in range(2):
        d = metropolis.sweep(ref, exchange=True)
        worst = min(worst, float(np.min(d["margin"])), float(np.min(d["temp_margin"])))
    mid = ctx.load_lcrbm(KITAEV, W, vb, hb)
    job = ctx.new_job(mid, KITAEV, L, T, (1.0, 1.0, 1.0), SEED, 0, bits0, FP64)
    job.local_run(2, exchange=True)
    if worst < 1e-10:
        pytest.skip("decision inside the FP64 margin")
    _compare(job, ref)
    job.release()


def test_open_kitaev_tempering_matches_oracle(ctx):
    from oracle import tempering
    from paper_2008_05401_gb300 import FP64, KITAEV
    L, edge, n = 4, 1, 6
    W, hb, vb = _params(edge, 2, 3, 5)
    J = (1.0, 1.0, 1.0)
    T = wl.kitaev_ladder(n, n, 0.05, 1.0)
    bx = wl.pack_bits(wl.random_lattices(n, L, seed=1))
    by = wl.pack_bits(wl.random_lattices(n, L, seed=2))
    px = _oracle(W, hb, vb, L, T, J, SEED, bx, edge)
    py = _oracle(W, hb, vb, L, T, J, 77, by, edge, cid_base=1000)
    worst = np.inf
    for _ in range(3):
        d = tempering.cycle(px, py, 2)
        worst = min(worst, float(np.min(d["swap_margin"])), float(np.min(d["temp_margin"])))
    mid = ctx.load_lcrbm(KITAEV, W, vb, hb)
    jx = ctx.new_job(mid, KITAEV, L, T, J, SEED, 0, bx, FP64)
    jy = ctx.new_job(mid, KITAEV, L, T, J, 77, 1000, by, FP64)
    ctx.pt_run(jx, jy, 3, g=2)
    if worst < 1e-10:
        pytest.skip("decision inside the FP64 margin")
    _compare(jx, px)
    np.testing.assert_array_equal(jy.state()[0], wl.pack_bits(py.v))
    jx.release()
    jy.release()


def test_lcrbm_rejections(ctx):
    from paper_2008_05401_gb300 import FP64, ISING, KITAEV, MIXED, CrbmError
    W, hb, vb = _params(2, 2, 3, 1)
    with pytest.raises(CrbmError):
        ctx.load_lcrbm(ISING, W, vb, hb)                  # the open-boundary physics is Kitaev's
    mid = ctx.load_lcrbm(KITAEV, W, vb, hb)
    with pytest.raises(CrbmError):
        ctx.new_job(mid, KITAEV, 3, np.full(2, 0.5), (1.0, 1.0, 1.0), 1)   # L < 2 edge
    job = ctx.new_job(mid, KITAEV, 5, np.full(2, 0.5), (1.0, 1.0, 1.0), 1, 0, None, FP64)
    with pytest.raises(CrbmError):
        job.run(1, precision=MIXED)
    job.release()
