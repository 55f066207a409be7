"""Behaviour of the C ABI on the GPU: batching, checkpoints, edge cases, errors."""
import numpy as np
import pytest

import crbm_workloads as wl
from _common import gpu_ctx

pytestmark = pytest.mark.gpu

SEED = 77


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


def _ising_model(ctx, K=4, k=5, std=0.2, seed=5):
    from paper_2008_05401_gb300 import ISING
    W, hb, vb = wl.gaussian_crbm(K, k, std, seed=seed)
    return ctx.load_model(ISING, W, vb, hb)


def _snapshot(job):
    bits, step = job.state()
    lp, F, E = job.energies()
    sums, acc, rec = job.observables()
    return dict(bits=bits, step=step, lp=lp, F=F, E=E, sums=sums, acc=acc, rec=rec)


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_equals_each_job_alone(ctx, prec):
    """Chains of different L and temperature in one launch give the results
    each job gives alone (random streams are keyed by chain id)."""
    from paper_2008_05401_gb300 import ISING
    mid = _ising_model(ctx)
    mid2 = _ising_model(ctx, seed=6)          # another model of the same shape
    spec = [(16, 40, mid, 0), (32, 9, mid2, 1000), (64, 3, mid, 5000)]

    def make():
        return [ctx.new_job(m, ISING, L, wl.ising_ladder(n, 8), (1.0,), SEED, base,
                            wl.pack_bits(wl.random_lattices(n, L, seed=L)), prec) for L, n, m, base in spec]

    batch = make()
    ctx.run_batch(batch, 7, precision=prec)
    alone = make()
    for j in alone:
        j.run(7, precision=prec)
    for a, b in zip(batch, alone):
        sa, sb = _snapshot(a), _snapshot(b)
        for key in sa:
            np.testing.assert_array_equal(sa[key], sb[key], err_msg=key)
        a.release()
        b.release()


@pytest.mark.parametrize("prec", [0, 1])
def test_kitaev_batch_of_mixed_sizes_equals_alone(ctx, prec):
    """Kitaev jobs of small and large matrices (chain groups of 32, 64, 128
    and 256 threads; several chains per CTA and short last tiles) in one
    launch give every job the results it has alone."""
    from paper_2008_05401_gb300 import KITAEV
    W, hb, vb = wl.gaussian_crbm(4, 3, 0.05, seed=3)
    mid = ctx.load_model(KITAEV, W, vb, hb)
    spec = [(4, 5, 0), (6, 7, 100), (10, 3, 200), (12, 2, 300), (8, 9, 400)]

    def make():
        return [ctx.new_job(mid, KITAEV, L, wl.kitaev_ladder(n, 24), (1.0, 1.0, 1.0), SEED, base,
                            wl.pack_bits(wl.random_lattices(n, L, seed=L)), prec) for L, n, base in spec]

    batch = make()
    ctx.run_batch(batch, 3, precision=prec)
    alone = make()
    for j in alone:
        j.run(3, precision=prec)
    for a, b in zip(batch, alone):
        sa, sb = _snapshot(a), _snapshot(b)
        for key in sa:
            np.testing.assert_array_equal(sa[key], sb[key], err_msg=key)
        a.release()
        b.release()


@pytest.mark.parametrize("L,prec", [(6, 1), (6, 0), (4, 0)])
def test_autotuned_kitaev_groups_keep_parity(ctx, L, prec):
    """crbm_tune picks the chains (thread groups) per CTA of a Kitaev shape;
    a job created afterwards, with a short last tile, reproduces the oracle."""
    from _common import decisions_are_clear, oracle_chains, run_oracle
    from paper_2008_05401_gb300 import KITAEV
    W, hb, vb = wl.gaussian_crbm(4, 3, 0.05, seed=9)
    mid = ctx.load_model(KITAEV, W, vb, hb)
    nc, us = ctx.tune(mid, L, prec)
    assert nc in (1, 2, 4, 8) and us > 0
    n, S, J = 2 * nc + 3, 3, (1.0, 1.0, 1.0)
    T = wl.kitaev_ladder(n, 24)
    bits0 = wl.pack_bits(wl.random_lattices(n, L, seed=45))
    job = ctx.new_job(mid, KITAEV, L, T, J, SEED, 0, bits0, prec)
    job.run(S, precision=prec)
    ref = oracle_chains("kitaev", W, hb, vb, L, T, J, SEED, n, bits0)
    worst = run_oracle(ref, S)
    if decisions_are_clear(worst):
        np.testing.assert_array_equal(job.state()[0], wl.pack_bits(ref.v))
        np.testing.assert_array_equal(job.observables()[1], ref.accepts)
        lp, F, E = job.energies()
        np.testing.assert_allclose(lp, ref.logpi, rtol=1e-10, atol=1e-9)
        np.testing.assert_allclose(F, ref.F, rtol=1e-10, atol=1e-10)
    job.release()


def test_split_runs_and_checkpoint_resume(ctx):
    from paper_2008_05401_gb300 import ISING, MIXED
    mid = _ising_model(ctx)
    T = wl.ising_ladder(12, 4)
    bits0 = wl.pack_bits(wl.random_lattices(12, 32, seed=3))
    straight = ctx.new_job(mid, ISING, 32, T, (1.0,), SEED, 0, bits0, MIXED)
    straight.run(12, precision=MIXED)
    split = ctx.new_job(mid, ISING, 32, T, (1.0,), SEED, 0, bits0, MIXED)
    split.run(5, precision=MIXED).run(7, precision=MIXED)
    a, b = _snapshot(straight), _snapshot(split)
    np.testing.assert_array_equal(a["bits"], b["bits"])
    np.testing.assert_array_equal(a["acc"], b["acc"])
    np.testing.assert_array_equal(a["sums"], b["sums"])      # sums continue in place
    # checkpoint after 5 proposals, restore into a fresh job, continue 7
    first = ctx.new_job(mid, ISING, 32, T, (1.0,), SEED, 0, bits0, MIXED)
    first.run(5, precision=MIXED)
    ck_bits, ck_step = first.state()
    assert ck_step == 5
    sums5, acc5, _ = first.observables()
    resumed = ctx.new_job(mid, ISING, 32, T, (1.0,), SEED, 0, wl.pack_bits(wl.random_lattices(12, 32, seed=9)), MIXED)
    resumed.write_state(ck_bits, ck_step)
    resumed.run(7, precision=MIXED)
    r = _snapshot(resumed)
    assert r["step"] == 12
    np.testing.assert_array_equal(r["bits"], a["bits"])
    np.testing.assert_array_equal(r["acc"] + acc5, a["acc"])
    np.testing.assert_allclose(r["sums"] + sums5, a["sums"], rtol=1e-12)
    # restoring with the mixed evaluation (FP32 F with its bound) continues identically
    resumed_m = ctx.new_job(mid, ISING, 32, T, (1.0,), SEED, 0, bits0, MIXED)
    resumed_m.write_state(ck_bits, ck_step, MIXED)
    resumed_m.run(7, precision=MIXED)
    rm = _snapshot(resumed_m)
    np.testing.assert_array_equal(rm["bits"], a["bits"])
    np.testing.assert_array_equal(rm["acc"] + acc5, a["acc"])
    for j in (straight, split, first, resumed, resumed_m):
        j.release()


@pytest.mark.parametrize("prec", [0, 1])
def test_write_states_equals_write_state_job_by_job(ctx, prec):
    """crbm_write_states (several jobs, one evaluation launch) leaves every job
    exactly as crbm_write_state does job by job -- jobs of several sides, an
    empty job and a Kitaev job of another filter shape in one call -- and the
    chains then continue identically; a repeated job id is rejected."""
    from paper_2008_05401_gb300 import ISING, KITAEV, CrbmError
    mid = _ising_model(ctx)
    W, hb, vb = wl.gaussian_crbm(4, 3, 0.05, seed=5)
    kid = ctx.load_model(KITAEV, W, vb, hb)
    specs = [(mid, ISING, 16, 40, (1.0,)), (mid, ISING, 64, 9, (1.0,)), (mid, ISING, 8, 0, (1.0,)),
             (kid, KITAEV, 4, 10, (1.0, 1.0, 1.0))]

    def make(seed):
        out = []
        for m, kind, L, n, J in specs:
            T = wl.ising_ladder(n, 4) if kind == ISING else wl.kitaev_ladder(n, 24)
            out.append(ctx.new_job(m, kind, L, T, J, SEED, 100, wl.pack_bits(wl.random_lattices(n, L, seed=seed)),
                                   prec))
        return out

    a, b = make(1), make(1)
    new_bits = [wl.pack_bits(wl.random_lattices(n, L, seed=L + 50)) for _, _, L, n, _ in specs]
    steps = [7, 3, 0, 11]
    ctx.write_states(a, new_bits, steps, prec)
    for j, bits, st in zip(b, new_bits, steps):
        j.write_state(bits, st, prec)
    for ja, jb in zip(a, b):
        sa, sb = _snapshot(ja), _snapshot(jb)
        for key in sa:
            np.testing.assert_array_equal(sa[key], sb[key], err_msg=key)
    for ja, jb in zip(a, b):
        ja.run(4, precision=prec)
        jb.run(4, precision=prec)
        sa, sb = _snapshot(ja), _snapshot(jb)
        for key in sa:
            np.testing.assert_array_equal(sa[key], sb[key], err_msg=key)
    with pytest.raises(CrbmError):
        ctx.write_states([a[0], a[0]], [new_bits[0], new_bits[0]], [1, 1], prec)
    for j in a + b:
        j.release()


def test_read_states_equals_job_by_job_reads(ctx):
    """crbm_read_states returns every job's lattices, step counter and
    observable sums as crbm_read_state and crbm_read_observables do, for jobs
    of several sides and an empty one; None entries are skipped."""
    from paper_2008_05401_gb300 import ISING, MIXED, NOBS
    mid = _ising_model(ctx)
    specs = [(16, 40), (64, 9), (8, 0), (32, 12)]
    jobs = [ctx.new_job(mid, ISING, L, wl.ising_ladder(n, 4), (1.0,), SEED, 0,
                        wl.pack_bits(wl.random_lattices(n, L, seed=L)), MIXED) for L, n in specs]
    ctx.run_batch(jobs, 5, precision=MIXED)
    bits = [np.empty((n, (L * L + 31) // 32), dtype=np.uint32) for L, n in specs]
    sums = [np.empty((n, NOBS)) for _, n in specs]
    bits[3] = None
    steps = ctx.read_states(jobs, bits, sums)
    for q, j in enumerate(jobs):
        b, st = j.state()
        assert steps[q] == st == 5
        if bits[q] is not None:
            np.testing.assert_array_equal(bits[q], b)
        np.testing.assert_array_equal(sums[q], j.observables()[0])
    for j in jobs:
        j.release()


def test_empty_job_and_zero_steps(ctx):
    from paper_2008_05401_gb300 import FP64, ISING, KITAEV
    mid = _ising_model(ctx)
    empty = ctx.new_job(mid, ISING, 16, np.zeros(0), (1.0,), SEED)
    empty.run(10)
    bits, step = empty.state()
    assert bits.shape == (0, 8) and step == 10
    empty.release()
    job = ctx.new_job(mid, ISING, 16, np.full(3, 2.0), (1.0,), SEED, 0, None, FP64)
    s0 = _snapshot(job)
    job.run(0)
    s1 = _snapshot(job)
    for key in s0:
        np.testing.assert_array_equal(s0[key], s1[key])
    job.release()
    # kernel as large as the lattice (k = L) on both models
    W, hb, vb = wl.gaussian_crbm(2, 3, 0.3)
    for kind, J in ((ISING, (1.0,)), (KITAEV, (1.0, 1.0, 1.0))):
        m = ctx.load_model(kind, W, vb, hb)
        j = ctx.new_job(m, kind, 3, np.full(2, 0.7), J, SEED)
        j.run(3)
        assert j.state()[1] == 3
        j.release()


def test_errors_are_reported_and_context_survives(ctx):
    from paper_2008_05401_gb300 import FP64, ISING, KITAEV, CrbmError, binding
    mid = _ising_model(ctx)
    h = ctx.h

    def code(fn, *a):
        with pytest.raises(CrbmError) as e:
            fn(*a)
        return e.value.code

    assert code(binding.crbm_load_model, h, 7, np.zeros((1, 2, 2)), 0.0, np.zeros(1)) == -1
    assert code(binding.crbm_load_model, h, ISING, np.zeros((9, 2, 2)), 0.0, np.zeros(9)) == -1
    assert code(binding.crbm_load_model, h, ISING, np.zeros((1, 8, 8)), 0.0, np.zeros(1)) == -1
    assert code(binding.crbm_load_model, h, ISING, np.full((1, 2, 2), np.nan), 0.0, np.zeros(1)) == -1
    import torch
    mem = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    T = np.full(4, 2.0)
    args = (h, mid, 16, T, (1.0,), SEED, 0, None, mem.data_ptr(), mem.numel())
    assert code(binding.crbm_init_chains, h, 99, *args[2:]) == -1                   # bad model id
    assert code(binding.crbm_init_chains, h, mid, 48, *args[3:]) == -1               # L unsupported
    assert code(binding.crbm_init_chains, h, mid, 4, *args[3:]) == -1                # k = 5 > L = 4
    assert code(binding.crbm_init_chains, h, mid, 16, np.array([2.0, 0.0, 1.0, 1.0]), *args[4:]) == -1
    assert code(binding.crbm_init_chains, h, mid, 16, T, (1.0,), SEED, 2 ** 32 - 2, None,
                mem.data_ptr(), mem.numel()) == -1                                    # chain ids past 2^32
    assert code(binding.crbm_init_chains, h, mid, 16, T, (1.0,), SEED, 0, None, mem.data_ptr(), 1024) == -2
    assert code(binding.crbm_init_chains, h, mid, 16, T, (1.0,), SEED, 0, None, mem.data_ptr() + 8,
                mem.numel() - 8) == -1                                                # misaligned
    job = ctx.new_job(mid, ISING, 16, T, (1.0,), SEED, 0, None, FP64, mem=mem)
    assert code(binding.crbm_run, h, job.id, -1) == -1
    assert code(binding.crbm_run, h, job.id, 1, 0) == -1                             # g = 0
    assert code(binding.crbm_run, h, 12345, 1) == -1
    W, hb, vb = wl.gaussian_crbm(4, 5, 0.1)
    kid = ctx.load_model(KITAEV, W, vb, hb)
    kj = ctx.new_job(kid, KITAEV, 6, np.full(2, 0.5), (1.0, 1.0, 1.0), SEED)
    assert code(binding.crbm_run_batch, h, [job.id, kj.id], 1) == -1                 # mixed kinds
    assert code(binding.crbm_run_batch, h, [job.id, job.id], 1) == -1                # repeated job
    assert "batch" in binding.crbm_last_error(h) or "twice" in binding.crbm_last_error(h)
    # the context still works
    job.run(3)
    assert job.state()[1] == 3
    job.release()
    kj.release()
    assert code(binding.crbm_read_state, h, job.id, 4, 16) == -1                     # released


def test_hbm_budget_admission():
    from paper_2008_05401_gb300 import ISING, Context, CrbmError, crbm_job_bytes
    need = crbm_job_bytes(ISING, 64, 100)
    c = gpu_ctx()
    c.close()
    ctx = Context(0, hbm_budget_bytes=int(2.5 * need))
    mid = _ising_model(ctx)
    a = ctx.new_job(mid, ISING, 64, np.full(100, 2.0), (1.0,), SEED)
    b = ctx.new_job(mid, ISING, 64, np.full(100, 2.0), (1.0,), SEED, 100)
    with pytest.raises(CrbmError) as e:
        ctx.new_job(mid, ISING, 64, np.full(100, 2.0), (1.0,), SEED, 200)
    assert e.value.code == -2
    a.release()
    c3 = ctx.new_job(mid, ISING, 64, np.full(100, 2.0), (1.0,), SEED, 200)   # admitted after release
    b.release()
    c3.release()
    ctx.close()


def test_run_on_a_side_stream(ctx):
    import torch
    from paper_2008_05401_gb300 import ISING, MIXED
    mid = _ising_model(ctx)
    bits0 = wl.pack_bits(wl.random_lattices(16, 16, seed=1))
    ref = ctx.new_job(mid, ISING, 16, np.full(16, 2.5), (1.0,), SEED, 0, bits0, MIXED)
    ref.run(9, precision=MIXED)
    side = torch.cuda.Stream()
    job = ctx.new_job(mid, ISING, 16, np.full(16, 2.5), (1.0,), SEED, 0, bits0, MIXED)
    job.run(9, precision=MIXED, stream=side)
    np.testing.assert_array_equal(job.state()[0], ref.state()[0])
    job.release()
    ref.release()


@pytest.mark.parametrize("kind", [0, 1])
def test_cuda_graph_replay_equals_direct_runs(ctx, kind):
    """A captured graph of 3 batched runs replayed twice continues the chains
    exactly like 6 direct runs (device-resident step counters)."""
    from paper_2008_05401_gb300 import KITAEV, MIXED, CrbmError
    if kind == 0:
        mid = _ising_model(ctx)
        spec, J = [(16, 8, 0), (32, 3, 100)], (1.0,)
    else:
        W, hb, vb = wl.gaussian_crbm(4, 3, 0.05, seed=4)
        mid = ctx.load_model(KITAEV, W, vb, hb)
        spec, J = [(4, 5, 0), (10, 2, 100)], (1.0, 1.0, 1.0)

    def make():
        return [ctx.new_job(mid, kind, L, wl.ising_ladder(n, 4) if kind == 0 else wl.kitaev_ladder(n, 24), J,
                            SEED, base, wl.pack_bits(wl.random_lattices(n, L, seed=L)), MIXED)
                for L, n, base in spec]

    graphed, direct = make(), make()
    gr = ctx.graph(graphed, 4, precision=MIXED, repeats=3)
    gr.launch()
    gr.launch()
    for _ in range(6):
        ctx.run_batch(direct, 4, precision=MIXED)
    with pytest.raises(CrbmError) as e:
        graphed[0].release()
    assert e.value.code == -5                                   # job of a live graph
    for a, b in zip(graphed, direct):
        sa, sb = _snapshot(a), _snapshot(b)
        assert sa["step"] == 24
        for key in sa:
            np.testing.assert_array_equal(sa[key], sb[key], err_msg=key)
    gr.destroy()
    for j in graphed + direct:
        j.release()


def test_autotuned_tile_shape_keeps_parity(ctx):
    """crbm_tune picks chains-per-CTA by timing; jobs created afterwards use it
    and still reproduce the oracle bit for bit."""
    from _common import decisions_are_clear, oracle_chains, run_oracle
    from paper_2008_05401_gb300 import ISING, MIXED
    W, hb, vb = wl.gaussian_crbm(4, 5, 0.2, seed=8)
    mid = ctx.load_model(ISING, W, vb, hb)
    nc, us = ctx.tune(mid, 16, MIXED)
    assert nc in (1, 2, 4, 8, 16, 32) and us > 0
    n, L, S = 37, 16, 6
    T = wl.ising_ladder(n, 8)
    bits0 = wl.pack_bits(wl.random_lattices(n, L, seed=44))
    job = ctx.new_job(mid, ISING, L, T, (1.0,), SEED, 0, bits0, MIXED)
    job.run(S, precision=MIXED)
    ref = oracle_chains("ising", W, hb, vb, L, T, (1.0,), SEED, n, bits0)
    worst = run_oracle(ref, S)
    if decisions_are_clear(worst):
        np.testing.assert_array_equal(job.state()[0], wl.pack_bits(ref.v))
        np.testing.assert_array_equal(job.observables()[1], ref.accepts)
    job.release()
