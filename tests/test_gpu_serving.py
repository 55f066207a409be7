"""Continuous batching: results are the same alone and in the mix; admission
waits for HBM; groups of different model kinds, and two batches of one group,
overlap on separate streams (CUDA event timestamps of the launches)."""
import numpy as np
import pytest

from _common import gpu_ctx

pytestmark = pytest.mark.gpu


def _requests(n, seed, max_proposals=300):
    from paper_2008_05401_gb300.serving import synthetic_requests
    return synthetic_requests(n, rate_hz=2000.0, seed=seed, min_proposals=20, max_proposals=max_proposals,
                              precision=1)


def _same(a, b):
    np.testing.assert_array_equal(a.bits, b.bits)
    assert a.step == b.step
    np.testing.assert_array_equal(a.sums, b.sums)
    np.testing.assert_array_equal(a.accepts, b.accepts)
    np.testing.assert_array_equal(a.logpi, b.logpi)


def test_each_result_same_alone_and_in_the_mix():
    gpu_ctx().close()
    from paper_2008_05401_gb300.serving import Server
    reqs = _requests(24, seed=5)
    srv = Server(quantum=37)                     # odd quantum: every job is split unevenly
    mixed = srv.run(reqs, realtime=True)
    st = srv.stats()
    srv.close()
    assert st["requests"] == 24 and st["p99_latency_s"] >= st["p50_latency_s"]
    for r in _requests(24, seed=5)[:8]:
        alone_srv = Server(quantum=10 ** 6)      # one launch for the whole job
        alone = alone_srv.run([r], realtime=False)
        alone_srv.close()
        _same(alone[r.rid], mixed[r.rid])


def test_admission_waits_for_memory():
    gpu_ctx().close()
    from paper_2008_05401_gb300 import crbm_job_bytes
    from paper_2008_05401_gb300.serving import Server
    reqs = _requests(10, seed=9, max_proposals=100)
    biggest = max(crbm_job_bytes(r.kind, r.L, len(r.T)) for r in reqs)
    srv = Server(hbm_budget_bytes=int(1.5 * biggest), quantum=50)
    res = srv.run(reqs, realtime=False)
    srv.close()
    assert len(res) == 10
    # never more than the budget allows at once: at least one request had to wait
    assert max(r.admitted for r in res.values()) > min(r.finished for r in res.values())


def test_a_failing_request_fails_alone():
    """Host-side fault injection: malformed requests (unsupported lattice side,
    non-positive temperature, larger than the whole HBM budget) are reported
    and dropped; every other request completes with its exact result."""
    gpu_ctx().close()
    from paper_2008_05401_gb300.serving import Server
    reqs = _requests(8, seed=21, max_proposals=60)
    bad_L = _requests(1, seed=22)[0]
    bad_L.rid, bad_L.kind, bad_L.L = 100, 0, 48
    bad_T = _requests(1, seed=23)[0]
    bad_T.rid = 101
    bad_T.T = np.zeros(len(bad_T.T))
    srv = Server(quantum=16)
    res = srv.run(reqs + [bad_L, bad_T], realtime=False)
    assert set(srv.failed) == {100, 101}
    assert set(res) == {r.rid for r in reqs}
    srv.close()
    too_big = _requests(1, seed=24)[0]
    small = Server(hbm_budget_bytes=1024)
    small.run([too_big], realtime=False)
    assert too_big.rid in small.failed and "budget" in small.failed[too_big.rid]
    small.close()
    ref_srv = Server(quantum=10 ** 6)
    ref = ref_srv.run(_requests(8, seed=21, max_proposals=60)[:2], realtime=False)
    ref_srv.close()
    for rid in ref:
        _same(ref[rid], res[rid])


def test_launches_of_different_groups_and_of_one_group_overlap():
    """The Ising and Kitaev groups run on their own streams, and each group
    keeps a second batch in flight for jobs that are not in its first: the
    device-side intervals [start, end] of launches of the two groups intersect,
    and so do those of two batches of one group."""
    gpu_ctx().close()
    from paper_2008_05401_gb300.serving import Server
    reqs = _requests(24, seed=5, max_proposals=300)
    for r in reqs[12:]:
        r.arrival += 0.05                         # a second wave arrives while the first runs
    srv = Server(quantum=37)
    srv.run(reqs, realtime=True)
    iv = srv.launch_intervals()
    srv.close()
    assert {key[0] for key, _, _, _ in iv} == {0, 1}

    def meet(a, b):
        return a[2] < b[3] and b[2] < a[3]

    assert any(meet(a, b) for a in iv for b in iv if a[0][0] != b[0][0])
    assert any(meet(a, b) for a in iv for b in iv if a[0] == b[0] and a[1] != b[1])
