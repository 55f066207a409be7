"""Stored expected values of tests/golden/ (written by tests/golden/make_golden.py
from the oracle alone; the paper prints no worked numerical example of the
method).  CPU: the oracle still reproduces them.  GPU: the CUDA path's FP64
evaluation of the stored lattices (through the C ABI, at job creation) agrees
with the stored F (Eq. 13), log pi and E (Eq. 14; Sec. IV) to 1e-10.
"""
import json
import os

import numpy as np
import pytest

import crbm_workloads as wl
from _common import ROOT, gpu_ctx

GOLDEN = os.path.join(ROOT, "tests", "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def lattices(case):
    return np.array([[[int(c) for c in row] for row in lat] for lat in case["lattices"]], dtype=np.uint8)


def params(fx):
    return np.array(fx["W"]), np.array(fx["h_bias"]), float(fx["v_bias"])


@pytest.mark.parametrize("name", ["ising_crbm.json", "kitaev_crbm.json"])
def test_oracle_reproduces_model_fixture(name):
    from oracle import chain, crbm
    fx = load(name)
    W, hb, vb = params(fx)
    model = chain.ISING if fx["model"] == "ising" else chain.KITAEV
    for case in fx["cases"]:
        v = lattices(case)
        T = np.array(case["T"])
        F = crbm.free_energy(v, W, hb, vb)
        lp, E, _ = chain.target(model, v, 1.0 / T, tuple(case["J"]))
        np.testing.assert_allclose(F, case["F"], rtol=1e-13, atol=1e-12)
        np.testing.assert_allclose(lp, case["log_pi"], rtol=1e-13, atol=1e-12)
        np.testing.assert_allclose(E, case["E"], rtol=1e-13, atol=1e-12)


def test_oracle_reproduces_analytic_crbm_fixture():
    """App. C at T_c: the stored kernels, and F - beta E the same constant for
    all 512 lattices of L = 3."""
    from oracle import crbm, ising
    fx = load("analytic_crbm_Tc.json")
    beta = fx["beta"]
    assert beta == pytest.approx(np.log(1.0 + np.sqrt(2.0)) / 2.0, rel=1e-15)
    W, hb, vb = ising.analytic_crbm(beta, k=2)
    np.testing.assert_allclose(W, fx["W"], rtol=1e-14)
    np.testing.assert_allclose(hb, fx["h_bias"], rtol=1e-14)
    assert vb == pytest.approx(fx["v_bias"], rel=1e-14)
    s = ising.all_states(3)
    d = crbm.free_energy(s, W, hb, vb) - beta * ising.energy(s)
    assert d.max() - d.min() < 1e-12
    assert d.mean() == pytest.approx(fx["F_minus_beta_E_L3"], rel=1e-13)


def test_oracle_reproduces_philox_fixture():
    from oracle import philox
    for row in load("philox_words.json")["rows"]:
        w = philox.words(row["seed"], np.array([row["chain"]], dtype=np.uint64), row["step"], row["tag"], 8)[0]
        assert [int(x) for x in w] == row["words"]


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["ising_crbm.json", "kitaev_crbm.json"])
def test_cuda_path_matches_stored_values(name):
    from paper_2008_05401_gb300 import FP64, ISING, KITAEV, MIXED
    ctx = gpu_ctx()
    try:
        fx = load(name)
        W, hb, vb = params(fx)
        kind = ISING if fx["model"] == "ising" else KITAEV
        mid = ctx.load_model(kind, W, vb, hb)
        for case in fx["cases"]:
            L, T, J = case["L"], np.array(case["T"]), tuple(case["J"])
            bits = wl.pack_bits(lattices(case))
            for prec in (FP64, MIXED):
                job = ctx.new_job(mid, kind, L, T, J, 1, 0, bits, prec)
                lp, F, E = job.energies()
                np.testing.assert_allclose(F, case["F"], rtol=1e-10, atol=1e-10)
                np.testing.assert_allclose(lp, case["log_pi"], rtol=1e-10, atol=1e-9)
                np.testing.assert_allclose(E, case["E"], rtol=1e-10, atol=1e-9)
                np.testing.assert_array_equal(job.state()[0], bits)
                job.release()
    finally:
        ctx.close()
