"""Write the stored expected values under tests/golden/ (run from the repo root:
``python tests/golden/make_golden.py``).

The paper prints no worked numerical example of the method (its tables are
timings and its results are plots), so these fixtures are regression values of
the oracle, written by this script from ``oracle/`` alone, on small seeded
inputs that the fixtures store in full.  ``tests/test_golden.py`` checks that
the oracle still reproduces them (CPU) and that the CUDA path's FP64
evaluation of the same lattices agrees (GPU).  Each fixture names the
passages it follows.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import chain, crbm, ising, kitaev, philox  # noqa: E402


def lattice_rows(v):
    return ["".join(str(int(b)) for b in row) for row in v]


def crbm_params(rng, K, k, std):
    return rng.normal(0.0, std, (K, k, k)), rng.normal(0.0, std, K), float(rng.normal(0.0, std))


def model_fixture(model, name, cite, cases, K, k, std, seed):
    rng = np.random.default_rng(seed)
    W, hb, vb = crbm_params(rng, K, k, std)
    out = {"cite": cite, "model": name, "W": W.tolist(), "h_bias": hb.tolist(), "v_bias": vb, "cases": []}
    for L, n, J, T in cases:
        v = (rng.random((n, L, L)) < 0.5).astype(np.uint8)
        Tn = np.full(n, T) if np.isscalar(T) else np.asarray(T, dtype=np.float64)
        F = crbm.free_energy(v, W, hb, vb)
        lp, E, _ = chain.target(model, v, 1.0 / Tn, J)
        out["cases"].append({"L": L, "J": list(J), "T": Tn.tolist(),
                             "lattices": [lattice_rows(x) for x in v],
                             "F": F.tolist(), "log_pi": lp.tolist(), "E": E.tolist()})
    return out


def main():
    fixtures = {}
    fixtures["ising_crbm.json"] = model_fixture(
        chain.ISING, "ising",
        "Eq. (13) CRBM free energy with periodic convolutions (Sec. II); Eq. (14) Ising energy, "
        "log pi = -beta E (Sec. III)",
        [(4, 4, (1.0,), [1.5, 2.269, 3.0, 3.5]), (6, 3, (1.0,), [2.0, 2.269, 2.6])],
        K=2, k=3, std=0.3, seed=20080541)
    fixtures["kitaev_crbm.json"] = model_fixture(
        chain.KITAEV, "kitaev",
        "Eq. (13) CRBM free energy; Sec. IV: Majorana hopping matrix of Eq. (16) in the Z2 gauge "
        "eta, log pi = sum_l log 2cosh(beta eps_l / 2), e = -sum_l (eps_l / 2) tanh(beta eps_l / 2)",
        [(3, 3, (0.8, 1.1, 1.3), [0.005, 0.1, 1.0]), (4, 3, (1.0, 1.0, 1.0), [0.01, 0.2, 1.0])],
        K=2, k=3, std=0.1, seed=20080542)
    # App. C: the analytic CRBM of the Ising model at T_c = 2 / ln(1 + sqrt 2) (Sec. III)
    beta = np.log(1.0 + np.sqrt(2.0)) / 2.0
    W, hb, vb = ising.analytic_crbm(beta, k=2)
    states = ising.all_states(3)
    diff = crbm.free_energy(states, W, hb, vb) - beta * ising.energy(states)
    fixtures["analytic_crbm_Tc.json"] = {
        "cite": "App. C, Eqs. (C1)-(C5): kernels [[W,0],[W,0]] and [[W,W],[0,0]], h_bias and v_bias "
                "from W; T_c = 2 / ln(1 + sqrt 2) (Sec. III)",
        "beta": beta, "W": W.tolist(), "h_bias": hb.tolist(), "v_bias": vb,
        "F_minus_beta_E_L3": float(diff.mean()), "F_minus_beta_E_L3_spread": float(diff.max() - diff.min())}
    # Philox4x32-10 words of the oracle's generator (counter (q, tag, step, chain), key from the seed)
    rows = []
    for seed, cid, step, tag in ((0, 0, 0, 0), (2008054010, 7, 3, 5), (1, 4095, 1000, 0xFFFFFFFB),
                                 (2 ** 63 - 1, 2 ** 32 - 1, 2 ** 32 - 1, 17)):
        w = philox.words(seed, np.array([cid], dtype=np.uint64), step, tag, 8)[0]
        rows.append({"seed": seed, "chain": cid, "step": step, "tag": tag, "words": [int(x) for x in w]})
    fixtures["philox_words.json"] = {
        "cite": "Philox4x32-10 (Salmon et al., SC'11); the paper names no generator: words n = 0..7 of "
                "one chain, counter (n / 4, tag, step, chain)",
        "rows": rows}
    for name, obj in fixtures.items():
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(obj, f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main()
