"""The Sec. IV study on the GPU (paper_2501_17334_gb300.experiment), at a small size."""
import csv
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_bures_truth_is_algorithm_1_of_the_seeded_latent(qst, oracle_mod, cuda_ok, q):
    from paper_2501_17334_gb300 import experiment as E, workload as W
    seed = 123 + q
    rho = E.bures_truth(q, seed)
    D = 1 << q
    x = np.random.default_rng(seed).standard_normal((1, 4 * D * D)).astype(np.float32).astype(np.float64)
    prob = W.config_problem(q, num_chains=8)
    ref, _, _ = oracle_mod.evaluate(prob, x, want_p=False)
    assert np.abs(rho - ref[0]).max() < 2e-6
    assert abs(np.trace(rho).real - 1.0) < 1e-12
    assert np.linalg.eigvalsh(rho).min() > -1e-6


def test_paper_problem_has_the_sec4_shots(qst, cuda_ok):
    from paper_2501_17334_gb300 import experiment as E
    for q in (1, 3):
        p = E.paper_problem(q, 16)
        per_setting = p.counts.reshape(3 ** q, 1 << q).sum(axis=1)
        assert np.all(per_setting == 25 * (1 << q))


def test_small_sweep_writes_consistent_rows(qst, cuda_ok, tmp_path):
    from paper_2501_17334_gb300 import experiment as E
    rows = E.sweep([1, 2], [0, 2], [1, 8], 256, str(tmp_path))
    for name in ("acf", "tau", "frob", "fidelity"):
        assert os.path.getsize(tmp_path / f"{name}.csv") > 0
    frob = {(q, t, r): (ne, e) for q, t, r, ne, e in rows["frob"]}
    fid = {(q, t, r): f for q, t, r, _, f in rows["fidelity"]}
    for q in (1, 2):
        assert frob[(q, 4, 8)][1] == 0.0                 # the reference pool itself
        assert abs(fid[(q, 4, 8)]) < 1e-7                # F(rho, rho) = 1 to the eigensolver's round-off
        for key, (ne, e) in frob.items():
            assert np.isfinite(e) and e >= 0.0
            assert np.isnan(ne) or ne > 0.0                  # undefined where tau <= 0
    acf = [r for r in rows["acf"] if r[2] == 0]
    assert all(abs(c - 1.0) < 1e-12 for *_, c in acf)     # c[0] = 1 by normalisation
    with open(tmp_path / "tau.csv") as f:
        taus = [float(r["tau_mean"]) for r in csv.DictReader(f)]
    assert all(np.isfinite(t) for t in taus)


def test_sweep_points_recomputed_by_the_oracle(qst, oracle_mod, cuda_ok, tmp_path):
    """eps_F^2 (Eq. fro) and 1 - F (Eq. fid) of a small sweep, Q = 1, T in {1, 2}, R in {1, 8},
    against the same quantities of the oracle's chains on the same data, seed and chain ids.

    Every accept decision of those chains lies at least 1e-5 from its threshold in the oracle's
    own trace (asserted below), far outside the GPU's log L error at one qubit, so the two chain
    sets agree step for step and their pooled means differ only by FP32 rounding of rho."""
    from paper_2501_17334_gb300 import experiment as E
    keep, chains, thins = 256, (1, 8), (1, 2)
    rows = E.sweep([1], [0, 1], list(chains), keep, str(tmp_path))
    prob = E.paper_problem(1, max(chains))
    means = {}
    for t in thins:
        r = oracle_mod.run(prob, num_chains=max(chains), num_steps=keep * t, thin=t, trace_steps=keep * t,
                           want_chain_pool=True)
        margin = np.abs(r["trace_log_alpha"] - (r["trace_logl_prop"] - r["trace_logl_cur"]))
        assert np.nanmin(margin[np.isfinite(margin)]) > 1e-5
        assert r["num_pooled"] == keep * max(chains)
        means[(t, max(chains))] = r["mean"]
        means[(t, 1)] = r["chain_pool"][0] / keep
    ref = means[(max(thins), max(chains))]
    frob = {(t, rr): e for q, t, rr, _, e in rows["frob"]}
    fid = {(t, rr): f for q, t, rr, _, f in rows["fidelity"]}
    for key, m in means.items():
        eps = E.frobenius_sq(m, ref)
        one_minus_f = 1.0 - E.fidelity(ref, m)
        assert abs(frob[key] - eps) <= 1e-6 * np.sqrt(eps) + 1e-12, (key, frob[key], eps)
        assert abs(fid[key] - one_minus_f) <= 1e-6, (key, fid[key], one_minus_f)
    assert frob[(1, 1)] > frob[(1, 8)] > 0.0   # one chain is further from the reference pool than eight
