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
