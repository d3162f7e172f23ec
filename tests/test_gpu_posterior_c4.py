"""Configuration 4 (four qubits) over a long run: 1024 chains x 1000 steps with the paper's
adaptation (M_A = 500) and the first 500 steps left out of the pool, on the GPU and in the
FP64 oracle.  The pooled posterior means of Eq. BME2 must agree element by element within
three Monte Carlo standard errors (jackknife over 32 groups of 32 independent chains, from
the oracle's per-chain sums), and so must their fidelities to the true state (Eq. fid).
The oracle takes about half a minute for this on the GPU host's cores.
"""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W

pytestmark = pytest.mark.gpu

R, S, BURN, GROUPS = 1024, 1000, 500, 32


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_four_qubit_long_run_pooled_mean_matches_oracle(qst, oracle_mod, cuda_ok, prec):
    prob = W.config_problem(4, num_chains=R, num_steps=S)
    p = {"bf16x3": qst.PREC_BF16X3, "fp32": qst.PREC_FP32}[prec]
    s = qst.Sampler(prob, precision=p, diag_chains=0, burn_in=BURN, adapt_interval=500)
    s.run_chains(S)
    rho, n = s.posterior_mean()
    st = s.get_state()
    s.close()
    ref = oracle_mod.run(prob, num_steps=S, want_chain_pool=True, want_final=True, burn_in=BURN, adapt_interval=500)
    kept = S - BURN
    assert n == ref["num_pooled"] == R * kept
    groups = ref["chain_pool"].reshape(GROUPS, R // GROUPS, 16, 16).sum(axis=1)
    total = groups.sum(axis=0)
    loo = (total[None] - groups) / ((R - R // GROUPS) * kept)      # leave-one-group-out means
    se = np.sqrt((GROUPS - 1) / GROUPS * (np.abs(loo - loo.mean(axis=0)) ** 2).sum(axis=0))   # |.|^2: complex entries
    assert np.all(np.abs(rho - ref["mean"]) <= 3 * se + 1e-9), np.max(np.abs(rho - ref["mean"]) / (se + 1e-30))
    f_loo = np.array([oracle_mod.fidelity(m, prob.truth) for m in loo])
    se_f = np.sqrt((GROUPS - 1) / GROUPS * ((f_loo - f_loo.mean()) ** 2).sum())
    f_gpu = oracle_mod.fidelity(rho, prob.truth)
    f_ref = oracle_mod.fidelity(ref["mean"], prob.truth)
    assert abs(f_gpu - f_ref) <= 3 * se_f, (f_gpu, f_ref, se_f)
    # the chains moved towards the data: the pooled mean is closer to the truth than the
    # maximally mixed state is
    assert f_gpu > oracle_mod.fidelity(np.eye(16) / 16, prob.truth)
    # and adapted their step size on the same schedule as the oracle's
    assert np.allclose(np.sort(st["beta"]), np.sort(ref["final_beta"]), rtol=0, atol=1e-12)
