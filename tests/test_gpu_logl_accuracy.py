"""log L against the FP64 oracle at four qubits, in absolute terms.

The benchmark's chain-steps/s are quoted at a log-likelihood error of at most 1e-3 absolute
(Eq. likelihood, about 81,000 shots: |log L| ~ 2 10^5).  The 1e-5 relative bar of
test_gpu_parity.py allows about 1 there; this file holds the absolute one, on the states the
chains actually visit (1024 chains of configuration 4, identical latent vectors on both
sides), for the mixed (BF16x3) and the plain FP32 form:

* after 2000 steps at least 99.5% of the chains are within 1e-3 of the oracle's log L and all
  within 1.5e-3;
* at the prior draws the chains start from (their log L lies ~10^4 below the posterior's, so
  the terms c_kl log p_kl are largest), at least 97% of the chains are within 1e-3 and all
  within 2.5e-3.

The other workloads' errors, as stated with the benchmark: configurations 1 and 2 and the
1-3 qubit problems of configuration 5 within 1e-3; its 4- and 5-qubit problems carry up to
4000 shots per basis, and its five-qubit U is first-order unless qr_passes 4 asks for the
refinement (the target is the four-qubit one).

With U refined to the exact factor, what remains is the FP32 rounding of W = (U + I) G, of
W W^dag and of the stored rho: a CPU emulation of the kernels' arithmetic puts the largest of
1024 chain states at 8-9e-4 after 2000 steps and 1.2e-3 at the prior draws, so a chain or two
per thousand can pass 1e-3 by a little, depending on the states the chains happen to visit.
An error of 1.5e-3 in the log-ratio changes an acceptance probability by at most 0.15% of
itself.  A refinement that fails (one first-order pass at cond(H) ~ 10^5 left 6e-3) exceeds
the caps.
"""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W

pytestmark = pytest.mark.gpu


def _logl_errors(s, oracle_mod, prob):
    import torch
    st = s.get_state()
    y = st["y"]
    _, _, ll = s.evaluate(torch.from_numpy(y).cuda(), want_rho=False, want_p=False)
    torch.cuda.synchronize()
    _, _, ll_ref = oracle_mod.evaluate(prob, y.astype(np.float64), want_rho=False, want_p=False)
    return np.abs(ll.cpu().numpy() - ll_ref)


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_four_qubit_logl_within_1e3_absolute(qst, oracle_mod, cuda_ok, prec):
    R = 1024
    prob = W.config_problem(4, num_chains=R, num_steps=2000)
    p = {"bf16x3": qst.PREC_BF16X3, "fp32": qst.PREC_FP32}[prec]
    s = qst.Sampler(prob, precision=p, diag_chains=0)
    e0 = _logl_errors(s, oracle_mod, prob)          # the prior draws y^0
    s.run_chains(2000)
    e = _logl_errors(s, oracle_mod, prob)
    s.close()
    assert np.all(np.isfinite(e0)) and np.all(np.isfinite(e))
    assert np.mean(e <= 1e-3) >= 0.995 and e.max() <= 1.5e-3, (prec, np.mean(e <= 1e-3), e.max(), np.median(e))
    assert np.mean(e0 <= 1e-3) >= 0.97 and e0.max() <= 2.5e-3, (prec, np.mean(e0 <= 1e-3), e0.max())


def _batch_errors(s, oracle_mod, probs, per_problem):
    """|log L - oracle| on per_problem chains of every problem of a handle, grouped by qubits."""
    import torch
    out = {}
    for i, p in enumerate(probs):
        y = s.get_state(i)["y"][np.linspace(0, p.num_chains - 1, per_problem).astype(np.int64)]
        _, _, ll = s.evaluate(torch.from_numpy(y).cuda(), problem=i, want_rho=False, want_p=False)
        torch.cuda.synchronize()
        _, _, ref = oracle_mod.evaluate(p, y.astype(np.float64), want_rho=False, want_p=False)
        out.setdefault(p.num_qubits, []).append(np.abs(ll.cpu().numpy() - ref))
    return {q: np.concatenate(v) for q, v in out.items()}


def test_small_configurations_logl_within_1e3(qst, oracle_mod, cuda_ok):
    """Configurations 1 and 2 (plain FP32 form) after their chains have run: every chain within
    1e-3 (measured: max 1.4e-4)."""
    for c, steps in ((1, 2000), (2, 1000)):
        prob = W.config_problem(c)
        s = qst.Sampler(prob, precision=qst.PREC_FP32, diag_chains=0)
        s.run_chains(steps)
        e = _batch_errors(s, oracle_mod, [prob], min(prob.num_chains, 1024))[prob.num_qubits]
        s.close()
        assert e.max() <= 1e-3, (c, e.max())


def test_heterogeneous_batch_logl_by_qubit_count(qst, oracle_mod, cuda_ok):
    """Configuration 5 (64 problems of 1-5 qubits, per-problem form) after 1000 steps, 32 chains
    of every problem: 1-3 qubits all within 1e-3; four qubits (up to 4x configuration 4's shots)
    at least 95% within 1e-3 and all within 2e-3; five qubits, whose U is first-order by default,
    at least 85% within 1e-3 and at least 90% with the refinement of U (qr_passes 4), which also
    lowers the largest error (measured: 89% / 95%, max 5.8e-3 / 3.2e-3)."""
    batch = W.heterogeneous_batch(64)
    errs = {}
    for qp in (3, 4):
        s = qst.Sampler(batch, precision=qst.PREC_AUTO, diag_chains=0, qr_passes=qp)
        s.run_chains(1000)
        errs[qp] = _batch_errors(s, oracle_mod, batch, 32)
        s.close()
    e = errs[3]
    for q in (1, 2, 3):
        assert e[q].max() <= 1e-3, (q, e[q].max())
    assert np.mean(e[4] <= 1e-3) >= 0.95 and e[4].max() <= 2e-3, (np.mean(e[4] <= 1e-3), e[4].max())
    assert np.mean(e[5] <= 1e-3) >= 0.85, np.mean(e[5] <= 1e-3)
    assert np.mean(errs[4][5] <= 1e-3) >= 0.90 and errs[4][5].max() < e[5].max()
