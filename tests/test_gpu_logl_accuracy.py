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
