"""The pooled mean (Eq. BME2) summed over many accept CTAs, each with its own FP64 pool slot:
at two and four qubits (128 chains per CTA) and at five and six qubits (as few as 8), each
with a ragged last CTA.  With a single kept step (thinning 1, burn-in S - 1) the pooled
mean is the mean over the chains of their current rho, which the test forms independently
of the pool: from the chains' own latent states, read back and passed through the
evaluation entry point."""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W
from tests._helpers import unpack_rho

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("q,R", [(2, 3001), (4, 1000), (5, 2001), (6, 300)])
def test_pooled_mean_over_many_accept_ctas(qst, cuda_ok, q, R):
    import torch
    S = 4
    if q <= 4:
        prob = W.config_problem(q, num_chains=R, num_steps=S)   # configurations 2 and 4
    else:
        make = W.five_qubit_problem if q == 5 else W.six_qubit_problem
        prob = make(num_chains=R, num_steps=S)
    assert prob.dim == 1 << q
    s = qst.Sampler(prob, precision=qst.PREC_PAULI, diag_chains=0, thin=1, burn_in=S - 1)
    s.run_chains(S)
    mean, n = s.posterior_mean()
    st = s.get_state()
    rho_p, _, _ = s.evaluate(torch.from_numpy(st["y"]).cuda(), want_p=False)
    torch.cuda.synchronize()
    s.close()
    assert n == R
    assert st["accepts"].sum() > 0          # some chains hold an accepted proposal
    rho = unpack_rho(rho_p.cpu().numpy().astype(np.float64), 1 << q).mean(axis=0)
    # entries ~1/D; the stored states are FP32 and re-scaled by 1/Tr at accept
    assert np.abs(mean - rho).max() < 1e-6
    assert abs(np.trace(mean).real - 1) < 1e-6
