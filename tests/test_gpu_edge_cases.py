"""Degenerate and boundary cases of the CUDA path against the oracle.

* One chain: the tensor-core tile, the proposal CTA and the accept CTA each hold a single
  valid chain; at 1-4 qubits in the three forms, the first 200 decisions and the final state.
* A chain count one past a whole number of 128-chain tiles (the last tile holds one chain):
  the decisions of the chains on both sides of every tile boundary.
* beta0 = 1 with the adaptation off: sqrt(1 - beta^2) = 0, so y' = eta and the pCN proposal
  degenerates to independent draws from the prior; the first 200 decisions.
* Nothing pooled yet: zero steps run is a no-op and the posterior mean is refused with
  QST_ERR_STATE (qst.h).

Decisions may differ from the oracle's only at near ties, as in test_gpu_parity.py.
"""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W
from tests._helpers import near_tie_band

pytestmark = pytest.mark.gpu

PREC = ["fp32", "bf16x3", "pauli"]


def _prec(qst, name):
    return {"fp32": qst.PREC_FP32, "bf16x3": qst.PREC_BF16X3, "pauli": qst.PREC_PAULI}[name]


def _check_decisions(acc_gpu, ll_prop_gpu, ref, max_mismatch):
    """acc_gpu, ll_prop_gpu: [chains, steps]; the oracle's trace in ref."""
    acc_ref = ref["trace_accept"]
    margin = ref["trace_log_alpha"] - (ref["trace_logl_prop"] - ref["trace_logl_cur"])
    tol = near_tie_band(acc_gpu, acc_ref, ll_prop_gpu, ref["trace_logl_prop"])
    mism = 0
    for r in range(acc_ref.shape[0]):
        bad = np.nonzero(acc_gpu[r] != acc_ref[r])[0]
        if bad.size:
            assert abs(margin[r, bad[0]]) < tol, (r, bad[0], margin[r, bad[0]], tol)
            mism += 1
    assert mism <= max_mismatch, mism
    return np.all(acc_gpu == acc_ref, axis=1)


@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_one_chain(qst, oracle_mod, cuda_ok, prec, q):
    S = 200
    prob = W.config_problem(q, num_chains=1, num_steps=S)
    s = qst.Sampler(prob, precision=_prec(qst, prec), trace_steps=S, diag_chains=1)
    s.run_chains(S)
    acc, llp = s.get_trace()
    st = s.get_state()
    rho, n = s.posterior_mean()
    s.close()
    ref = oracle_mod.run(prob, num_steps=S, trace_steps=S, want_final=True)
    same = _check_decisions(acc.T, llp.T, ref, max_mismatch=1)
    assert n == ref["num_pooled"] == S
    if same[0]:
        assert np.abs(st["y"] - ref["final_y"]).max() < 1e-3
        assert np.abs(rho - ref["mean"]).max() < 1e-5   # the same S states, FP32 rho against FP64
    assert abs(np.trace(rho).real - 1.0) < 1e-6


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_last_tile_of_one_chain(qst, oracle_mod, cuda_ok, prec):
    """257 four-qubit chains: tiles of 128, 128 and 1 chain; the chains at every boundary."""
    R, S = 257, 60
    prob = W.config_problem(4, num_chains=R, num_steps=S)
    s = qst.Sampler(prob, precision=_prec(qst, prec), trace_steps=S, diag_chains=0)
    s.run_chains(S)
    acc, llp = s.get_trace()
    s.close()
    for c in (0, 127, 128, 255, 256):
        ref = oracle_mod.run(prob, num_chains=1, chain_begin=c, num_steps=S, trace_steps=S)
        _check_decisions(acc.T[c:c + 1], llp.T[c:c + 1], ref, max_mismatch=1)


@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("q", [2, 3])
def test_beta_one_proposes_independent_prior_draws(qst, oracle_mod, cuda_ok, prec, q):
    R, S = 256, 200
    prob = W.config_problem(q, num_chains=R, num_steps=S)
    prob.beta0 = 1.0
    s = qst.Sampler(prob, precision=_prec(qst, prec), trace_steps=S, diag_chains=0, adapt_interval=0)
    s.run_chains(S)
    acc, llp = s.get_trace()
    st = s.get_state()
    s.close()
    assert np.all(st["beta"] == 1.0)
    ref = oracle_mod.run(prob, num_steps=S, trace_steps=S, want_final=True, adapt_interval=0)
    same = _check_decisions(acc.T, llp.T, ref, max_mismatch=max(2, R // 50))
    assert np.abs(st["y"][same] - ref["final_y"][same]).max() < 1e-3


def test_nothing_pooled_yet(qst, cuda_ok):
    prob = W.config_problem(2, num_chains=64, num_steps=10)
    s = qst.Sampler(prob, precision=qst.PREC_FP32, diag_chains=0)
    s.run_chains(0)
    assert s.diagnostics()["steps_done"] == 0
    with pytest.raises(qst.QstError) as e:
        s.posterior_mean()
    assert e.value.status == 6   # QST_ERR_STATE
    s.run_chains(3)
    rho, n = s.posterior_mean()
    assert n == 3 * 64
    s.close()
