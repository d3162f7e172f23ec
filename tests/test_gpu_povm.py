"""General (non-Pauli) POVMs through the dense forms, against the FP64 oracle.

The method needs only the measurement operators Lambda_kl (Sec. III, Steps 1-4: p_kl =
Tr Lambda_kl rho and the multinomial likelihood), so a problem measured in other bases must
give the same rho, p, log L and accept decisions as the oracle's direct trace over the same
arrays.  Two families (workload.py): Haar-random bases of the whole register, whose packed
projectors are not exact in bf16 (the FP32 form), and products of entangled two-qubit bases
with dyadic entries (Bell, Bell with a phase i, a +-1/2 basis), exact in bf16, so that the
tensor-core form applies too.  Bars as in test_gpu_parity.py: rho 2e-6 and p 1e-6 on rows
with cond(H) <= 1e3; the FP64 reduction of the GPU's own p within sum_{c>0} c 6 2^-24; the
first 200 decisions identical except at a near tie.
"""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W
from tests._helpers import near_tie_band, unpack_rho
from tests.test_gpu_parity import _compare_decisions, _cond

pytestmark = pytest.mark.gpu

CASES = [("random", 2, "fp32"), ("random", 3, "fp32"), ("dyadic", 2, "fp32"), ("dyadic", 2, "bf16x3"),
         ("dyadic", 4, "fp32"), ("dyadic", 4, "bf16x3")]


def _problem(kind, q, num_chains=256, num_steps=200):
    if kind == "random":
        return W.random_basis_problem(q, num_settings=2 * (1 << q), num_chains=num_chains, num_steps=num_steps)
    return W.dyadic_basis_problem(q, num_chains=num_chains, num_steps=num_steps)


def _prec(qst, name):
    return {"fp32": qst.PREC_FP32, "bf16x3": qst.PREC_BF16X3}[name]


@pytest.mark.parametrize("kind,q,prec", CASES)
def test_general_povm_evaluate_matches_oracle(qst, oracle_mod, cuda_ok, kind, q, prec):
    import torch
    n = 600
    prob = _problem(kind, q, num_chains=1024)   # evaluate takes up to num_chains rows
    D = 1 << q
    s = qst.Sampler(prob, precision=_prec(qst, prec), diag_chains=0)
    x32 = W.latent_batch(n, q, seed=300 + q).astype(np.float32)
    rho_p, p_gpu, ll_gpu = s.evaluate(torch.from_numpy(x32).cuda())
    torch.cuda.synchronize()
    s.close()
    rho_gpu = unpack_rho(rho_p.cpu().numpy(), D)
    p_gpu = p_gpu.cpu().numpy().astype(np.float64)
    ll_gpu = ll_gpu.cpu().numpy()
    rho_ref, p_ref, ll_ref = oracle_mod.evaluate(prob, x32.astype(np.float64))
    ok = _cond(x32.astype(np.float64), D) <= 1e3
    assert ok.mean() > 0.95
    assert np.abs(rho_gpu - rho_ref).max(axis=(1, 2))[ok].max() < 2e-6
    assert np.abs(p_gpu - p_ref).max(axis=1)[ok].max() < 1e-6
    # each setting of these POVMs sums to the identity, so every setting's p sums to 1
    assert np.abs(p_gpu.reshape(n, -1, D).sum(-1) - 1.0).max() < 1e-5
    # the FP64 reduction of the GPU's own (per-setting renormalised) p
    pu = (p_gpu.reshape(n, -1, D) / p_gpu.reshape(n, -1, D).sum(-1, keepdims=True)).reshape(n, -1)
    ll_own = np.array([oracle_mod.loglik(prob.counts, pu[i]) for i in range(n)])
    fin = np.isfinite(ll_own)
    assert np.abs(ll_gpu[fin] - ll_own[fin]).max() < np.sum(prob.counts) * 6 * 2.0 ** -24
    rel = np.abs(ll_gpu - ll_ref) / np.abs(ll_ref)
    assert np.nanmax(rel[ok]) < 1e-5


@pytest.mark.parametrize("kind,q,prec", CASES)
def test_general_povm_first_200_decisions(qst, oracle_mod, cuda_ok, kind, q, prec):
    R = 256
    prob = _problem(kind, q, num_chains=R, num_steps=200)
    s = qst.Sampler(prob, precision=_prec(qst, prec), trace_steps=200, diag_chains=0)
    s.run_chains(200)
    acc_gpu, ll_prop_gpu = s.get_trace()
    s.close()
    ref = oracle_mod.run(prob, num_steps=200, trace_steps=200, want_final=True)
    margin = ref["trace_log_alpha"] - (ref["trace_logl_prop"] - ref["trace_logl_cur"])
    # a decision may differ only where the margin is within twice the measured log L error
    tol = near_tie_band(acc_gpu.T, ref["trace_accept"], ll_prop_gpu.T, ref["trace_logl_prop"])
    compared, mism = _compare_decisions(acc_gpu.T, ref["trace_accept"], margin, tol=tol)
    assert mism <= max(2, R // 50)
    assert compared >= 0.9 * R * 200
