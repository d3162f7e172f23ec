"""GPU parity of the Hilbert-Schmidt prior (QST_PRIOR_HS: rho = G G^dag / Tr, the QR of
Algorithm 1 skipped) against the FP64 oracle with the same prior: rho, p and log L on identical
latent rows at 1 to 5 qubits in the plain, tensor-core and structured forms, and the first 200
accept decisions per chain."""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W
from tests._helpers import unpack_rho, near_tie_band

pytestmark = pytest.mark.gpu


def _prec(qst, name):
    return {"fp32": qst.PREC_FP32, "bf16x3": qst.PREC_BF16X3, "pauli": qst.PREC_PAULI}[name]


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "pauli"])
@pytest.mark.parametrize("q,n", [(1, 300), (2, 517), (3, 700), (4, 333), (5, 130)])
def test_hs_prior_evaluate_matches_oracle(qst, oracle_mod, cuda_ok, prec, q, n):
    import torch
    prob = W.config_problem(q, num_chains=max(n, 256), num_steps=1) if q <= 4 else \
        W.five_qubit_problem(num_chains=max(n, 256), num_steps=1)
    s = qst.Sampler(prob, precision=_prec(qst, prec), diag_chains=0, prior=qst.PRIOR_HS)
    D = 1 << q
    x32 = W.latent_batch(n, q, seed=400 + q).astype(np.float32)
    rho_p, p_gpu, ll_gpu = s.evaluate(torch.from_numpy(x32).cuda())
    torch.cuda.synchronize()
    s.close()
    rho_ref, p_ref, ll_ref = oracle_mod.evaluate(prob, x32.astype(np.float64), prior=oracle_mod.PRIOR_HS)
    # G G^dag / Tr needs no QR: no conditioning caveat
    assert np.abs(unpack_rho(rho_p.cpu().numpy(), D) - rho_ref).max() < 2e-6
    assert np.abs(p_gpu.cpu().numpy().astype(np.float64) - p_ref).max() < 1e-6
    rel = np.abs(ll_gpu.cpu().numpy() - ll_ref) / np.abs(ll_ref)
    assert np.nanmax(rel) < 1e-5


@pytest.mark.parametrize("q", [2, 3])
def test_hs_prior_first_200_decisions(qst, oracle_mod, cuda_ok, q):
    R, S = 256, 200
    prob = W.config_problem(q, num_chains=R, num_steps=S)
    s = qst.Sampler(prob, precision=qst.PREC_FP32, trace_steps=S, diag_chains=0, prior=qst.PRIOR_HS)
    s.run_chains(S)
    acc_gpu, ll_prop = s.get_trace()
    rho, n = s.posterior_mean()
    s.close()
    ref = oracle_mod.run(prob, num_steps=S, trace_steps=S, want_final=True, prior=oracle_mod.PRIOR_HS)
    margin = ref["trace_log_alpha"] - (ref["trace_logl_prop"] - ref["trace_logl_cur"])
    band = near_tie_band(acc_gpu.T, ref["trace_accept"], ll_prop.T, ref["trace_logl_prop"])
    mism = 0
    compared = 0
    for r in range(R):
        bad = np.nonzero(acc_gpu.T[r] != ref["trace_accept"][r])[0]
        if bad.size == 0:
            compared += S
            continue
        assert abs(margin[r, bad[0]]) < band, (r, bad[0], margin[r, bad[0]], band)
        compared += bad[0]
        mism += 1
    assert mism <= max(2, R // 50)
    assert compared >= 0.9 * R * S
    assert n == ref["num_pooled"]
    same = np.all(acc_gpu.T == ref["trace_accept"], axis=1)
    if same.all():
        assert np.abs(rho - ref["mean"]).max() < 1e-5
