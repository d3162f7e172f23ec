"""Five qubits (D = 32, 7776 Pauli projectors) on the GPU against the FP64 oracle.

At D = 32 the proposal kernel runs one warp per chain and streams the second operand of
every product from shared memory.  The tensor-core projection streams the A operand with
every 256-column N tile.  The parity bars are those of the D <= 16 tests:
- rho within 2e-6 and p within 1e-6 on rows with cond(H) <= 1e3;
- the reduction within sum c * 6 * 2^-24 of the oracle's sum on the GPU's own p (for the
  tensor-core form, p renormalised per setting as that form does);
- accept decisions that agree except at near-ties.
Both QR settings run: the default (qr_passes 3, first-order at five qubits) and the refinement of
U (qr_passes 4), with which the rho and p bars hold on every row, whatever cond(H).
"""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W
from tests._helpers import unpack_rho, near_tie_band

pytestmark = pytest.mark.gpu
PRECISIONS = ["fp32", "bf16x3", "pauli"]


def _prec(qst, name):
    return {"fp32": qst.PREC_FP32, "bf16x3": qst.PREC_BF16X3, "pauli": qst.PREC_PAULI}[name]


@pytest.fixture(scope="module")
def prob5():
    return W.five_qubit_problem(num_chains=300, num_steps=40)


@pytest.mark.parametrize("qr", [3, 4])
@pytest.mark.parametrize("prec", PRECISIONS)
def test_five_qubit_evaluate_matches_oracle(qst, oracle_mod, cuda_ok, prob5, prec, qr):
    import torch
    n = 300   # several 128-chain tiles and a ragged one; evaluate takes at most num_chains rows
    s = qst.Sampler(prob5, precision=_prec(qst, prec), diag_chains=0, qr_passes=qr)
    x32 = W.latent_batch(n, 5, seed=505).astype(np.float32)
    rho_p, p_gpu, ll_gpu = s.evaluate(torch.from_numpy(x32).cuda())
    torch.cuda.synchronize()
    s.close()
    rho_gpu = unpack_rho(rho_p.cpu().numpy(), 32)
    p_gpu = p_gpu.cpu().numpy().astype(np.float64)
    ll_gpu = ll_gpu.cpu().numpy()
    rho_ref, p_ref, ll_ref = oracle_mod.evaluate(prob5, x32.astype(np.float64))
    x = x32.astype(np.float64)
    H = (x[:, 2048:3072] + 1j * x[:, 3072:]).reshape(n, 32, 32).transpose(0, 2, 1)
    ok = np.linalg.cond(H) <= 1e3
    assert ok.mean() > 0.9
    if qr == 4:   # the refined U: every row
        ok = np.ones(n, dtype=bool)
    assert np.abs(rho_gpu - rho_ref).max(axis=(1, 2))[ok].max() < 2e-6
    assert np.abs(p_gpu - p_ref).max(axis=1)[ok].max() < 1e-6
    c = prob5.counts.astype(np.float64)
    p_used = p_gpu
    if prec in ("bf16x3", "pauli"):   # both renormalise every setting by its own sum
        p_used = (p_gpu.reshape(n, -1, 32) / p_gpu.reshape(n, -1, 32).sum(-1, keepdims=True)).reshape(n, -1)
    ll_own = np.array([oracle_mod.loglik(prob5.counts, p_used[i]) for i in range(n)])
    fin = np.isfinite(ll_own)
    assert np.abs(ll_gpu[fin] - ll_own[fin]).max() < np.sum(c) * 6 * 2.0 ** -24
    rel = np.abs(ll_gpu - ll_ref) / np.abs(ll_ref)
    assert np.nanmax(rel[ok]) < 1e-5


@pytest.mark.parametrize("qr", [3, 4])
@pytest.mark.parametrize("prec", PRECISIONS)
def test_five_qubit_decisions_match_oracle(qst, oracle_mod, cuda_ok, prec, qr):
    R, S = 32, 40
    prob = W.five_qubit_problem(num_chains=R, num_steps=S)
    s = qst.Sampler(prob, precision=_prec(qst, prec), trace_steps=S, diag_chains=0, qr_passes=qr)
    s.run_chains(S)
    acc_gpu, ll_prop = s.get_trace()
    mean, n = s.posterior_mean()
    s.close()
    ref = oracle_mod.run(prob, num_steps=S, trace_steps=S, want_final=True)
    margin = ref["trace_log_alpha"] - (ref["trace_logl_prop"] - ref["trace_logl_cur"])
    band = near_tie_band(acc_gpu.T, ref["trace_accept"], ll_prop.T, ref["trace_logl_prop"])
    mism = 0
    for r in range(R):
        bad = np.nonzero(acc_gpu.T[r] != ref["trace_accept"][r])[0]
        if bad.size:
            assert abs(margin[r, bad[0]]) < band, (r, bad[0], margin[r, bad[0]], band)
            mism += 1
    assert mism <= 2
    assert n == ref["num_pooled"] == R * S
    assert abs(np.trace(mean).real - 1) < 1e-6
    same = np.all(acc_gpu.T == ref["trace_accept"], axis=1)
    if same.all():
        assert np.abs(mean - ref["mean"]).max() < 1e-5
