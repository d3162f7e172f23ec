"""GPU parity of the TF32 tensor-core forms against the FP64 oracle.

TF32x2 holds rho as hi + lo, two TF32 terms (22 significant bits), with the hi and lo products
in two FP32 accumulators: its p and log L meet the bars of the BF16x3 form.  TF32 rounds rho
once to 11 significant bits: every packed entry moves by at most 2^-11 of itself, so
|p_gpu - p_oracle| <= 2^-11 sum_i |P_ki| |rho_i| + the FP32 assembly's 1e-6, and |P_ki| <= 1
for Pauli projectors.  Its log L error is reported, not bounded (it is a comparison form).
"""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W
from tests._helpers import unpack_rho, near_tie_band

pytestmark = pytest.mark.gpu


def _cond(x, D):
    d = D * D
    H = (x[:, 2 * d:3 * d] + 1j * x[:, 3 * d:]).reshape(-1, D, D).transpose(0, 2, 1)
    return np.linalg.cond(H)


def _evaluate(qst, oracle_mod, prec, q, n, seed):
    import torch
    prob = W.config_problem(q, num_chains=max(n, 256), num_steps=1)
    s = qst.Sampler(prob, precision=prec, diag_chains=0)
    D = 1 << q
    x32 = W.latent_batch(n, q, seed=seed).astype(np.float32)
    rho_p, p_gpu, ll_gpu = s.evaluate(torch.from_numpy(x32).cuda())
    torch.cuda.synchronize()
    out = {
        "prob": prob, "D": D, "x": x32,
        "rho_packed": rho_p.cpu().numpy().astype(np.float64),
        "p": p_gpu.cpu().numpy().astype(np.float64),
        "ll": ll_gpu.cpu().numpy(),
    }
    s.close()
    out["rho_ref"], out["p_ref"], out["ll_ref"] = oracle_mod.evaluate(prob, x32.astype(np.float64))
    out["ok"] = _cond(x32.astype(np.float64), D) <= 1e3
    return out


def _own_reduction_gap(oracle_mod, r):
    """|log L_gpu - sum c log p| on the GPU's own p after the per-setting renormalisation."""
    n, D = r["p"].shape[0], r["D"]
    p3 = r["p"].reshape(n, -1, D)
    p_used = (p3 / p3.sum(-1, keepdims=True)).reshape(n, -1)
    ll_own = np.array([oracle_mod.loglik(r["prob"].counts, p_used[i]) for i in range(n)])
    fin = np.isfinite(ll_own)
    bound = np.sum(r["prob"].counts.astype(np.float64)) * 6 * 2.0 ** -24
    return np.abs(r["ll"][fin] - ll_own[fin]).max(), bound


@pytest.mark.parametrize("q,n", [(1, 300), (2, 517), (3, 1000)])
def test_tf32x2_evaluate_matches_oracle(qst, oracle_mod, cuda_ok, q, n):
    r = _evaluate(qst, oracle_mod, qst.PREC_TF32X2, q, n, seed=200 + q)
    ok = r["ok"]
    assert ok.mean() > 0.95
    rho_gpu = unpack_rho(r["rho_packed"], r["D"])
    assert np.abs(rho_gpu - r["rho_ref"]).max(axis=(1, 2))[ok].max() < 2e-6
    assert np.abs(r["p"] - r["p_ref"]).max(axis=1)[ok].max() < 1e-6
    gap, bound = _own_reduction_gap(oracle_mod, r)
    assert gap < bound
    rel = np.abs(r["ll"] - r["ll_ref"]) / np.abs(r["ll_ref"])
    assert np.nanmax(rel[ok]) < 1e-5


@pytest.mark.parametrize("q,n", [(1, 300), (2, 517), (3, 1000), (4, 333)])
def test_tf32_evaluate_error_is_the_tf32_rounding(qst, oracle_mod, cuda_ok, q, n):
    r = _evaluate(qst, oracle_mod, qst.PREC_TF32, q, n, seed=300 + q)
    ok = r["ok"]
    bound = 2.0 ** -11 * np.abs(r["rho_packed"]).sum(axis=1) + 1e-6
    err = np.abs(r["p"] - r["p_ref"]).max(axis=1)
    assert np.all(err[ok] <= bound[ok])
    # the rounding is there: TF32 is not silently more precise than its 11 bits
    assert np.median(err) > 1e-6
    gap, red_bound = _own_reduction_gap(oracle_mod, r)
    assert gap < red_bound


def test_tf32x2_first_200_decisions(qst, oracle_mod, cuda_ok):
    q, R = 3, 256
    prob = W.config_problem(q, num_chains=R, num_steps=200)
    s = qst.Sampler(prob, precision=qst.PREC_TF32X2, trace_steps=200, diag_chains=0)
    s.run_chains(200)
    acc_gpu, ll_prop = s.get_trace()
    s.close()
    ref = oracle_mod.run(prob, num_steps=200, trace_steps=200, want_final=True)
    margin = ref["trace_log_alpha"] - (ref["trace_logl_prop"] - ref["trace_logl_cur"])
    acc_gpu = acc_gpu.T
    band = near_tie_band(acc_gpu, ref["trace_accept"], ll_prop.T, ref["trace_logl_prop"])
    mism = 0
    compared = 0
    for c in range(R):
        bad = np.nonzero(acc_gpu[c] != ref["trace_accept"][c])[0]
        if bad.size == 0:
            compared += 200
            continue
        assert abs(margin[c, bad[0]]) < band, f"chain {c}: decisions differ away from a tie"
        compared += bad[0]
        mism += 1
    assert mism <= max(2, R // 50)
    assert compared >= 0.9 * R * 200
