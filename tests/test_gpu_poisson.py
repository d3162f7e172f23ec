"""The Poisson likelihood (QST_LIKELIHOOD_POISSON) on the GPU against the oracle.

Pauli settings measured through lossy detectors (workload.lossy_pauli_problem: elements
eta_kl Lambda_kl whose sum over a setting falls short of the identity, counts Poisson of mean
mu_k p_kl): rho, p and log L of given latent rows in the FP32 and BF16x3 forms, the reduction
on the GPU's own p, the first 200 accept decisions and the pooled mean; and the structured
Pauli form, whose settings are complete, on the Pauli problem of configuration 3 read as
Poisson counts.  The bars are those of the multinomial parity tests (test_gpu_parity.py), the
reduction's with the term sum_k mu_k S_k added to its rounding budget.
"""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W
from tests._helpers import near_tie_band, unpack_rho

pytestmark = pytest.mark.gpu


def _prec(qst, name):
    return {"fp32": qst.PREC_FP32, "bf16x3": qst.PREC_BF16X3, "pauli": qst.PREC_PAULI}[name]


def _cond(x, D):
    d = D * D
    H = (x[:, 2 * d:3 * d] + 1j * x[:, 3 * d:]).reshape(-1, D, D).transpose(0, 2, 1)
    return np.linalg.cond(H)


def _pauli_as_poisson(q, num_chains, num_steps):
    prob = W.config_problem(q, num_chains=num_chains, num_steps=num_steps)
    K, D = prob.num_povms, prob.dim
    prob.likelihood = 1
    prob.trials = prob.counts.reshape(K, D).sum(1).astype(np.float64)   # integers: exact in FP32
    return prob


def _problem(form, q, num_chains, num_steps=1):
    if form == "pauli":
        return _pauli_as_poisson(q, num_chains, num_steps)
    return W.lossy_pauli_problem(q, num_chains=num_chains, num_steps=num_steps)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "pauli"])
@pytest.mark.parametrize("q,n", [(1, 300), (2, 517), (3, 1000), (4, 777)])
def test_poisson_evaluate_matches_oracle(qst, oracle_mod, cuda_ok, prec, q, n):
    import torch
    prob = _problem(prec, q, max(n, 1024))
    s = qst.Sampler(prob, precision=_prec(qst, prec), diag_chains=0)
    D = 1 << q
    x32 = W.latent_batch(n, q, seed=200 + q).astype(np.float32)
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
    # the reduction on the GPU's own p: FP32 logarithms and terms (the multinomial bar) plus the
    # rounding of the mu_k S_k terms and of p itself
    c = prob.counts.astype(np.float64)
    mu = np.repeat(prob.trials, D)
    for i in range(n):
        own = oracle_mod.loglik_poisson(prob.counts, p_gpu[i], prob.trials)
        if not np.isfinite(own):
            continue
        bound = np.sum(c) * 6 * 2.0 ** -24 + np.sum(mu * np.abs(p_gpu[i])) * 4 * 2.0 ** -24
        assert abs(ll_gpu[i] - own) < bound, (i, ll_gpu[i], own, bound)
    rel = np.abs(ll_gpu - ll_ref) / np.abs(ll_ref)
    assert np.nanmax(rel[ok]) < 1e-5


def _compare_decisions(acc_gpu, acc_ref, margin, tol):
    R, S = acc_ref.shape
    compared, mism = 0, 0
    for r in range(R):
        bad = np.nonzero(acc_gpu[r] != acc_ref[r])[0]
        if bad.size == 0:
            compared += S
            continue
        t = bad[0]
        assert abs(margin[r, t]) < tol, f"chain {r} step {t + 1}: decisions differ away from a tie ({margin[r, t]})"
        compared += t
        mism += 1
    return compared, mism


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "pauli"])
@pytest.mark.parametrize("q", [2, 3])
def test_poisson_first_200_decisions(qst, oracle_mod, cuda_ok, prec, q):
    R = 256
    prob = _problem(prec, q, R, num_steps=200)
    s = qst.Sampler(prob, precision=_prec(qst, prec), trace_steps=200, diag_chains=0)
    s.run_chains(200)
    acc_gpu, ll_prop_gpu = s.get_trace()
    st = s.get_state()
    s.close()
    ref = oracle_mod.run(prob, num_steps=200, trace_steps=200, want_final=True)
    margin = ref["trace_log_alpha"] - (ref["trace_logl_prop"] - ref["trace_logl_cur"])
    tol = near_tie_band(acc_gpu.T, ref["trace_accept"], ll_prop_gpu.T, ref["trace_logl_prop"])
    compared, mism = _compare_decisions(acc_gpu.T, ref["trace_accept"], margin, tol=tol)
    assert mism <= max(2, R // 50), f"{mism} chains hit near-tie mismatches"
    assert compared >= 0.9 * R * 200
    assert ref["trace_accept"].mean() > 0.05   # the chains move: the test compares real decisions
    same = np.all(acc_gpu.T == ref["trace_accept"], axis=1)
    assert np.abs(st["y"][same] - ref["final_y"][same]).max() < 1e-3
    assert np.array_equal(st["beta"][same], ref["final_beta"][same])


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_poisson_pooled_mean_matches_oracle(qst, oracle_mod, cuda_ok, prec):
    """Two qubits through lossy detectors: the pooled posterior mean agrees with the oracle's
    within 3 jackknife standard errors (32 groups of the oracle's per-chain sums) + 1e-9."""
    R, S = 512, 300
    prob = W.lossy_pauli_problem(2, num_chains=R, num_steps=S)
    s = qst.Sampler(prob, precision=_prec(qst, prec), diag_chains=0)
    s.run_chains(S)
    rho, n = s.posterior_mean()
    s.close()
    ref = oracle_mod.run(prob, num_steps=S, want_chain_pool=True)
    assert n == ref["num_pooled"] == R * S
    groups = ref["chain_pool"].reshape(32, R // 32, 4, 4).sum(axis=1)
    total = groups.sum(axis=0)
    loo = (total[None] - groups) / (n - n // 32)
    se = np.sqrt((32 - 1) / 32 * np.sum(np.abs(loo - loo.mean(0)) ** 2, axis=0))
    assert np.all(np.abs(rho - ref["mean"]) <= 3 * se + 1e-9), np.abs(rho - ref["mean"]).max()
    # the truth is recovered far better than by the prior mean I / D
    assert np.linalg.norm(rho - prob.truth) < 0.6 * np.linalg.norm(np.eye(4) / 4 - prob.truth)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_poisson_five_qubits(qst, oracle_mod, cuda_ok, prec):
    """D = 32 (the streamed tensor-core kernel and the FP32 form's split settings): rho, p and
    log L of 64 latent rows through lossy detectors against the oracle."""
    import torch
    q, n = 5, 64
    prob = W.lossy_pauli_problem(q, num_chains=256)
    s = qst.Sampler(prob, precision=_prec(qst, prec), diag_chains=0)
    x32 = W.latent_batch(n, q, seed=205).astype(np.float32)
    rho_p, p_gpu, ll_gpu = s.evaluate(torch.from_numpy(x32).cuda())
    torch.cuda.synchronize()
    s.close()
    p_gpu = p_gpu.cpu().numpy().astype(np.float64)
    ll_gpu = ll_gpu.cpu().numpy()
    _, p_ref, ll_ref = oracle_mod.evaluate(prob, x32.astype(np.float64), want_rho=False)
    ok = _cond(x32.astype(np.float64), 32) <= 1e3
    assert ok.mean() > 0.9
    assert np.abs(p_gpu - p_ref).max(axis=1)[ok].max() < 1e-6
    c = prob.counts.astype(np.float64)
    mu = np.repeat(prob.trials, 32)
    for i in range(n):
        own = oracle_mod.loglik_poisson(prob.counts, p_gpu[i], prob.trials)
        bound = np.sum(c) * 6 * 2.0 ** -24 + np.sum(mu * np.abs(p_gpu[i])) * 4 * 2.0 ** -24
        assert abs(ll_gpu[i] - own) < bound, (i, ll_gpu[i], own, bound)
    assert np.nanmax((np.abs(ll_gpu - ll_ref) / np.abs(ll_ref))[ok]) < 1e-5


def test_poisson_with_the_other_features(qst, oracle_mod, cuda_ok):
    """The Poisson likelihood beside the rest of the sampler: under QST_PREC_AUTO in a batch with
    multinomial problems (every problem's chains equal, bit for bit, a handle of it alone in the
    form chosen for it); under the Hilbert-Schmidt prior (the oracle's log L of the same latent
    rows); and across a checkpoint (a restored run continues bit-exactly)."""
    import torch
    lossy = W.lossy_pauli_problem(3, num_chains=300, num_steps=30)
    batch = [W.config_problem(2, num_chains=256, num_steps=30), lossy,
             W.lossy_pauli_problem(2, num_chains=200, num_steps=30, seed=1301)]
    s = qst.Sampler(batch, precision=qst.PREC_AUTO, diag_chains=0)
    s.run_chains(30)
    forms = [s.diagnostics(i)["projection_form"] for i in range(len(batch))]
    for i, p in enumerate(batch):
        ref = qst.Sampler(p, precision=forms[i], diag_chains=0, autotune=0)
        ref.run_chains(30)
        a, b = s.get_state(i), ref.get_state()
        ref.close()
        assert np.array_equal(a["y"], b["y"]), (i, forms[i])
        assert np.array_equal(a["accepts"], b["accepts"])
    s.close()
    # the Hilbert-Schmidt prior
    hs = qst.Sampler(lossy, precision=qst.PREC_BF16X3, diag_chains=0, prior=qst.PRIOR_HS)
    x32 = W.latent_batch(256, 3, seed=77).astype(np.float32)
    _, _, ll = hs.evaluate(torch.from_numpy(x32).cuda(), want_rho=False, want_p=False)
    torch.cuda.synchronize()
    hs.close()
    _, _, ll_ref = oracle_mod.evaluate(lossy, x32.astype(np.float64), want_rho=False, want_p=False,
                                       prior=oracle_mod.PRIOR_HS)
    assert np.nanmax(np.abs(ll.cpu().numpy() - ll_ref) / np.abs(ll_ref)) < 1e-5
    # checkpoint and restore
    kw = dict(precision=qst.PREC_FP32, diag_chains=0, adapt_interval=10)
    straight = qst.Sampler(lossy, **kw)
    straight.run_chains(30)
    first = qst.Sampler(lossy, **kw)
    first.run_chains(12)
    ck = first.checkpoint()
    first.close()
    second = qst.Sampler(lossy, **kw)
    second.restore(ck)
    second.run_chains(18)
    a, b = straight.get_state(), second.get_state()
    for k in ("y", "logl", "beta", "accepts"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(straight.posterior_mean()[0], second.posterior_mean()[0])
    straight.close()
    second.close()
