"""GPU parity tests: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (derived from the arithmetic of each step):
* Philox words: bit-exact.
* p_kl on identical latent x: 1e-6 absolute whenever cond(H) <= 1e3.  The FP32
  assembly's forward error in U is O(cond(H) * 2^-24), and p inherits it.
* log L reduction: |logL_gpu - sum c log p_gpu (FP64)| <= sum_{c>0} c * 6 * 2^-24 (per term, one
  rounding each for p*invf, logf and the product, doubled for the FP32 partial sums).
* accept decisions: identical, except where |log alpha - Delta log L| is below the
  measured log L error (a near tie); a chain's later steps are not compared after one.
"""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W
from tests._helpers import near_tie_band, unpack_rho

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


PRECISIONS = ["fp32", "bf16x3", "pauli"]


def _prec(qst, name):
    return {"fp32": qst.PREC_FP32, "bf16x3": qst.PREC_BF16X3, "pauli": qst.PREC_PAULI}[name]


def _sampler(qst, prob, prec="fp32", **kw):
    return qst.Sampler(prob, precision=_prec(qst, prec), **kw)


# ------------------------------------------------------------------------------- Philox

@pytest.mark.parametrize("seed", [0, 3004, 0xFEDCBA9876543210])
@pytest.mark.parametrize("tag", [0, 1, 2])
def test_philox_bit_exact(qst, oracle_mod, cuda_ok, seed, tag):
    torch = _torch()
    for step, chain0, nchains, block0, nblocks in [(0, 0, 3, 0, 16), (17, 5, 4, 3, 5),
                                                   (4294967295, 4294967290, 5, 250, 6), (1000, 65530, 7, 0, 256)]:
        got = qst.philox_blocks(seed, step, tag, chain0, nchains, block0, nblocks)
        torch.cuda.synchronize()
        got = got.cpu().numpy().view(np.uint32)
        for i in range(nchains):
            want = oracle_mod.philox_blocks(seed, step, chain0 + i, tag, block0, nblocks)
            assert np.array_equal(got[i], want), (step, chain0 + i)


# ------------------------------------------------------------------------------- evaluation

def _cond(x, D):
    d = D * D
    H = (x[:, 2 * d:3 * d] + 1j * x[:, 3 * d:]).reshape(-1, D, D).transpose(0, 2, 1)
    return np.linalg.cond(H)


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("q,n", [(1, 300), (2, 517), (3, 1000), (4, 777)])
def test_evaluate_matches_oracle(qst, oracle_mod, cuda_ok, prec, q, n):
    torch = _torch()
    prob = W.config_problem(q, num_chains=max(n, 1024), num_steps=1)
    s = _sampler(qst, prob, prec, diag_chains=0)
    D = 1 << q
    x32 = W.latent_batch(n, q, seed=100 + q).astype(np.float32)
    rho_p, p_gpu, ll_gpu = s.evaluate(torch.from_numpy(x32).cuda())
    torch.cuda.synchronize()
    rho_gpu = unpack_rho(rho_p.cpu().numpy(), D)
    p_gpu = p_gpu.cpu().numpy().astype(np.float64)
    ll_gpu = ll_gpu.cpu().numpy()
    rho_ref, p_ref, ll_ref = oracle_mod.evaluate(prob, x32.astype(np.float64))
    kappa = _cond(x32.astype(np.float64), D)
    ok = kappa <= 1e3
    assert ok.mean() > 0.95
    # rho and p on identical x
    assert np.abs(rho_gpu - rho_ref).max(axis=(1, 2))[ok].max() < 2e-6
    assert np.abs(p_gpu - p_ref).max(axis=1)[ok].max() < 1e-6
    # log-likelihood reduction on the GPU's own p (the tensor-core and Pauli forms renormalise every
    # setting by its own sum, p_kl / sum_l p_kl, which is exact for a complete POVM)
    c = prob.counts.astype(np.float64)
    p_used = p_gpu
    if prec in ("bf16x3", "pauli"):   # both renormalise every setting by its own sum
        p_used = (p_gpu.reshape(n, -1, D) / p_gpu.reshape(n, -1, D).sum(-1, keepdims=True)).reshape(n, -1)
    ll_own = np.array([oracle_mod.loglik(prob.counts, p_used[i]) for i in range(n)])
    bound = np.sum(c) * 6 * 2.0 ** -24
    finite = np.isfinite(ll_own)
    assert np.abs(ll_gpu[finite] - ll_own[finite]).max() < bound
    # end to end against the oracle's own p (relative; prior draws have large |log L|)
    rel = np.abs(ll_gpu - ll_ref) / np.abs(ll_ref)
    assert np.nanmax(rel[ok]) < 1e-5
    s.close()


@pytest.mark.parametrize("n", [0, 1, 127, 128, 129])
def test_evaluate_ragged_sizes(qst, oracle_mod, cuda_ok, n):
    torch = _torch()
    prob = W.config_problem(3, num_chains=256, num_steps=1)
    s = _sampler(qst, prob, "fp32", diag_chains=0)
    x32 = W.latent_batch(max(n, 1), 3, seed=7).astype(np.float32)[:n]
    rho_p, p_gpu, ll_gpu = s.evaluate(torch.from_numpy(x32).cuda().reshape(n, 4 * 64))
    torch.cuda.synchronize()
    if n:
        _, p_ref, _ = oracle_mod.evaluate(prob, x32.astype(np.float64))
        assert np.abs(p_gpu.cpu().numpy() - p_ref).max() < 1e-6
    s.close()


# ------------------------------------------------------------------------------- chains

def _compare_decisions(acc_gpu, acc_ref, margin, tol):
    """Per chain, the first mismatch must be a near tie; returns (compared, mismatched)."""
    R, S = acc_ref.shape
    compared = 0
    mism = 0
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


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("q,R,beta0", [(1, 256, 0.1), (2, 256, 0.05), (3, 256, 0.1), (4, 256, 0.02)])
def test_first_200_decisions(qst, oracle_mod, cuda_ok, prec, q, R, beta0):
    prob = W.config_problem(q, num_chains=R, num_steps=200)
    prob.beta0 = beta0
    s = _sampler(qst, prob, prec, trace_steps=200, diag_chains=0)
    s.run_chains(200)
    acc_gpu, ll_prop_gpu = s.get_trace()
    st = s.get_state()
    s.close()
    ref = oracle_mod.run(prob, num_steps=200, trace_steps=200, want_final=True)
    margin = ref["trace_log_alpha"] - (ref["trace_logl_prop"] - ref["trace_logl_cur"])
    # log L of the proposals agree where trajectories still coincide: relative error of
    # the FP32 assembly, largest for proposals deep in the tails (p_kl -> 0 for counted
    # outcomes, which are rejected anyway)
    same = np.all(acc_gpu.T == ref["trace_accept"], axis=1)
    d = np.abs(ll_prop_gpu.T[same] - ref["trace_logl_prop"][same])
    fin = np.isfinite(ref["trace_logl_prop"][same])
    # a decision may differ only at a near tie: where |log alpha - Delta log L| is within
    # twice the log L error measured in this run (the current and the proposed state each
    # carry one)
    tol = near_tie_band(acc_gpu.T, ref["trace_accept"], ll_prop_gpu.T, ref["trace_logl_prop"])
    compared, mism = _compare_decisions(acc_gpu.T, ref["trace_accept"], margin, tol=tol)
    assert mism <= max(2, R // 50), f"{mism} chains hit near-tie mismatches"
    assert compared >= 0.9 * R * 200
    rel = d[fin] / np.abs(ref["trace_logl_prop"][same][fin])
    assert np.median(rel) < 1e-7
    assert rel.max() < 1e-4
    # the final states of identical chains agree to FP32 drift
    assert np.abs(st["y"][same] - ref["final_y"][same]).max() < 1e-3
    assert np.array_equal(st["beta"][same], ref["final_beta"][same])


@pytest.mark.parametrize("prec", PRECISIONS)
def test_four_qubit_posterior_fidelity_within_monte_carlo_error(qst, oracle_mod, cuda_ok, prec):
    """Configuration 4 (4 qubits): pooled posterior mean and its fidelity to the truth agree
    with the oracle's within 3 Monte Carlo standard errors (jackknife over 32 chain groups of
    the oracle's per-chain sums; chains are independent, so groups are i.i.d.)."""
    R, S = 512, 120
    prob = W.config_problem(4, num_chains=R, num_steps=S)
    s = _sampler(qst, prob, prec, diag_chains=0)
    s.run_chains(S)
    rho, n = s.posterior_mean()
    s.close()
    ref = oracle_mod.run(prob, num_steps=S, want_chain_pool=True)
    assert n == ref["num_pooled"] == R * S
    groups = ref["chain_pool"].reshape(32, R // 32, 16, 16).sum(axis=1)      # [32][D][D] sums
    total = groups.sum(axis=0)
    loo = (total[None] - groups) / ((R - R // 32) * S)                      # leave-one-group-out means
    se = np.sqrt((32 - 1) / 32 * (np.abs(loo - loo.mean(axis=0)) ** 2).sum(axis=0))   # |.|^2: complex entries
    assert np.all(np.abs(rho - ref["mean"]) <= 3 * se + 1e-9)
    f_loo = np.array([oracle_mod.fidelity(m, prob.truth) for m in loo])
    se_f = np.sqrt((32 - 1) / 32 * ((f_loo - f_loo.mean()) ** 2).sum())
    f_gpu = oracle_mod.fidelity(rho, prob.truth)
    f_ref = oracle_mod.fidelity(ref["mean"], prob.truth)
    assert abs(f_gpu - f_ref) <= 3 * se_f, (f_gpu, f_ref, se_f)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_pooled_mean_and_acf_match_oracle(qst, oracle_mod, cuda_ok, prec):
    prob = W.config_problem(2, num_chains=512, num_steps=600)
    s = _sampler(qst, prob, prec, diag_chains=8, traj_capacity=600, acf_lmax=50, adapt_interval=100)
    s.run_chains(600)
    rho, n = s.posterior_mean()
    dg = s.diagnostics()
    s.close()
    ref = oracle_mod.run(prob, num_steps=600, traj_chains=8, traj_capacity=600, want_chain_pool=True,
                         adapt_interval=100)
    assert n == ref["num_pooled"] == 512 * 600
    # Monte Carlo error from the spread of per-chain means (chains are independent)
    per_chain = ref["chain_pool"] / 600
    se = per_chain.std(axis=0) / np.sqrt(512)
    assert np.all(np.abs(rho - ref["mean"]) <= 3 * se + 1e-7)
    assert abs(oracle_mod.fidelity(ref["mean"], rho) - 1) < 1e-6
    # IACT of the diagnostic chains
    taus = np.array([oracle_mod.iact(oracle_mod.acf(ref["traj"][c], 50)) for c in range(8)])
    assert dg["diag_chains"] == 8
    assert np.allclose(np.sort(dg["tau"]), np.sort(taus), rtol=0.05, atol=0.05)
    assert abs(dg["tau_mean"] - taus.mean()) < 0.05 * taus.mean() + 0.05


def test_zero_counts_sample_the_prior(qst, oracle_mod, cuda_ok):
    prob = W.config_problem(2, num_chains=4096, num_steps=300)
    prob.counts = np.zeros_like(prob.counts)
    s = _sampler(qst, prob, "fp32", adapt_interval=100, diag_chains=0)
    s.run_chains(300)
    st = s.get_state()
    rho, n = s.posterior_mean()
    dg = s.diagnostics()
    s.close()
    assert np.all(st["accepts"] == 300)
    assert dg["accept_rate"] == 1.0
    assert np.all(st["beta"] == min(prob.beta0 * 1.1 * 1.1 * 1.1, 1.0))
    assert np.abs(rho - np.eye(4) / 4).max() < 5 * 0.5 / np.sqrt(4096)
    y = st["y"].astype(np.float64)
    assert abs(y.var() - 1) < 5 * np.sqrt(2 / y.size)


@pytest.mark.parametrize("thin,burn", [(1, 0), (3, 0), (4, 10)])
def test_thinning_counts_and_trajectories(qst, oracle_mod, cuda_ok, thin, burn):
    prob = W.config_problem(2, num_chains=64, num_steps=100)
    s = _sampler(qst, prob, "fp32", thin=thin, burn_in=burn, diag_chains=2, traj_capacity=100, acf_lmax=5)
    s.run_chains(100)
    rho, n = s.posterior_mean()
    s.close()
    ref = oracle_mod.run(prob, num_steps=100, thin=thin, burn_in=burn)
    assert n == ref["num_pooled"]
    assert np.abs(rho - ref["mean"]).max() < 1e-3


def test_multi_problem_handle_matches_single(qst, cuda_ok):
    probs = [W.config_problem(q, num_chains=R, num_steps=50) for q, R in [(1, 100), (3, 300), (2, 257)]]
    multi = _sampler(qst, probs, "fp32", diag_chains=0)
    multi.run_chains(50)
    for i, p in enumerate(probs):
        single = _sampler(qst, p, "fp32", diag_chains=0)
        single.run_chains(50)
        a = multi.get_state(i)
        b = single.get_state(0)
        assert np.array_equal(a["y"], b["y"])
        assert np.array_equal(multi.posterior_mean(i)[0], single.posterior_mean(0)[0])
        single.close()
    multi.close()


@pytest.mark.parametrize("prec", PRECISIONS)
def test_graph_replay_matches_plain_launches(qst, cuda_ok, prec):
    """A step captured once as a CUDA graph (device-side step counter) and replayed gives the
    same bits as plain launches, across several qst_run_chains calls, thinning and burn-in."""
    probs = [W.config_problem(q, num_chains=R, num_steps=40) for q, R in [(1, 100), (4, 300), (2, 257)]]
    kw = dict(diag_chains=4, traj_capacity=16, acf_lmax=4, thin=3, burn_in=5, adapt_interval=7)
    g = _sampler(qst, probs, prec, use_graph=1, **kw)
    p = _sampler(qst, probs, prec, use_graph=0, **kw)
    for n in (20, 1, 17):
        g.run_chains(n)
        p.run_chains(n)
    for i in range(len(probs)):
        a, b = g.get_state(i), p.get_state(i)
        for k in a:
            assert np.array_equal(a[k], b[k]), (i, k)
        assert np.array_equal(g.posterior_mean(i)[0], p.posterior_mean(i)[0])
        da, db = g.diagnostics(i), p.diagnostics(i)
        assert np.array_equal(da["tau"], db["tau"]) and da["num_pooled"] == db["num_pooled"]
    assert g.launch_count() == p.launch_count()
    g.close()
    p.close()


@pytest.mark.parametrize("prec", PRECISIONS)
def test_autotuned_schedule_gives_the_same_chains(qst, cuda_ok, prec):
    """The autotuner changes how the projection's N tiles are split over CTAs (the partial
    sums are the same numbers associated differently in FP64) and how many chains share a
    proposal CTA (the same per-chain arithmetic), so the chains agree: the latent states bit
    for bit, log L to FP64 association.  Every proposal CTA size is forced once."""
    for q, R in [(2, 700), (4, 300)]:
        prob = W.config_problem(q, num_chains=R, num_steps=30)
        tuned = _sampler(qst, prob, prec, diag_chains=0, autotune=1)
        runs = [tuned] + [_sampler(qst, prob, prec, diag_chains=0, autotune=0, propose_threads=t)
                          for t in (128, 64, 32)]
        for s in runs:
            s.run_chains(30)
        a = tuned.get_state()
        dg = tuned.diagnostics()
        assert dg["column_groups"] >= 1
        assert dg["propose_chains_per_cta"] in (128 >> q, 64 >> q, 32 >> q)
        assert dg["accept_chains_per_cta"] >= 8
        for s, t in zip(runs[1:], (128, 64, 32)):
            b = s.get_state()
            assert s.diagnostics()["propose_chains_per_cta"] == t >> q
            assert np.array_equal(a["y"], b["y"]), (q, t)
            assert np.array_equal(a["accepts"], b["accepts"])
            assert np.allclose(a["logl"], b["logl"], rtol=1e-12, atol=0)
        for s in runs:
            s.close()


def test_chain_offset_partition_is_exact(qst, cuda_ok):
    """Chains keyed by global id: [0,96) at once equals [0,40) + [40,96) as two handles."""
    prob = W.config_problem(3, num_chains=96, num_steps=40)
    full = _sampler(qst, prob, "fp32", diag_chains=0)
    full.run_chains(40)
    a_p = W.config_problem(3, num_chains=40, num_steps=40)
    b_p = W.config_problem(3, num_chains=56, num_steps=40)
    a = qst.Sampler(a_p, chain_offsets=[0], diag_chains=0)
    b = qst.Sampler(b_p, chain_offsets=[40], diag_chains=0)
    a.run_chains(40)
    b.run_chains(40)
    y = full.get_state()["y"]
    assert np.array_equal(np.concatenate([a.get_state()["y"], b.get_state()["y"]]), y)
    ra, na = a.posterior_mean()
    rb, nb = b.posterior_mean()
    rf, nf = full.posterior_mean()
    assert na + nb == nf
    # pooled sums differ only by the order of the FP32 per-CTA tile sums
    assert np.abs((ra * na + rb * nb) / nf - rf).max() < 1e-7
    for h in (full, a, b):
        h.close()


def test_checkpoint_restore_is_bit_exact(qst, cuda_ok):
    prob = W.config_problem(3, num_chains=200, num_steps=60)
    straight = _sampler(qst, prob, "fp32", diag_chains=4, traj_capacity=64, acf_lmax=5, adapt_interval=20)
    straight.run_chains(60)
    first = _sampler(qst, prob, "fp32", diag_chains=4, traj_capacity=64, acf_lmax=5, adapt_interval=20)
    first.run_chains(30)
    ck = first.checkpoint()
    first.close()
    second = _sampler(qst, prob, "fp32", diag_chains=4, traj_capacity=64, acf_lmax=5, adapt_interval=20)
    second.restore(ck)
    second.run_chains(30)
    a, b = straight.get_state(), second.get_state()
    for k in ("y", "logl", "beta", "accepts"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(straight.posterior_mean()[0], second.posterior_mean()[0])
    straight.close()
    second.close()


def test_nan_injection_is_contained(qst, cuda_ok):
    prob = W.config_problem(2, num_chains=256, num_steps=50)
    s = _sampler(qst, prob, "fp32", diag_chains=0)
    s.run_chains(10)
    before = s.get_state()
    s.inject_nan(17)
    s.run_chains(40)
    after = s.get_state()
    rho, n = s.posterior_mean()
    assert np.all(np.isfinite(rho))
    assert after["accepts"][17] == before["accepts"][17]   # every later proposal rejected
    assert np.isfinite(after["logl"][17])                   # keeps its last valid state
    assert after["accepts"].sum() > before["accepts"].sum()
    s.close()


# ------------------------------------------------------------------------------- full size

@pytest.mark.parametrize("prec", PRECISIONS)
def test_config4_full_size_sampled_chains(qst, oracle_mod, cuda_ok, prec):
    """65536 chains in the benchmark's launch configuration; 24 sampled chains are
    re-run alone by the oracle (chains are independent and keyed by global id)."""
    prob = W.config_problem(4, num_chains=65536, num_steps=40)
    s = _sampler(qst, prob, prec, trace_steps=40)
    s.run_chains(40)
    st = s.get_state()
    acc, _ = s.get_trace()
    rho, n = s.posterior_mean()
    s.close()
    assert n == 65536 * 40
    assert abs(np.trace(rho).real - 1) < 1e-6
    assert np.linalg.eigvalsh(rho).min() > -1e-7
    rng = np.random.default_rng(0)
    sample = np.concatenate([[0, 1, 65535], rng.choice(65536, 21, replace=False)])
    agree = 0
    for c in sample:
        ref = oracle_mod.run(prob, num_chains=1, chain_begin=int(c), num_steps=40, trace_steps=40, want_final=True)
        if np.array_equal(acc[:, c], ref["trace_accept"][0]):
            agree += 1
            assert np.abs(st["y"][c] - ref["final_y"][0]).max() < 1e-3
            assert abs(st["logl"][c] - ref["final_logl"][0]) < 1e-3 * max(1.0, abs(ref["final_logl"][0]) * 1e-6) + 5e-3
    assert agree >= len(sample) - 1


def test_bounded_wait_runs_out_and_the_context_stays_usable(qst, cuda_ok):
    """The kernels' bounded mbarrier wait, on a barrier nothing completes, gives up after its
    limit, reports QST_ERR_TIMEOUT through the status word, and leaves the context and the
    handle working (no trap, no fault)."""
    import time
    prob = W.config_problem(2, num_chains=256, num_steps=10)
    s = _sampler(qst, prob, "bf16x3", diag_chains=0)
    s.run_chains(5)
    t0 = time.perf_counter()
    with pytest.raises(qst.QstError) as err:
        s.probe_wait_timeout(50)
    waited = time.perf_counter() - t0
    assert err.value.status == 4                      # QST_ERR_TIMEOUT
    assert 0.04 <= waited < 5.0
    s.run_chains(5)                                    # the same handle keeps sampling
    s.synchronize()
    rho, n = s.posterior_mean()
    assert n == 256 * 10 and np.isfinite(rho).all()
    with pytest.raises(qst.QstError):
        s.probe_wait_timeout(0)                        # out of range: refused on the host
    s.close()


def test_builtin_pauli_povms_give_the_same_chains(qst, cuda_ok):
    """NULL POVM arrays (the built-in Pauli set) and the explicit Pauli arrays give bitwise the
    same chains."""
    import copy
    prob = W.config_problem(3, num_chains=256, num_steps=20)
    null = copy.copy(prob)
    null.povm_re = None
    null.povm_im = None
    out = []
    for p in (prob, null):
        s = _sampler(qst, p, "bf16x3", diag_chains=0)
        s.run_chains(20)
        out.append(s.get_state())
        s.close()
    assert np.array_equal(out[0]["y"], out[1]["y"])
    assert np.array_equal(out[0]["logl"], out[1]["logl"])


def test_config5_full_batch_sampled_chains(qst, oracle_mod, cuda_ok):
    """Configuration 5 as the benchmark runs it (64 problems of 1-5 qubits, 552,149 chains, one
    handle, graph replay, autotuned, mixed form): chains sampled from four problems, including
    the largest five-qubit one, re-run alone by the oracle give the same accept decisions
    (chains are independent and keyed by their problem's seed and global id)."""
    batch = W.heterogeneous_batch(64)
    S = 12
    s = qst.Sampler(batch, precision=qst.PREC_BF16X3, trace_steps=S, diag_chains=0)
    s.run_chains(S)
    five = [i for i, p in enumerate(batch) if p.num_qubits == 5]
    picks = [0, 1, five[0], max(five, key=lambda i: batch[i].num_chains)]
    rng = np.random.default_rng(5)
    checked = agree = 0
    for i in picks:
        p = batch[i]
        acc, _ = s.get_trace(i)
        for c in [0, p.num_chains - 1] + list(rng.choice(p.num_chains, 2, replace=False)):
            ref = oracle_mod.run(p, num_chains=1, chain_begin=int(c), num_steps=S, trace_steps=S)
            checked += 1
            agree += int(np.array_equal(acc[:, c], ref["trace_accept"][0]))
        rho, n = s.posterior_mean(i)
        assert n == p.num_chains * S
        assert abs(np.trace(rho).real - 1) < 1e-6
    s.close()
    assert agree >= checked - 1, f"{agree} of {checked} sampled chains agree"
