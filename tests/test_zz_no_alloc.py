"""qst_loglik_noalloc: the log-likelihood entry point for callers that must not allocate
device memory (its scratch is a fixed array inside the library).

Through the C ABI, consecutive calls must give the same log L as the existing
qst_evaluate (FP32 form) on the same latent vectors, and as the FP64 oracle.  The comparison uses the bound of
the parity tests for the FP64 reduction of FP32 terms: sum_{c>0} c * 6 * 2^-24.  The calls
change the problem size so a call that follows a larger one must not read that one's
leftovers from the shared scratch.  Kept in its own file, collected last.
"""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W

pytestmark = pytest.mark.gpu


def _evaluate_with_handle(qst, prob, x):
    s = qst.Sampler(prob, precision=qst.PREC_FP32, diag_chains=0)
    _, _, ll = s.evaluate(x, want_rho=False, want_p=False)
    out = ll.cpu().numpy()
    s.close()
    return out


def test_noalloc_matches_evaluate_on_consecutive_calls(qst, cuda_ok):
    import torch
    cases = [(3, 1000, 11), (2, 300, 12), (4, 4096, 13), (1, 7, 14)]
    for q, n, seed in cases:
        prob = W.config_problem(q, num_chains=n, num_steps=1)
        P = torch.from_numpy(qst.pack_projectors(q, prob.povm_re, prob.povm_im)).cuda()
        x = torch.from_numpy(W.latent_batch(n, q, seed=seed).astype(np.float32)).cuda()
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        qst.loglik_noalloc(q, prob.num_povms, P, prob.counts, x, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = _evaluate_with_handle(qst, prob, x)
        bound = float(np.sum(prob.counts)) * 6 * 2.0 ** -24
        assert np.all(np.isfinite(got)), (q, n)
        assert np.abs(got - want).max() <= bound, (q, n, np.abs(got - want).max(), bound)


def test_noalloc_matches_the_oracle(qst, oracle_mod, cuda_ok):
    """The same log L as the FP64 oracle on identical latent vectors: 1e-5 relative (the
    end-to-end bar of the parity tests) and, at four qubits, 2.5e-3 absolute on prior draws
    (the bar of test_gpu_logl_accuracy.py).  Run on a stream of its own, twice in a row."""
    import torch
    stream = torch.cuda.Stream()
    for q, n, seed in [(2, 700, 21), (4, 1024, 22)]:
        prob = W.config_problem(q, num_chains=n, num_steps=1)
        x64 = W.latent_batch(n, q, seed=seed)
        x32 = x64.astype(np.float32)
        with torch.cuda.stream(stream):
            P = torch.from_numpy(qst.pack_projectors(q, prob.povm_re, prob.povm_im)).cuda()
            x = torch.from_numpy(x32).cuda()
            outs = [torch.full((n,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
            for out in outs:
                qst.loglik_noalloc(q, prob.num_povms, P, prob.counts, x, out, stream=stream)
        stream.synchronize()
        _, _, ref = oracle_mod.evaluate(prob, x32.astype(np.float64), want_rho=False, want_p=False)
        for out in outs:
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-5, q
            if q == 4:
                assert np.abs(got - ref).max() <= 2.5e-3


def test_noalloc_rejects_sizes_beyond_its_scratch(qst, cuda_ok):
    import torch
    prob = W.config_problem(2, num_chains=8, num_steps=1)
    P = torch.from_numpy(qst.pack_projectors(2, prob.povm_re, prob.povm_im)).cuda()
    n = qst.NOALLOC_MAX_ROWS + 1
    x = torch.zeros((n, 64), dtype=torch.float32, device="cuda")
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(qst.QstError) as e:
        qst.loglik_noalloc(2, prob.num_povms, P, prob.counts, x, out)
    assert e.value.status == 1
    assert "QST_NOALLOC_MAX_ROWS" in str(e.value)
