"""Pins of the oracle's Algorithm 2 (pCN chains, adaptation, thinning, pooling).

* Posterior by quadrature (1 qubit): rho = (I + r.sigma)/2 with the Bures prior
  density prop. to (1 - |r|^2)^(-1/2) on the Bloch ball and the multinomial
  likelihood prod_a ((1 + r_a)/2)^{c_a+} ((1 - r_a)/2)^{c_a-}.  The pooled mean of
  independent chains (Eq. BME2) must match the quadrature mean within Monte Carlo
  error; with weak data it must also be far from the flat-prior mean.
* Zero counts: log L = 0, so every proposal is accepted (log alpha < 0) and the
  chains sample the prior N(0, I) exactly (pCN is prior-reversible): the state is
  standard normal, rho is Bures (mean purity 7/8 for a qubit), beta grows by the
  adaptation factor every M_A steps up to the clamp.
* Thinning / burn-in bookkeeping and chain independence (a chain's result does
  not depend on which other chains run beside it).
"""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W

SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, -1j], [1j, 0]])
SZ = np.array([[1, 0], [0, -1]], dtype=complex)


def _qubit(r):
    return (np.eye(2) + r[0] * SX + r[1] * SY + r[2] * SZ) / 2


def _bloch(rhos):
    return np.stack([np.einsum("nab,ba->n", rhos, S).real for S in (SX, SY, SZ)], 1)


def _quadrature_sphere(c, prior="bures", n=96):
    """Posterior mean Bloch vector on the full ball; |r| = sin(psi) removes the edge singularity."""
    xg, wg = np.polynomial.legendre.leggauss(n)
    psi, wpsi = (xg + 1) * np.pi / 4, wg * np.pi / 4
    th, wth = (xg + 1) * np.pi / 2, wg * np.pi / 2
    ph, wph = (xg + 1) * np.pi, wg * np.pi
    P, T, F = np.meshgrid(psi, th, ph, indexing="ij")
    s = np.sin(P)
    R = [s * np.sin(T) * np.cos(F), s * np.sin(T) * np.sin(F), s * np.cos(T)]
    # Bures: s^2 (1 - s^2)^(-1/2) ds = sin^2(psi) dpsi ; flat: s^2 ds = sin^2(psi) cos(psi) dpsi
    meas = np.sin(P) ** 2 * np.sin(T) * (1.0 if prior == "bures" else np.cos(P))
    w3 = wpsi[:, None, None] * wth[None, :, None] * wph[None, None, :]
    logl = sum(c[a, 0] * np.log((1 + R[a]) / 2) + c[a, 1] * np.log((1 - R[a]) / 2) for a in range(3))
    lw = logl + np.log(meas * w3 + 1e-300)
    w = np.exp(lw - lw.max())
    return np.array([(w * R[a]).sum() / w.sum() for a in range(3)])


def _quadrature_box(c, n=64, width=9.0):
    """Posterior mean for concentrated data: Gauss-Legendre box of +-width sigma around the MLE."""
    rhat = (c[:, 0] - c[:, 1]) / c.sum(1)
    sig = np.sqrt((1 - rhat ** 2) / c.sum(1))
    xg, wg = np.polynomial.legendre.leggauss(n)
    axes = [rhat[a] + width * sig[a] * xg for a in range(3)]
    wts = [width * sig[a] * wg for a in range(3)]
    RX, RY, RZ = np.meshgrid(*axes, indexing="ij")
    w3 = wts[0][:, None, None] * wts[1][None, :, None] * wts[2][None, None, :]
    rr = RX ** 2 + RY ** 2 + RZ ** 2
    inside = rr < 1
    rr = np.where(inside, rr, 0.0)
    with np.errstate(all="ignore"):
        logl = sum(c[a, 0] * np.log((1 + R) / 2) + c[a, 1] * np.log((1 - R) / 2)
                   for a, R in enumerate((RX, RY, RZ)))
        lp = np.where(inside, logl - 0.5 * np.log(1 - rr) + np.log(w3), -np.inf)
    w = np.exp(lp - lp.max())
    return np.array([(w * R).sum() / w.sum() for R in (RX, RY, RZ)])


def _pooled_bloch_per_chain(res, R):
    per_chain = res["chain_pool"] / (res["num_pooled"] / R)
    return _bloch(per_chain)


def test_qubit_posterior_weak_data(oracle_mod):
    prob = W.make_problem(1, _qubit([0.3, -0.4, 0.5]), 12, 512, 3000, 0.1, data_seed=21, chain_seed=22)
    c = prob.counts.reshape(3, 2).astype(float)
    bures = _quadrature_sphere(c, "bures")
    assert np.abs(bures - _quadrature_sphere(c, "bures", n=128)).max() < 1e-10
    flat = _quadrature_sphere(c, "flat")
    res = oracle_mod.run(prob, burn_in=1000, want_chain_pool=True)
    rc = _pooled_bloch_per_chain(res, 512)
    mean, se = rc.mean(0), rc.std(0) / np.sqrt(512)
    assert np.all(np.abs(mean - bures) < 4 * se), (mean, bures, se)
    assert np.any(np.abs(mean - flat) > 8 * se)


def test_qubit_posterior_concentrated(oracle_mod):
    prob = W.make_problem(1, _qubit([0.3, -0.4, 0.5]), 1000, 256, 4000, 0.1, data_seed=11, chain_seed=12)
    c = prob.counts.reshape(3, 2).astype(float)
    quad = _quadrature_box(c)
    res = oracle_mod.run(prob, burn_in=1000, want_chain_pool=True)
    rc = _pooled_bloch_per_chain(res, 256)
    mean, se = rc.mean(0), rc.std(0) / np.sqrt(256)
    assert np.all(np.abs(mean - quad) < 4 * se), (mean, quad, se)


@pytest.mark.parametrize("q", [1, 2])
def test_zero_counts_sample_the_prior(oracle_mod, q):
    prob = W.config_problem(q, num_chains=2048, num_steps=1000)
    prob.counts = np.zeros_like(prob.counts)
    res = oracle_mod.run(prob, beta0=0.1, adapt_interval=100, want_final=True, trace_steps=50)
    # every proposal is accepted
    assert np.all(res["accepts"] == 1000)
    assert np.all(res["trace_accept"] == 1)
    assert np.all(res["trace_logl_prop"] == 0.0)
    # beta grows by 1.1 every M_A steps (acceptance 1 > 0.6), clamped at 1
    want = 0.1
    for _ in range(10):
        want = min(1.1 * want, 1.0)
    assert np.all(res["final_beta"] == want)
    # the state is still N(0, I)
    y = res["final_y"]
    assert abs(y.mean()) < 5 / np.sqrt(y.size)
    assert abs(y.var() - 1.0) < 5 * np.sqrt(2.0 / y.size)
    rho, _, _ = oracle_mod.evaluate(prob, y, want_p=False)
    D = 1 << q
    pur = np.einsum("nab,nba->n", rho, rho).real
    assert abs(pur.mean() - (5 * D * D + 1) / (2 * D * (D * D + 2))) < 5 * pur.std() / np.sqrt(pur.size)
    # pooled mean is I/D
    se = 5 * 0.5 / np.sqrt(2048)
    assert np.abs(res["mean"] - np.eye(D) / D).max() < se


def test_low_acceptance_shrinks_beta(oracle_mod):
    prob = W.config_problem(2, num_chains=16, num_steps=200)
    res = oracle_mod.run(prob, beta0=1.0, adapt_interval=50, want_final=True)
    rate = res["accepts"] / 200.0
    assert rate.max() < 0.2
    assert np.allclose(res["final_beta"], 1.0 / 1.1 ** 4, rtol=0, atol=0)


def test_fixed_beta_without_adaptation(oracle_mod):
    prob = W.config_problem(2, num_chains=8, num_steps=300)
    res = oracle_mod.run(prob, beta0=0.05, adapt_interval=0, want_final=True)
    assert np.all(res["final_beta"] == 0.05)


@pytest.mark.parametrize("thin,burn", [(1, 0), (3, 0), (4, 10), (7, 21)])
def test_thinning_and_burn_in(oracle_mod, thin, burn):
    prob = W.config_problem(1, num_chains=5, num_steps=100)
    res = oracle_mod.run(prob, thin=thin, burn_in=burn, traj_chains=2, traj_capacity=200)
    kept = 100 // thin - burn // thin
    assert res["num_pooled"] == 5 * kept
    traj = res["traj"][:, :kept]
    assert np.abs(np.einsum("cnaa->cn", traj) - 1).max() < 1e-13
    assert np.abs(res["traj"][:, kept:]).max() == 0.0


def test_accept_rule_in_trace(oracle_mod):
    prob = W.config_problem(2, num_chains=32, num_steps=200)
    res = oracle_mod.run(prob, trace_steps=200)
    acc = res["trace_accept"].astype(bool)
    rule = res["trace_log_alpha"] < res["trace_logl_prop"] - res["trace_logl_cur"]
    assert np.array_equal(acc, rule)
    assert 0 < acc.mean() < 1


def test_chains_are_independent(oracle_mod):
    """Chain r's result depends only on its global id: running ids [0,6) at once or as
    [0,2) and [2,6) gives bit-identical per-chain pools and final states."""
    prob = W.config_problem(2, num_chains=6, num_steps=120)
    full = oracle_mod.run(prob, want_final=True, want_chain_pool=True)
    a = oracle_mod.run(prob, num_chains=2, chain_begin=0, want_final=True, want_chain_pool=True)
    b = oracle_mod.run(prob, num_chains=4, chain_begin=2, want_final=True, want_chain_pool=True)
    assert np.array_equal(np.concatenate([a["chain_pool"], b["chain_pool"]]), full["chain_pool"])
    assert np.array_equal(np.concatenate([a["final_y"], b["final_y"]]), full["final_y"])
    assert a["num_pooled"] + b["num_pooled"] == full["num_pooled"]
