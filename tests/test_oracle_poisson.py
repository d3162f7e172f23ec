"""Pins of the oracle's Poisson likelihood (a non-multinomial likelihood: the paper's method
changes only the likelihood step of Algorithm 2 for it, Sec. III).

The counts c_kl are independent Poisson variables of mean mu_k p_kl, p_kl = Tr(Lambda_kl rho),
mu_k the expected trials of setting k; the elements of a setting need not sum to the identity
(lossy detectors).  log L = sum_kl [c_kl log(mu_k p_kl) - mu_k p_kl], the data-only - log c!
left out as the multinomial form leaves out its coefficient.

* the definition against scipy's Poisson log-pmf (plus log c!);
* for complete POVMs (sum_l p_kl = 1) it differs from the multinomial log L by the constant
  sum_kl c_kl log mu_k - sum_k mu_k, whatever rho is;
* the zero-count and p <= 0 conventions;
* Algorithm 2 under it: the pooled posterior mean of a qubit measured through lossy detectors
  against quadrature of the Bures prior times that likelihood, and far from the posterior the
  multinomial likelihood of the same counts gives.
"""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W

SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, -1j], [1j, 0]])
SZ = np.array([[1, 0], [0, -1]], dtype=complex)


def _qubit(r):
    return (np.eye(2) + r[0] * SX + r[1] * SY + r[2] * SZ) / 2


def test_poisson_loglik_matches_scipy(oracle_mod):
    stats = pytest.importorskip("scipy.stats")
    special = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(5)
    D, K = 4, 9
    p = rng.dirichlet(np.ones(D), size=K).reshape(-1) * rng.uniform(0.5, 1.0, K * D)
    mu = rng.uniform(50.0, 500.0, K)
    lam = np.repeat(mu, D) * p
    c = rng.poisson(lam).astype(np.int32)
    c[3] = 0
    ref = np.sum(stats.poisson.logpmf(c, lam) + special.gammaln(c + 1.0))
    got = oracle_mod.loglik_poisson(c, p, mu)
    assert abs(got - ref) < 1e-9 * abs(ref)


def test_complete_povm_differs_from_multinomial_by_a_constant(oracle_mod):
    prob = W.config_problem(2, num_chains=8)
    K, D = prob.num_povms, prob.dim
    mu = np.random.default_rng(3).uniform(100.0, 2000.0, K)
    c = prob.counts.astype(np.float64)
    const = np.sum(c * np.repeat(np.log(mu), D)) - mu.sum()
    x = W.latent_batch(6, 2, seed=9).astype(np.float64)
    rhos, ps, _ = oracle_mod.evaluate(prob, x)
    for p in ps:
        diff = oracle_mod.loglik_poisson(prob.counts, p, mu) - oracle_mod.loglik(prob.counts, p)
        assert abs(diff - const) < 1e-8 * abs(const)


def test_poisson_conventions(oracle_mod):
    mu = np.array([10.0])
    c = np.array([0, 3], dtype=np.int32)
    p = np.array([0.25, 0.5])
    # an outcome never observed contributes - mu p only
    assert np.isclose(oracle_mod.loglik_poisson(c, p, mu), -2.5 + 3 * np.log(5.0) - 5.0, rtol=1e-14)
    # a counted outcome with p <= 0 gives -inf
    assert oracle_mod.loglik_poisson(c, np.array([0.25, 0.0]), mu) == -np.inf
    assert oracle_mod.loglik_poisson(c, np.array([0.25, -0.1]), mu) == -np.inf


def _lossy_qubit_problem(eta, trials, r_true, num_chains, num_steps, seed):
    re, im = W.pauli_povms(1)
    re = re * eta[:, None, None]
    im = im * eta[:, None, None]
    rho = _qubit(r_true)
    p = np.einsum("mab,ba->m", re + 1j * im, rho).real
    mu = np.full(3, float(trials))
    counts = np.random.default_rng(seed).poisson(np.repeat(mu, 2) * p).astype(np.int32)
    return W.Problem(1, re, im, counts, rho, num_chains, num_steps, 0.1, seed + 1, "lossy_qubit",
                     likelihood=1, trials=mu)


def _quadrature(logl_of_r, n=96):
    """Posterior mean Bloch vector under the Bures prior on the full ball (|r| = sin psi)."""
    xg, wg = np.polynomial.legendre.leggauss(n)
    psi, wpsi = (xg + 1) * np.pi / 4, wg * np.pi / 4
    th, wth = (xg + 1) * np.pi / 2, wg * np.pi / 2
    ph, wph = (xg + 1) * np.pi, wg * np.pi
    P, T, F = np.meshgrid(psi, th, ph, indexing="ij")
    s = np.sin(P)
    R = [s * np.sin(T) * np.cos(F), s * np.sin(T) * np.sin(F), s * np.cos(T)]
    meas = np.sin(P) ** 2 * np.sin(T)   # Bures: s^2 (1 - s^2)^(-1/2) ds = sin^2(psi) dpsi
    w3 = wpsi[:, None, None] * wth[None, :, None] * wph[None, None, :]
    lw = logl_of_r(R) + np.log(meas * w3 + 1e-300)
    w = np.exp(lw - lw.max())
    return np.array([(w * R[a]).sum() / w.sum() for a in range(3)])


def test_qubit_posterior_under_poisson_by_quadrature(oracle_mod):
    eta = np.array([1.0, 0.5, 0.75, 0.5, 0.5, 1.0])   # per outcome (X+, X-, Y+, Y-, Z+, Z-)
    prob = _lossy_qubit_problem(eta, 12.0, [0.3, -0.4, 0.5], 512, 3000, seed=31)
    c = prob.counts.reshape(3, 2).astype(float)
    mu = prob.trials

    def poisson(R):
        out = 0.0
        for a in range(3):
            for s, sign in enumerate((1.0, -1.0)):
                lam = mu[a] * eta[2 * a + s] * (1 + sign * R[a]) / 2
                out = out + c[a, s] * np.log(lam) - lam
        return out

    def multinomial(R):   # the same counts read as multinomial (the detectors' losses ignored)
        return sum(c[a, 0] * np.log((1 + R[a]) / 2) + c[a, 1] * np.log((1 - R[a]) / 2) for a in range(3))

    quad = _quadrature(poisson)
    assert np.abs(quad - _quadrature(poisson, n=128)).max() < 1e-10
    other = _quadrature(multinomial)
    res = oracle_mod.run(prob, burn_in=1000, want_chain_pool=True)
    per_chain = res["chain_pool"] / (res["num_pooled"] / 512)
    rc = np.stack([np.einsum("nab,ba->n", per_chain, S).real for S in (SX, SY, SZ)], 1)
    mean, se = rc.mean(0), rc.std(0) / np.sqrt(512)
    assert np.all(np.abs(mean - quad) < 4 * se), (mean, quad, se)
    assert np.any(np.abs(mean - other) > 8 * se), (mean, other, se)
