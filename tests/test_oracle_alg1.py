"""Pins of the oracle's Algorithm 1 (x -> rho through the Bures construction).

* QR + phase fix against LAPACK's Householder QR (numpy) with the fix applied
  here: U is the unique unitary factor whose R has a positive real diagonal.
* rho is Hermitian, unit-trace, positive semidefinite (Sec. II; Sec. III says
  Algorithm 1 enforces both automatically).
* The law of rho is the Bures measure (Sec. III, citing Sommers & Zyczkowski 2003
  and Al Osipov et al. 2010): for a qubit the Bloch radius has density
  (4/pi) r^2 / sqrt(1 - r^2), and for any D the mean purity is
  (5 D^2 + 1) / (2 D (D^2 + 2)) -- 7/8 for a qubit, versus 2D/(D^2+1) for the
  Hilbert-Schmidt law a dropped "+ I" would give.
* E[rho] = I/D by unitary invariance.
"""
import numpy as np
import pytest
from scipy import stats

from paper_2501_17334_gb300 import workload as W


def _lapack_unitary(H):
    q, r = np.linalg.qr(H)
    lam = np.diag(r) / np.abs(np.diag(r))
    return q * lam[None, :]


@pytest.mark.parametrize("D", [2, 4, 8, 16, 32])
def test_qr_unitary_matches_lapack(oracle_mod, D):
    rng = np.random.default_rng(D)
    for _ in range(5):
        H = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
        U, rd = oracle_mod.qr_unitary(H)
        assert np.abs(U.conj().T @ U - np.eye(D)).max() < 1e-13
        # R' = U^dag H is upper triangular with a positive real diagonal
        Rp = U.conj().T @ H
        assert np.abs(np.tril(Rp, -1)).max() < 1e-12 * np.abs(H).max()
        assert np.all(np.diag(Rp).real > 0)
        assert np.abs(np.diag(Rp).imag).max() < 1e-12 * np.abs(H).max()
        assert np.abs(U - _lapack_unitary(H)).max() < 1e-12
        # the diagonal of R before the fix has the modulus of the fixed one
        assert np.allclose(np.abs(rd), np.diag(Rp).real, rtol=1e-12)


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_rho_is_a_density_matrix(oracle_mod, q):
    prob = W.config_problem(min(q, 4), num_chains=1, num_steps=1)
    x = W.latent_batch(200, q, seed=10 + q)
    rho, p, ll = oracle_mod.evaluate(prob, x)
    D = 1 << q
    assert np.abs(np.einsum("naa->n", rho) - 1).max() < 1e-13
    assert np.abs(rho - rho.conj().transpose(0, 2, 1)).max() < 1e-15
    assert np.linalg.eigvalsh(rho).min() > -1e-14
    assert rho.shape == (200, D, D)


def test_latent_layout_column_major(oracle_mod):
    """G, H fill column-major from x (the reading of Algorithm 1 steps 2-3 in MATLAB order):
    permuting x into row-major order must change rho, and the column-major build agrees."""
    q, D = 2, 4
    prob = W.config_problem(2, num_chains=1, num_steps=1)
    x = W.latent_batch(1, q, seed=3)[0]
    d2 = D * D
    G = (x[:d2] + 1j * x[d2:2 * d2]).reshape(D, D, order="F")
    H = (x[2 * d2:3 * d2] + 1j * x[3 * d2:]).reshape(D, D, order="F")
    U = _lapack_unitary(H)
    Wm = (U + np.eye(D)) @ G
    want = Wm @ Wm.conj().T
    want /= np.trace(want).real
    rho, _, _ = oracle_mod.evaluate(prob, x)
    assert np.abs(rho[0] - want).max() < 1e-13
    xt = np.concatenate([b.reshape(D, D).T.reshape(-1) for b in x.reshape(4, d2)])
    rho_t, _, _ = oracle_mod.evaluate(prob, xt)
    assert np.abs(rho_t[0] - rho[0]).max() > 1e-3


def test_qubit_bures_radial_law(oracle_mod):
    prob = W.config_problem(1, num_chains=1, num_steps=1)
    x = W.latent_batch(40000, 1, seed=2024)
    rho, _, _ = oracle_mod.evaluate(prob, x, want_p=False)
    purity = np.einsum("nab,nba->n", rho, rho).real
    r = np.sqrt(np.clip(2 * purity - 1, 0, 1))
    cdf = lambda t: (2 / np.pi) * (np.arcsin(np.clip(t, 0, 1)) - t * np.sqrt(np.clip(1 - t * t, 0, 1)))
    assert stats.kstest(r, cdf).pvalue > 1e-3
    # E[r^2] = 3/4  <=>  E[Tr rho^2] = 7/8
    se = purity.std() / np.sqrt(purity.size)
    assert abs(purity.mean() - 7 / 8) < 4 * se


@pytest.mark.parametrize("q", [1, 2, 3])
def test_bures_mean_purity_and_mean(oracle_mod, q):
    D = 1 << q
    prob = W.config_problem(q, num_chains=1, num_steps=1)
    x = W.latent_batch(20000, q, seed=500 + q)
    rho, _, _ = oracle_mod.evaluate(prob, x, want_p=False)
    purity = np.einsum("nab,nba->n", rho, rho).real
    se = purity.std() / np.sqrt(purity.size)
    bures = (5 * D * D + 1) / (2 * D * (D * D + 2))
    hilbert_schmidt = 2 * D / (D * D + 1)
    assert abs(purity.mean() - bures) < 4 * se
    assert abs(purity.mean() - hilbert_schmidt) > 20 * se
    m = rho.mean(axis=0)
    se_m = rho.std(axis=0).max() / np.sqrt(rho.shape[0])
    assert np.abs(m - np.eye(D) / D).max() < 5 * se_m
