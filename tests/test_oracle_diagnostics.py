"""Pins of the mixing and accuracy diagnostics (Eq. ACFrho, Eq. IACT, Eq. fid, Eq. fro).

* A scalar AR(1) series x_n = phi x_{n-1} + e_n embedded in one real component of
  rho has c[l] = phi^l and tau = (1 + phi)/(1 - phi); an i.i.d. series has tau = 1.
* Fidelity: F(rho, rho) = 1; for a pure sigma = |psi><psi|, F = <psi|rho|psi>; for
  commuting diagonal states, F = (sum_i sqrt(p_i q_i))^2.
"""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W


def _ar1_traj(phi, n, D, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros(n)
    e = rng.standard_normal(n) * np.sqrt(1 - phi * phi)
    x[0] = rng.standard_normal()
    for i in range(1, n):
        x[i] = phi * x[i - 1] + e[i]
    traj = np.tile(np.eye(D, dtype=complex) / D, (n, 1, 1))
    traj[:, 0, 1] += 0.01 * x
    traj[:, 1, 0] += 0.01 * x
    return traj


@pytest.mark.parametrize("phi", [0.0, 0.5, 0.8])
def test_acf_iact_ar1(oracle_mod, phi):
    traj = _ar1_traj(phi, 200000, 2, seed=int(phi * 10))
    c = oracle_mod.acf(traj, 200)
    assert c[0] == 1.0
    assert np.abs(c[1:6] - phi ** np.arange(1, 6)).max() < 0.02
    tau = oracle_mod.iact(c)
    assert tau == pytest.approx((1 + phi) / (1 - phi), abs=0.15 * (1 + phi) / (1 - phi) + 0.05)


def test_acf_weights_real_and_imaginary_parts(oracle_mod):
    """Eq. ACFa: the sum runs over every (i, j) entry's real and imaginary parts."""
    rng = np.random.default_rng(1)
    n, D = 400, 2
    traj = np.tile(np.eye(D, dtype=complex) / D, (n, 1, 1))
    a = rng.standard_normal(n)
    b = rng.standard_normal(n)
    traj[:, 0, 1] += 0.01 * (a + 1j * b)
    traj[:, 1, 0] += 0.01 * (a - 1j * b)
    c = oracle_mod.acf(traj, 10)
    dev_a, dev_b = a - a.mean(), b - b.mean()
    m = n - 10
    raw = [2 * np.sum(dev_a[:m] * dev_a[l:l + m] + dev_b[:m] * dev_b[l:l + m]) for l in range(11)]
    assert np.allclose(c, np.array(raw) / raw[0], atol=1e-12)


def test_fidelity_pins(oracle_mod):
    rng = np.random.default_rng(3)
    for D in (2, 4, 8):
        rho = W.ginibre_state(D, D, rng)
        assert oracle_mod.fidelity(rho, rho) == pytest.approx(1.0, abs=1e-10)
        psi = rng.standard_normal(D) + 1j * rng.standard_normal(D)
        psi /= np.linalg.norm(psi)
        sigma = np.outer(psi, psi.conj())
        want = (psi.conj() @ rho @ psi).real
        assert oracle_mod.fidelity(sigma, rho) == pytest.approx(want, abs=1e-10)
        assert oracle_mod.fidelity(rho, sigma) == pytest.approx(want, abs=1e-10)
        p = rng.dirichlet(np.ones(D))
        q = rng.dirichlet(np.ones(D))
        assert oracle_mod.fidelity(np.diag(p).astype(complex), np.diag(q).astype(complex)) == \
            pytest.approx(np.sum(np.sqrt(p * q)) ** 2, abs=1e-12)


def test_frobenius(oracle_mod):
    a = np.array([[1, 2j], [-2j, 3]])
    b = np.array([[0, 1j], [-1j, 1]])
    assert oracle_mod.frobenius_sq(a, b) == pytest.approx(1 + 1 + 1 + 4)
