"""Pins of the measurement model and likelihood (Sec. II, Sec. III Step 4).

* completeness: sum_l Lambda_kl = I for every Pauli basis, so sum_l p_kl = 1;
* closed forms: a qubit rho = (I + r.sigma)/2 gives p(a, +-) = (1 +- r_a)/2, and a
  product state gives products of single-qubit probabilities;
* |0><0| by hand: p(Z+) = 1, p(Z-) = 0, p(X+-) = p(Y+-) = 1/2;
* log L = sum c log p with 0 log 0 = 0 and -inf for a counted outcome of probability 0.
"""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W

SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, -1j], [1j, 0]])
SZ = np.array([[1, 0], [0, -1]], dtype=complex)


class _P:
    def __init__(self, q, counts=None):
        self.num_qubits = q
        self.dim = 1 << q
        self.num_povms = 3 ** q
        self.povm_re, self.povm_im = W.pauli_povms(q)
        self.counts = np.zeros(self.num_povms * self.dim, np.int32) if counts is None else counts


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_povm_completeness(q):
    re, im = W.pauli_povms(q)
    D = 1 << q
    lam = (re + 1j * im).reshape(3 ** q, D, D, D)
    assert np.abs(lam.sum(axis=1) - np.eye(D)).max() < 1e-14
    # each element is a rank-one projector
    assert np.abs(np.einsum("kab,kbc->kac", lam.reshape(-1, D, D), lam.reshape(-1, D, D))
                  - lam.reshape(-1, D, D)).max() < 1e-14


def test_qubit_closed_form(oracle_mod):
    prob = _P(1)
    rng = np.random.default_rng(0)
    for _ in range(20):
        r = rng.standard_normal(3)
        r *= rng.uniform(0, 1) / np.linalg.norm(r)
        rho = (np.eye(2) + r[0] * SX + r[1] * SY + r[2] * SZ) / 2
        p = oracle_mod.probabilities(prob, rho)
        want = np.array([(1 + r[0]) / 2, (1 - r[0]) / 2, (1 + r[1]) / 2, (1 - r[1]) / 2,
                         (1 + r[2]) / 2, (1 - r[2]) / 2])
        assert np.abs(p - want).max() < 1e-15


def test_ket_zero_by_hand(oracle_mod):
    p = oracle_mod.probabilities(_P(1), np.diag([1.0, 0.0]).astype(complex))
    assert np.allclose(p, [0.5, 0.5, 0.5, 0.5, 1.0, 0.0], atol=1e-16)


def test_product_state_factorises(oracle_mod):
    rng = np.random.default_rng(4)
    a = W.ginibre_state(2, 2, rng)
    b = W.ginibre_state(2, 1, rng)
    p1 = oracle_mod.probabilities(_P(1), a).reshape(3, 2)
    p2 = oracle_mod.probabilities(_P(1), b).reshape(3, 2)
    p12 = oracle_mod.probabilities(_P(2), np.kron(a, b)).reshape(3, 3, 2, 2)
    want = p1[:, None, :, None] * p2[None, :, None, :]
    assert np.abs(p12 - want).max() < 1e-15


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_probabilities_sum_to_one(oracle_mod, q):
    prob = W.config_problem(q, num_chains=1, num_steps=1)
    x = W.latent_batch(20, q, seed=q)
    _, p, _ = oracle_mod.evaluate(prob, x)
    D = 1 << q
    assert np.abs(p.reshape(20, 3 ** q, D).sum(-1) - 1).max() < 1e-13
    assert p.min() > -1e-15


def test_loglik_brute_force(oracle_mod):
    counts = np.array([3, 0, 5, 1, 0, 7], np.int32)
    p = np.array([0.25, 0.75, 0.5, 0.5, 0.0, 1.0])
    want = 3 * np.log(0.25) + 5 * np.log(0.5) + 1 * np.log(0.5) + 7 * np.log(1.0)
    assert oracle_mod.loglik(counts, p) == pytest.approx(want, rel=1e-15)
    counts2 = counts.copy()
    counts2[4] = 1
    assert oracle_mod.loglik(counts2, p) == -np.inf


def test_loglik_of_x_consistent(oracle_mod):
    prob = W.config_problem(2, num_chains=1, num_steps=1)
    x = W.latent_batch(4, 2, seed=9)
    rho, p, ll = oracle_mod.evaluate(prob, x)
    for i in range(4):
        c = prob.counts.astype(float)
        assert ll[i] == pytest.approx(np.sum(c * np.log(p[i])), rel=1e-13)
        assert np.allclose(oracle_mod.probabilities(prob, rho[i]), p[i], atol=1e-15)
