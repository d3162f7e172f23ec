"""Oracle pins for the Pauli projectors built entry by entry (no POVM arrays): the same p as the
dense arrays of the seeded-input module at small Q, and at six qubits (where the dense arrays
would take 3 GB) properties that fix p: each setting's outcomes sum to Tr rho, every p of a
density matrix is in [0, 1], and individual p_kl equal Tr(Lambda_kl rho) with Lambda_kl formed
here as a Kronecker product of the single-qubit eigenprojectors."""
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W

# single-qubit eigenprojectors, [setting X, Y, Z][outcome +1, -1]
_X = np.array([[0, 1], [1, 0]], complex)
_Y = np.array([[0, -1j], [1j, 0]])
_Z = np.diag([1.0, -1.0]).astype(complex)
_PROJ = [[(np.eye(2) + P) / 2, (np.eye(2) - P) / 2] for P in (_X, _Y, _Z)]


def _random_rho(D, rng, rank=None):
    g = rng.standard_normal((D, rank or D)) + 1j * rng.standard_normal((D, rank or D))
    r = g @ g.conj().T
    return r / np.trace(r).real


def _lambda(Q, k, l):
    m = np.ones((1, 1), complex)
    for q in range(Q):
        s = (k // 3 ** (Q - 1 - q)) % 3
        b = (l >> (Q - 1 - q)) & 1
        m = np.kron(m, _PROJ[s][b])
    return m


def _problem(Q, dense):
    D = 1 << Q
    re, im = W.pauli_povms(Q) if dense else (None, None)
    return SimpleNamespace(dim=D, num_povms=3 ** Q, povm_re=re, povm_im=im)


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_builtin_pauli_projectors_match_the_dense_arrays(oracle_mod, q):
    rho = _random_rho(1 << q, np.random.default_rng(60 + q))
    p_dense = oracle_mod.probabilities(_problem(q, True), rho)
    p_built = oracle_mod.probabilities(_problem(q, False), rho)
    assert np.allclose(p_dense, p_built, atol=1e-15, rtol=0)


def test_six_qubit_pauli_probabilities(oracle_mod):
    Q, D = 6, 64
    rng = np.random.default_rng(66)
    rho = _random_rho(D, rng, rank=3)
    p = oracle_mod.probabilities(_problem(Q, False), rho).reshape(3 ** Q, D)
    assert np.allclose(p.sum(axis=1), 1.0, atol=1e-12)
    assert p.min() > -1e-13 and p.max() < 1 + 1e-13
    for k, l in [(0, 0), (1, 5), (364, 17), (728, 63), (500, 42)]:
        assert abs(p[k, l] - np.real(np.trace(_lambda(Q, k, l) @ rho))) < 1e-14
