"""Host analysis of the Sec. IV study (paper_2501_17334_gb300.experiment): Frobenius error and
fidelity against closed forms and against the oracle's independent implementation."""
import numpy as np
import pytest

from paper_2501_17334_gb300 import experiment as E


def _rand_state(D, rank, rng):
    g = rng.standard_normal((D, rank)) + 1j * rng.standard_normal((D, rank))
    r = g @ g.conj().T
    return r / np.trace(r).real


def test_fidelity_closed_forms():
    rng = np.random.default_rng(1)
    for D in (2, 4, 8):
        rho = _rand_state(D, D, rng)
        assert abs(E.fidelity(rho, rho) - 1.0) < 1e-12
        # pure states: F = |<psi|phi>|^2
        psi = rng.standard_normal(D) + 1j * rng.standard_normal(D)
        phi = rng.standard_normal(D) + 1j * rng.standard_normal(D)
        psi /= np.linalg.norm(psi)
        phi /= np.linalg.norm(phi)
        f = E.fidelity(np.outer(psi, psi.conj()), np.outer(phi, phi.conj()))
        assert abs(f - abs(np.vdot(psi, phi)) ** 2) < 1e-10
        # commuting (diagonal) states: F = (sum sqrt(p q))^2
        p = rng.random(D)
        q = rng.random(D)
        p /= p.sum()
        q /= q.sum()
        assert abs(E.fidelity(np.diag(p), np.diag(q)) - np.sum(np.sqrt(p * q)) ** 2) < 1e-12
        # symmetric in its arguments
        sig = _rand_state(D, 2, rng)
        assert abs(E.fidelity(sig, rho) - E.fidelity(rho, sig)) < 1e-9


@pytest.mark.parametrize("D", [2, 4, 16])
def test_fidelity_and_frobenius_match_the_oracle(oracle_mod, D):
    rng = np.random.default_rng(D)
    a, b = _rand_state(D, 3, rng), _rand_state(D, D, rng)
    assert abs(E.fidelity(a, b) - oracle_mod.fidelity(a, b)) < 1e-10
    assert abs(E.frobenius_sq(a, b) - np.sum(np.abs(a - b) ** 2)) < 1e-14
    assert E.frobenius_sq(a, a) == 0.0


def test_sweep_rejects_too_few_kept_states(tmp_path):
    with pytest.raises(ValueError):
        E.sweep([1], [0], [1], 200, str(tmp_path))
