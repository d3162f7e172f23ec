"""Oracle pins for the Hilbert-Schmidt prior (rho = G G^dag / Tr with G a D x D complex Ginibre
matrix): under that measure E[Tr rho^2] = 2 D / (D^2 + 1) and E[rho] = I / D (the induced
measure with an environment of dimension D), values the Bures prior of Algorithm 1 does not
give, so a prior switch that silently kept Algorithm 1 fails here."""
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W


def _problem(q):
    re, im = W.pauli_povms(q)
    D = 1 << q
    return SimpleNamespace(dim=D, num_povms=3 ** q, povm_re=re, povm_im=im,
                           counts=np.zeros(3 ** q * D, np.int32))


@pytest.mark.parametrize("q", [1, 2])
def test_hilbert_schmidt_purity_and_mean(oracle_mod, q):
    D = 1 << q
    n = 20000
    x = W.latent_batch(n, q, seed=90 + q)
    rho, _, _ = oracle_mod.evaluate(_problem(q), x, want_p=False, prior=oracle_mod.PRIOR_HS)
    purity = np.einsum("nij,nji->n", rho, rho).real
    expect = 2 * D / (D * D + 1)
    assert abs(purity.mean() - expect) < 4 * purity.std() / np.sqrt(n)
    se = np.sqrt(rho.real.var(axis=0) + rho.imag.var(axis=0)) / np.sqrt(n)   # per entry
    assert np.all(np.abs(rho.mean(axis=0) - np.eye(D) / D) < 5 * se + 1e-12)
    # and the Bures map on the same latents does not reproduce that purity
    rho_b, _, _ = oracle_mod.evaluate(_problem(q), x, want_p=False)
    purity_b = np.einsum("nij,nji->n", rho_b, rho_b).real
    assert abs(purity_b.mean() - expect) > 10 * purity.std() / np.sqrt(n)


def test_hilbert_schmidt_uses_only_g(oracle_mod):
    """H (the last 2 D^2 latent entries) does not enter the Hilbert-Schmidt rho."""
    q = 2
    x = W.latent_batch(4, q, seed=5)
    y = x.copy()
    y[:, 2 * 16:] = W.latent_batch(4, q, seed=6)[:, 2 * 16:]
    a, _, _ = oracle_mod.evaluate(_problem(q), x, want_p=False, prior=oracle_mod.PRIOR_HS)
    b, _, _ = oracle_mod.evaluate(_problem(q), y, want_p=False, prior=oracle_mod.PRIOR_HS)
    assert np.array_equal(a, b)
