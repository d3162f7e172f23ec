"""QST_PREC_AUTO: the projection form chosen per problem of one handle.

A batch of uneven problems (Pauli measurements at two, four and five qubits, entangled dyadic
bases at three qubits, Haar-random bases at two) runs in one handle with the form of every
problem picked at creation.  The forms must be the ones that apply (the dyadic bases only on
the tensor cores, the Haar-random bases only in FP32, the Pauli problems either), the fixed rule
without timing must give the structured form from five qubits on, and every problem's chains
must equal, bit for bit in the latent states, those of a handle of that problem alone in the
chosen form.
"""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W

pytestmark = pytest.mark.gpu


def _batch():
    return [W.config_problem(2, num_chains=512, num_steps=20),
            W.config_problem(4, num_chains=2048, num_steps=20),
            W.five_qubit_problem(num_chains=256, num_steps=20),
            W.dyadic_basis_problem(3, num_chains=256, num_steps=20),
            W.random_basis_problem(2, 8, num_chains=256, num_steps=20)]


def test_auto_form_per_problem(qst, cuda_ok):
    probs = _batch()
    s = qst.Sampler(probs, precision=qst.PREC_AUTO, diag_chains=0)
    s.run_chains(20)
    forms = [s.diagnostics(i)["projection_form"] for i in range(len(probs))]
    assert forms[3] == qst.PREC_BF16X3 and forms[4] == qst.PREC_FP32
    assert all(f in (qst.PREC_BF16X3, qst.PREC_PAULI) for f in forms[:3])
    for i, p in enumerate(probs):
        ref = qst.Sampler(p, precision=forms[i], diag_chains=0, autotune=0)
        ref.run_chains(20)
        a, b = s.get_state(i), ref.get_state()
        ref.close()
        assert np.array_equal(a["y"], b["y"]), (i, forms[i])
        assert np.array_equal(a["accepts"], b["accepts"])
        assert np.allclose(a["logl"], b["logl"], rtol=1e-12, atol=0)
    s.close()
    rule = qst.Sampler(probs, precision=qst.PREC_AUTO, diag_chains=0, autotune=0)
    assert [rule.diagnostics(i)["projection_form"] for i in range(len(probs))] == \
        [qst.PREC_BF16X3, qst.PREC_BF16X3, qst.PREC_PAULI, qst.PREC_BF16X3, qst.PREC_FP32]
    rule.close()
