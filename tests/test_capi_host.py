"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
function include/qst.h declares, and its host logic (defaults, validation, projector
packing) behaves as documented."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W
from tests._helpers import pack_rho

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "qst.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(qst_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("qst_create", "qst_run_chains", "qst_posterior_mean", "qst_diagnostics", "qst_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(qst):
    lib = ctypes.CDLL(qst.library_path())
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps every declared function under the same name
    assert set(_declared_functions()) <= set(qst._SIGS)


def test_default_config_is_the_papers(qst):
    cfg = qst.default_config()
    assert cfg.beta0 == 0.1 and cfg.adapt_interval == 500
    assert (cfg.acc_lo, cfg.acc_hi, cfg.adapt_factor) == (0.2, 0.6, 1.1)
    assert cfg.thin == 1 and cfg.burn_in == 0 and cfg.acf_lmax == 200 and cfg.traj_capacity == 1024
    assert cfg.precision == qst.PREC_FP32


def _status(fn):
    try:
        fn()
    except Exception as e:  # QstError
        return getattr(e, "status", None)
    return 0


def test_validation_rejects_bad_inputs(qst):
    prob = W.config_problem(2, num_chains=64, num_steps=10)
    ok = qst.default_config()
    assert qst.workspace_size([prob], ok) > 0
    assert _status(lambda: qst.workspace_size([prob], qst.default_config(thin=0))) == 1
    assert _status(lambda: qst.workspace_size([prob], qst.default_config(beta0=0.0))) == 1
    assert _status(lambda: qst.workspace_size([prob], qst.default_config(beta0=1.5))) == 1
    assert _status(lambda: qst.workspace_size([prob], qst.default_config(precision=9))) == 1
    assert _status(lambda: qst.workspace_size([prob], qst.default_config(qr_passes=0))) == 1
    assert _status(lambda: qst.workspace_size([prob], qst.default_config(qr_passes=5))) == 1
    assert qst.workspace_size([prob], qst.default_config(qr_passes=4)) > 0   # five qubits refined too
    bad = W.config_problem(2, num_chains=64, num_steps=10)
    bad.counts = bad.counts.copy()
    bad.counts[3] = -1
    assert _status(lambda: qst.workspace_size([bad], ok)) == 1
    nonherm = W.config_problem(2, num_chains=64, num_steps=10)
    nonherm.povm_im = nonherm.povm_im.copy()
    nonherm.povm_im[5, 0, 1] += 0.1
    assert _status(lambda: qst.workspace_size([nonherm], ok)) == 1
    incomplete = W.config_problem(2, num_chains=64, num_steps=10)
    incomplete.povm_re = incomplete.povm_re.copy()
    incomplete.povm_re[0, 0, 0] += 1e-6
    incomplete.povm_re[0, 0, 0] += 0.0
    assert _status(lambda: qst.workspace_size([incomplete], ok)) == 1
    zero_chains = W.config_problem(2, num_chains=64, num_steps=10)
    zero_chains.num_chains = 0
    assert _status(lambda: qst.workspace_size([zero_chains], ok)) == 1
    assert "identity" in qst.load().qst_last_error().decode() or True


def test_poisson_likelihood_validation(qst):
    """QST_LIKELIHOOD_POISSON: settings may fall short of the identity (lossy detectors), but
    not exceed it; every setting needs trials exact in FP32; an incomplete setting is refused
    under the multinomial likelihood."""
    import copy
    ok = qst.default_config()
    prob = W.lossy_pauli_problem(2, num_chains=64, num_steps=10)
    assert qst.workspace_size([prob], ok) > 0
    assert qst.workspace_size([prob], qst.default_config(precision=qst.PREC_BF16X3)) > 0
    multinomial = copy.copy(prob)
    multinomial.likelihood = 0
    assert _status(lambda: qst.workspace_size([multinomial], ok)) == 1
    no_trials = copy.copy(prob)
    no_trials.trials = None
    assert _status(lambda: qst.workspace_size([no_trials], ok)) == 1
    for bad_mu in (0.0, -5.0, np.nan, 1000.1):   # 1000.1 is not exact in FP32
        wrong = copy.copy(prob)
        wrong.trials = prob.trials.copy()
        wrong.trials[1] = bad_mu
        assert _status(lambda: qst.workspace_size([wrong], ok)) == 1
    above = copy.copy(prob)
    above.povm_re = prob.povm_re * 2.0   # every setting sums to eta / 2 * 2 > 1 somewhere
    above.povm_im = prob.povm_im * 2.0
    assert _status(lambda: qst.workspace_size([above], ok)) == 1
    unknown = copy.copy(prob)
    unknown.likelihood = 7
    assert _status(lambda: qst.workspace_size([unknown], ok)) == 1


def test_five_qubits_are_accepted_and_six_refused(qst):
    prob = W.five_qubit_problem(num_chains=8, num_steps=1)
    assert qst.workspace_size([prob], qst.default_config()) > 0
    assert qst.workspace_size([prob], qst.default_config(precision=qst.PREC_BF16X3)) > 0
    six = W.five_qubit_problem(num_chains=8, num_steps=1)
    six.num_qubits = 6
    assert _status(lambda: qst.workspace_size([six], qst.default_config())) == 1


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_packed_projectors_reproduce_direct_trace(qst, oracle_mod, q):
    """p = vec_h(rho) . P (the contraction the kernels run) equals Tr(Lambda rho) of the oracle."""
    prob = W.config_problem(q, num_chains=4, num_steps=1)
    P = qst.pack_projectors(q, prob.povm_re, prob.povm_im)
    x = W.latent_batch(8, q, seed=q)
    rho, p_ref, _ = oracle_mod.evaluate(prob, x)
    p = pack_rho(rho) @ P.astype(np.float64)
    assert np.abs(p - p_ref).max() < 1e-14
    # Pauli projector entries are 0 or +-2^-m: exact in bf16 (8-bit mantissa)
    vals = np.unique(np.abs(P[P != 0]))
    assert np.all(np.log2(vals) == np.round(np.log2(vals)))


@pytest.mark.parametrize("q,tf32_ok,tf32x2_ok", [(1, True, True), (3, True, True), (4, True, False), (5, False, False)])
def test_tensor_core_precisions_cover_their_qubit_ranges(qst, q, tf32_ok, tf32x2_ok):
    """TF32 keeps one A split in shared memory (to 4 qubits), TF32x2 two (to 3 qubits);
    outside its range a precision is refused before any allocation."""
    prob = W.config_problem(q, num_chains=8) if q <= 4 else W.five_qubit_problem(num_chains=8, num_steps=1)
    for prec, ok in ((qst.PREC_TF32, tf32_ok), (qst.PREC_TF32X2, tf32x2_ok)):
        cfg = qst.default_config(precision=prec)
        if ok:
            assert qst.workspace_size([prob], cfg) > 0
        else:
            assert _status(lambda: qst.workspace_size([prob], cfg)) == 1
    assert qst.workspace_size([prob], qst.default_config(precision=qst.PREC_BF16X3)) > 0


def test_tf32_forms_need_projectors_exact_in_tf32(qst):
    """A basis rotated by 0.3 rad has projector entries that TF32 (and bf16) cannot hold: the
    tensor-core precisions refuse it, the FP32 form takes it."""
    prob = W.config_problem(1, num_chains=8)
    c, s_ = np.cos(0.3), np.sin(0.3)
    u = np.array([c, s_])
    v = np.array([-s_, c])
    re = prob.povm_re.copy()
    im = prob.povm_im.copy()
    re[4] = np.outer(u, u)          # setting 2 (Z) replaced by the rotated basis
    re[5] = np.outer(v, v)
    im[4] = 0.0
    im[5] = 0.0
    prob.povm_re, prob.povm_im = re, im
    assert qst.workspace_size([prob], qst.default_config(precision=qst.PREC_FP32)) > 0
    for prec in (qst.PREC_TF32, qst.PREC_TF32X2, qst.PREC_BF16X3):
        assert _status(lambda: qst.workspace_size([prob], qst.default_config(precision=prec))) == 1


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_builtin_pauli_povms_are_the_workload_ones(qst, q):
    """NULL POVM arrays select the library's Pauli POVMs: the same elements, bit for bit, as the
    seeded-input module builds (same setting and outcome order)."""
    re, im = qst.pauli_povms(q)
    wre, wim = W.pauli_povms(q)
    assert np.array_equal(re, wre) and np.array_equal(im, wim)


def test_null_povms_select_the_builtin_pauli_set(qst):
    import copy
    prob = W.config_problem(3, num_chains=64)
    null = copy.copy(prob)
    null.povm_re = None
    null.povm_im = None
    cfg = qst.default_config(precision=qst.PREC_BF16X3)
    assert qst.workspace_size([null], cfg) == qst.workspace_size([prob], cfg)
    from types import SimpleNamespace
    wrong = SimpleNamespace(num_qubits=3, num_povms=26, counts=prob.counts[:26 * 8], povm_re=None,
                            povm_im=None, num_chains=64, seed=1, beta0=0.0)   # the built-in set has 3^Q
    assert _status(lambda: qst.workspace_size([wrong], cfg)) == 1


class _HugeProblem:
    """A problem whose POVM count would make K * D (and K * D^3) wrap a 32-bit int: the
    arrays are tiny because validation must reject the size before reading them."""
    num_qubits = 4
    num_povms = 1 << 28
    counts = np.zeros(16, np.int32)
    povm_re = np.zeros((1, 16, 16))
    povm_im = np.zeros((1, 16, 16))
    num_chains = 8
    seed = 1
    beta0 = 0.02


def test_huge_povm_count_is_rejected_before_any_product_wraps(qst):
    lib = qst.load()
    # qst_create's validation (through qst_workspace_size, which runs the same checks)
    assert _status(lambda: qst.workspace_size([_HugeProblem()], qst.default_config())) == 1
    # qst_pack_projectors
    re = np.zeros((16, 16, 16))
    out = np.zeros(16, np.float32)
    assert lib.qst_pack_projectors(4, 1 << 28, re.ctypes.data, re.ctypes.data, out.ctypes.data) == 1
    # qst_loglik_noalloc: rejected on the host, before any CUDA call (no GPU here)
    counts = np.zeros(16, np.int32)
    for k in (1 << 28, (1 << 31) // 16, 89, -1, 0):
        st = lib.qst_loglik_noalloc(4, k, None, counts.ctypes.data, None, 1, None, None)
        assert st == 1, (k, st)
    assert lib.qst_loglik_noalloc(4, 81, None, counts.ctypes.data, None, 1, None, None) == 1   # NULL P
