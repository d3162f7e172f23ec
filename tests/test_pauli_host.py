"""Host checks of the structured Pauli form (no GPU): the block-split identities it is built on,
written out here in numpy on the packed layout, reproduce p_kl = Tr(Lambda_kl rho) of the
oracle's direct trace for random density matrices, in the tree's output order; and the C ABI
accepts the form for the Pauli POVMs only.

The split: fixing the outcome of the most significant remaining qubit of a Hermitian block
M = [[A, B], [B^dag, C]] leaves (A + C +- (B + B^dag)) / 2 for X, (A + C +- i(B - B^dag)) / 2
for Y, and A, C for Z (the partial trace of (Pi (x) 1) M over that qubit).  Each function
below restates one piece of that in plain numpy so that a sign, a transposition or an order
mistake in the kernel's formulas shows up here first."""
import numpy as np
import pytest

from paper_2501_17334_gb300 import workload as W
from tests._helpers import pack_rho


def _packed(rho):
    D = rho.shape[0]
    return pack_rho(rho[None])[0].reshape(D, D)


def _random_rho(D, rng):
    g = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    r = g @ g.conj().T
    return r / np.trace(r).real


def _children_complex(M):
    """The six blocks of one split, on full complex matrices (the definition)."""
    h = M.shape[0] // 2
    A, B, C = M[:h, :h], M[:h, h:], M[h:, h:]
    S = A + C
    X = B + B.conj().T
    Y = 1j * (B - B.conj().T)
    return [(S + X) / 2, (S - X) / 2, (S + Y) / 2, (S - Y) / 2, A, C]


def _children_packed(P):
    """The same six blocks computed from the packed form only, entry by entry, with the
    kernel's formulas (entries on and above the diagonal: real parts; below: imaginary parts)."""
    n = P.shape[0]
    h = n // 2
    TL, BR, TR, BL = P[:h, :h], P[h:, h:], P[:h, h:], P[h:, :h]
    out = [np.zeros((h, h)) for _ in range(6)]
    for u in range(h):
        for v in range(h):
            s = TL[u, v] + BR[u, v]
            if u <= v:
                x = TR[u, v] + TR[v, u]
                y = BL[u, v] + BL[v, u]
            else:
                x = BL[u, v] - BL[v, u]
                y = TR[u, v] - TR[v, u]
            vals = [(s + x) / 2, (s - x) / 2, (s + y) / 2, (s - y) / 2, TL[u, v], BR[u, v]]
            for c in range(6):
                out[c][u, v] = vals[c]
    return out


def _tree_packed(P):
    """All Q splits on the packed form -> 6^Q values in tree order (first split most significant)."""
    blocks = [P]
    while blocks[0].shape[0] > 1:
        blocks = [child for b in blocks for child in _children_packed(b)]
    return np.array([b[0, 0] for b in blocks])


def _tree_order(Q):
    """Tree output o -> setting-major projector index k D + l."""
    D = 1 << Q
    perm = np.zeros(6 ** Q, dtype=np.int64)
    for o in range(6 ** Q):
        digits = [(o // 6 ** (Q - 1 - q)) % 6 for q in range(Q)]
        k = sum((dg // 2) * 3 ** (Q - 1 - q) for q, dg in enumerate(digits))
        l = sum((dg % 2) << (Q - 1 - q) for q, dg in enumerate(digits))
        perm[o] = k * D + l
    return perm


def _direct_p(rho, Q):
    re, im = W.pauli_povms(Q)
    lam = re + 1j * im
    return np.real(np.einsum("mij,ji->m", lam, rho))


@pytest.mark.parametrize("q", [1, 2, 3])
def test_one_split_matches_the_partial_trace(q):
    rng = np.random.default_rng(40 + q)
    rho = _random_rho(1 << q, rng)
    full = _children_complex(rho)
    packed = _children_packed(_packed(rho))
    for c in range(6):
        assert np.allclose(packed[c], _packed(full[c]), atol=1e-14)
        assert np.allclose(full[c], full[c].conj().T, atol=1e-14)   # every child is Hermitian


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_tree_gives_every_pauli_probability(q):
    rng = np.random.default_rng(10 + q)
    for _ in range(3):
        rho = _random_rho(1 << q, rng)
        vals = _tree_packed(_packed(rho))
        p = np.empty(6 ** q)
        p[_tree_order(q)] = vals
        assert np.allclose(p, _direct_p(rho, q), atol=1e-13)


def test_tree_order_is_a_permutation():
    for q in range(1, 6):
        perm = _tree_order(q)
        assert np.array_equal(np.sort(perm), np.arange(6 ** q))


def test_capi_takes_the_pauli_form_for_pauli_povms_only(qst):
    import copy
    prob = W.config_problem(2, num_chains=16)
    cfg = qst.default_config(precision=qst.PREC_PAULI)
    assert qst.workspace_size([prob], cfg) > 0
    null = copy.copy(prob)
    null.povm_re = None
    null.povm_im = None
    assert qst.workspace_size([null], cfg) > 0
    # a rotated basis in place of one setting: a valid POVM, but not the Pauli set
    c, s_ = np.cos(0.3), np.sin(0.3)
    rot = copy.copy(prob)
    re = prob.povm_re.copy()
    im = prob.povm_im.copy()
    u, v = np.array([c, s_]), np.array([-s_, c])
    re[32:36] = np.stack([np.kron(np.outer(a, a), np.outer(b, b))
                          for a in (u, v) for b in (np.array([1.0, 0.0]), np.array([0.0, 1.0]))])
    im[32:36] = 0.0
    rot.povm_re, rot.povm_im = re, im
    assert qst.workspace_size([rot], qst.default_config(precision=qst.PREC_FP32)) > 0
    with pytest.raises(Exception):
        qst.workspace_size([rot], cfg)


def test_six_qubits_only_in_the_pauli_form_with_builtin_povms(qst):
    """Six qubits run only in the structured form, and only with the built-in (NULL) POVM arrays,
    which the library then never materialises; every other combination is refused before any
    allocation."""
    import copy
    p6 = W.six_qubit_problem(num_chains=4, num_steps=1)
    assert p6.povm_re is None and p6.povm_im is None
    assert qst.workspace_size([p6], qst.default_config(precision=qst.PREC_PAULI)) > 0
    for prec in (qst.PREC_FP32, qst.PREC_BF16X3, qst.PREC_TF32, qst.PREC_TF32X2):
        with pytest.raises(Exception):
            qst.workspace_size([p6], qst.default_config(precision=prec))
    # five qubits with NULL arrays still work in the dense forms (materialised there)
    p5 = copy.copy(W.five_qubit_problem(num_chains=4, num_steps=1))
    p5.povm_re = p5.povm_im = None
    assert qst.workspace_size([p5], qst.default_config(precision=qst.PREC_FP32)) > 0
    assert qst.workspace_size([p5], qst.default_config(precision=qst.PREC_PAULI)) > 0
    # seven qubits: refused in every form
    p7 = copy.copy(p6)
    p7.num_qubits = 7
    with pytest.raises(Exception):
        qst.workspace_size([p7], qst.default_config(precision=qst.PREC_PAULI))
