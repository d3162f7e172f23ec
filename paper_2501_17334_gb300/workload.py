"""Seeded synthetic inputs for Pauli quantum state tomography.

This module only *makes data*: the measurement operators, a ground-truth
state, and the multinomial counts an experiment would have recorded
(Step 1 of the method, Sec. III "Steps").  It holds none of the sampler's
arithmetic -- no parameterisation, likelihood, proposal or pooling -- so both
the FP64 oracle and the CUDA path can consume its output as plain data.

Conventions (the paper is silent on them, Sec. IV uses "all possible Pauli
measurement combinations"):

* basis index ``k = sum_q s_q 3**(Q-1-q)`` with ``s = 0, 1, 2`` for X, Y, Z and
  qubit 0 the most significant factor of the Kronecker product;
* outcome index ``l = sum_q b_q 2**(Q-1-q)`` with ``b = 0`` the +1 eigenvalue;
* POVM element ``Lambda_kl`` is row ``k*D + l`` of a ``[K*D, D, D]`` array.

Workloads follow the five benchmark configurations (1 to 5 qubits); the seed of
the truth is ``1000 + c``, of the counts ``2000 + c`` and of the chains
``3000 + c`` for configuration ``c``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import functools

import numpy as np

# single-qubit eigenvectors, index [setting][outcome] ; setting 0=X, 1=Y, 2=Z
_S2 = 1.0 / math.sqrt(2.0)
_EIGVEC = np.array(
    [
        [[_S2, _S2], [_S2, -_S2]],            # X+ , X-
        [[_S2, 1j * _S2], [_S2, -1j * _S2]],  # Y+ , Y-
        [[1.0, 0.0], [0.0, 1.0]],             # Z+ , Z-
    ],
    dtype=np.complex128,
)


@functools.lru_cache(maxsize=None)
def pauli_vectors(num_qubits: int) -> np.ndarray:
    """Measurement vectors ``phi_kl`` (``Lambda_kl = |phi_kl><phi_kl|``), shape ``[K*D, D]``,
    index k*D + l as for ``pauli_povms``.  Cached per Q and read-only."""
    q = int(num_qubits)
    if q < 1:
        raise ValueError("num_qubits must be >= 1")
    t = np.ones((1, 1, 1), dtype=np.complex128)            # [setting, outcome, component]
    for _ in range(q):
        k, l, c = t.shape
        t = np.einsum("klc,sbm->ksblcm", t, _EIGVEC).reshape(k * 3, 2, l, c * 2)
        t = t.transpose(0, 2, 1, 3).reshape(k * 3, l * 2, c * 2)
    out = np.ascontiguousarray(t.reshape(-1, 1 << q))
    out.setflags(write=False)
    return out


# single-qubit eigenprojectors, index [setting][outcome], entries exactly 0, +-1/2, +-i/2, 1
_PROJ = np.array(
    [
        [[[0.5, 0.5], [0.5, 0.5]], [[0.5, -0.5], [-0.5, 0.5]]],            # X+ , X-
        [[[0.5, -0.5j], [0.5j, 0.5]], [[0.5, 0.5j], [-0.5j, 0.5]]],        # Y+ , Y-
        [[[1.0, 0.0], [0.0, 0.0]], [[0.0, 0.0], [0.0, 1.0]]],              # Z+ , Z-
    ],
    dtype=np.complex128,
)


@functools.lru_cache(maxsize=None)
def pauli_povms(num_qubits: int):
    """All ``3**Q`` Pauli-basis POVMs as real and imaginary ``[K*D, D, D]`` float64 arrays.

    Built as Kronecker products of the exact single-qubit projectors, so every entry is
    0 or +-2^-m (times 1 or i) with no rounding.  Index k*D + l with setting
    k = sum_q s_q 3^(Q-1-q) and outcome l = sum_q b_q 2^(Q-1-q), qubit 0 most significant.
    The arrays are cached per Q and read-only.
    """
    q = int(num_qubits)
    if q < 1:
        raise ValueError("num_qubits must be >= 1")
    t = np.ones((1, 1, 1, 1), dtype=np.complex128)          # [setting, outcome, row, col]
    for _ in range(q):
        k, l, r, c = t.shape
        t = np.einsum("klij,sbmn->ksblimjn", t, _PROJ)
        t = t.reshape(k * 3, 2, l, r * 2, c * 2)            # (k s), b, l, (i m), (j n)
        t = t.transpose(0, 2, 1, 3, 4).reshape(k * 3, l * 2, r * 2, c * 2)   # outcome l*2 + b
    lam = t.reshape(-1, 1 << q, 1 << q)
    re, im = np.ascontiguousarray(lam.real), np.ascontiguousarray(lam.imag)
    re.setflags(write=False)
    im.setflags(write=False)
    return re, im


def ginibre_state(dim: int, rank: int, rng: np.random.Generator) -> np.ndarray:
    """``G G^dagger / Tr`` with ``G`` a ``dim x rank`` standard complex Gaussian matrix."""
    g = rng.standard_normal((dim, rank)) + 1j * rng.standard_normal((dim, rank))
    rho = g @ g.conj().T
    return rho / np.trace(rho).real


def haar_pure_state(dim: int, rng: np.random.Generator) -> np.ndarray:
    """``|psi><psi|`` for a normalised complex Gaussian vector (Haar-random pure state)."""
    psi = rng.standard_normal(dim) + 1j * rng.standard_normal(dim)
    psi /= np.linalg.norm(psi)
    return np.outer(psi, psi.conj())


def depolarise(rho: np.ndarray, weight: float) -> np.ndarray:
    """``(1 - weight) rho + weight I/D``."""
    d = rho.shape[0]
    return (1.0 - weight) * rho + weight * np.eye(d) / d


def sample_counts(truth: np.ndarray, num_qubits: int, shots_per_basis, rng: np.random.Generator) -> np.ndarray:
    """Multinomial outcome counts ``c_kl`` (int32, length ``K*D``) of ``shots_per_basis`` draws per basis.

    Outcome probabilities follow the Born rule ``<phi_kl| truth |phi_kl>``.
    """
    phi = pauli_vectors(num_qubits)
    d = 1 << num_qubits
    k_count = 3 ** num_qubits
    born = np.einsum("ia,ab,ib->i", phi.conj(), truth, phi).real
    born = np.clip(born, 0.0, None).reshape(k_count, d)
    shots = np.broadcast_to(np.asarray(shots_per_basis, dtype=np.int64), (k_count,))
    counts = np.empty((k_count, d), dtype=np.int64)
    for k in range(k_count):
        pk = born[k] / born[k].sum()
        counts[k] = rng.multinomial(int(shots[k]), pk)
    return counts.reshape(-1).astype(np.int32)


@dataclasses.dataclass
class Problem:
    """One tomography problem: inputs for both the oracle and the CUDA sampler."""

    num_qubits: int
    povm_re: np.ndarray
    povm_im: np.ndarray
    counts: np.ndarray
    truth: np.ndarray
    num_chains: int
    num_steps: int
    beta0: float
    seed: int
    name: str = ""
    likelihood: int = 0                  # 0 multinomial (Eq. likelihood), 1 Poisson
    trials: Optional[np.ndarray] = None  # [K] expected trials mu_k per setting (Poisson)

    @property
    def dim(self) -> int:
        return 1 << self.num_qubits

    @property
    def num_povms(self) -> int:
        """Measurement settings K (3^Q for the Pauli problems): the counts hold K D outcomes."""
        return len(self.counts) // self.dim


def make_problem(
    num_qubits: int,
    truth: np.ndarray,
    shots_per_basis,
    num_chains: int,
    num_steps: int,
    beta0: float,
    data_seed: int,
    chain_seed: int,
    name: str = "",
) -> Problem:
    povm_re, povm_im = pauli_povms(num_qubits)
    counts = sample_counts(truth, num_qubits, shots_per_basis, np.random.default_rng(data_seed))
    return Problem(num_qubits, povm_re, povm_im, counts, truth, int(num_chains), int(num_steps),
                   float(beta0), int(chain_seed), name)


def config_problem(index: int, num_chains: Optional[int] = None, num_steps: Optional[int] = None) -> Problem:
    """Benchmark configuration ``index`` (1..4) with optional chain/step overrides.

    1: 1 qubit, Ginibre 2x2 truth, 1000 shots/basis, 64 chains x 2000 steps, beta0 0.1.
    2: 2 qubits, Ginibre truth mixed with I/D at weight 0.1, 1000 shots, 4096 x 5000, beta0 0.05.
    3: 3 qubits, rank-2 Ginibre mixed at 0.05, 2000 shots, 16384 x 2000, beta0 0.1 (the
       paper's initial beta, Algorithm 2, since the configuration names none).
    4: 4 qubits, Haar pure state depolarised at 0.02, 1000 shots, 65536 x 1000, beta0 0.02.
    """
    rng = np.random.default_rng(1000 + index)
    if index == 1:
        q, truth, shots, r, s, b = 1, ginibre_state(2, 2, rng), 1000, 64, 2000, 0.1
    elif index == 2:
        q, truth, shots, r, s, b = 2, depolarise(ginibre_state(4, 4, rng), 0.1), 1000, 4096, 5000, 0.05
    elif index == 3:
        q, truth, shots, r, s, b = 3, depolarise(ginibre_state(8, 2, rng), 0.05), 2000, 16384, 2000, 0.1
    elif index == 4:
        q, truth, shots, r, s, b = 4, depolarise(haar_pure_state(16, rng), 0.02), 1000, 65536, 1000, 0.02
    else:
        raise ValueError("configuration index must be 1..4 (use heterogeneous_batch for 5)")
    if num_chains is not None:
        r = num_chains
    if num_steps is not None:
        s = num_steps
    return make_problem(q, truth, shots, r, s, b, 2000 + index, 3000 + index, name=f"config{index}")


def five_qubit_problem(num_chains: int = 256, num_steps: int = 100, seed: int = 1006) -> Problem:
    """A 5-qubit problem (D = 32, 243 bases x 32 outcomes = 7776 projectors): Ginibre truth of
    rank 3 mixed with I/D at weight 0.05, 1000 shots per basis, beta0 0.05."""
    rng = np.random.default_rng(seed)
    truth = depolarise(ginibre_state(32, 3, rng), 0.05)
    return make_problem(5, truth, 1000, num_chains, num_steps, 0.05, seed + 1000, seed + 2000, name="five_qubits")


def six_qubit_problem(num_chains: int = 64, num_steps: int = 50, seed: int = 1007) -> Problem:
    """A 6-qubit problem (D = 64, 729 bases x 64 outcomes = 46656 projectors): Ginibre truth of
    rank 3 mixed with I/D at weight 0.05, 1000 shots per basis, beta0 0.02.  Its POVM arrays are
    left out (``None``: the built-in Pauli set) -- as dense [K*D, D, D] arrays they would take
    3 GB."""
    rng = np.random.default_rng(seed)
    truth = depolarise(ginibre_state(64, 3, rng), 0.05)
    counts = sample_counts(truth, 6, 1000, np.random.default_rng(seed + 1000))
    return Problem(6, None, None, counts, truth, int(num_chains), int(num_steps), 0.02, seed + 2000,
                   name="six_qubits")


def heterogeneous_batch(num_problems: int = 64, seed: int = 1005, max_qubits: int = 5,
                        chain_scale: float = 1.0) -> List[Problem]:
    """Batch of independent problems of uneven size (64 problems of 1-5 qubits by default).

    Qubits uniform in 1..max_qubits, shots per basis uniform in 500..4000, Ginibre truth of
    rank uniform in 1..D, chain counts log-uniform in [256, 32768] (times ``chain_scale``).
    """
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(num_problems):
        q = int(rng.integers(1, max_qubits + 1))
        d = 1 << q
        rank = int(rng.integers(1, d + 1))
        truth = ginibre_state(d, rank, rng)
        shots = int(rng.integers(500, 4001))
        chains = int(round(math.exp(rng.uniform(math.log(256), math.log(32768))) * chain_scale))
        chains = max(1, chains)
        probs.append(make_problem(q, truth, shots, chains, 1000, 0.05,
                                  int(rng.integers(1 << 31)), int(rng.integers(1 << 31)),
                                  name=f"batch{i}"))
    return probs


# ---- problems with other measurements (any complete POVM; the method only needs Lambda_kl) ----

def _haar_unitary(dim: int, rng: np.random.Generator) -> np.ndarray:
    """A Haar-random unitary: the Q factor of a complex Gaussian matrix, columns rephased so
    that R has a positive diagonal."""
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


# Two-qubit orthonormal bases (columns) whose projectors have dyadic entries (exact in bf16),
# none of them a product of Pauli eigenbases: the Bell basis, the Bell basis with a phase i on
# the second component, and a basis of real vectors with entries +-1/2.
_B = 1.0 / math.sqrt(2.0)
_TWO_QUBIT_BASES = (
    np.array([[_B, _B, 0, 0], [0, 0, _B, _B], [0, 0, _B, -_B], [_B, -_B, 0, 0]], dtype=np.complex128),
    np.array([[_B, _B, 0, 0], [0, 0, _B, _B], [0, 0, 1j * _B, -1j * _B], [1j * _B, -1j * _B, 0, 0]],
             dtype=np.complex128),
    0.5 * np.array([[1, 1, 1, -1], [1, -1, 1, 1], [1, 1, -1, 1], [-1, 1, 1, 1]], dtype=np.complex128),
)


def basis_problem(num_qubits: int, bases: np.ndarray, truth: np.ndarray, shots_per_setting: int, num_chains: int,
                  num_steps: int, beta0: float, data_seed: int, chain_seed: int, name: str = "",
                  dyadic: bool = False) -> Problem:
    """A problem measured in K orthonormal bases: ``bases`` is ``[K, D, D]`` with the outcome
    vectors as columns, ``Lambda_kl = |b_kl><b_kl|`` (each setting sums to the identity).
    Counts are multinomial over the Born probabilities of ``truth``.  With ``dyadic`` the
    projector entries, dyadic rationals up to the rounding of 1/sqrt(2) products, are set to
    those exact values (multiples of 2^-30)."""
    d = 1 << num_qubits
    bases = np.asarray(bases, dtype=np.complex128)
    k_count = bases.shape[0]
    if bases.shape != (k_count, d, d):
        raise ValueError("bases must be [K, D, D]")
    phi = bases.transpose(0, 2, 1).reshape(k_count * d, d)   # row k D + l = column l of basis k
    povm = phi[:, :, None] * phi.conj()[:, None, :]
    if dyadic:
        povm = np.round(povm.real * 2.0 ** 30) / 2.0 ** 30 + 1j * (np.round(povm.imag * 2.0 ** 30) / 2.0 ** 30)
    rng = np.random.default_rng(data_seed)
    born = np.clip(np.einsum("ia,ab,ib->i", phi.conj(), truth, phi).real, 0.0, None).reshape(k_count, d)
    counts = np.stack([rng.multinomial(int(shots_per_setting), b / b.sum()) for b in born]).reshape(-1)
    return Problem(num_qubits, np.ascontiguousarray(povm.real), np.ascontiguousarray(povm.imag),
                   counts.astype(np.int32), truth, int(num_chains), int(num_steps), float(beta0), int(chain_seed),
                   name)


def random_basis_problem(num_qubits: int, num_settings: int, seed: int = 1100, num_chains: int = 256,
                         num_steps: int = 200, shots_per_setting: int = 1000, beta0: float = 0.05) -> Problem:
    """Measurements in ``num_settings`` Haar-random bases of the whole register (entries not
    exact in bf16: the FP32 form), Ginibre truth of rank 2 mixed with I/D at weight 0.05."""
    d = 1 << num_qubits
    rng = np.random.default_rng(seed)
    truth = depolarise(ginibre_state(d, min(2, d), rng), 0.05)
    bases = np.stack([_haar_unitary(d, rng) for _ in range(num_settings)])
    return basis_problem(num_qubits, bases, truth, shots_per_setting, num_chains, num_steps, beta0, seed + 1000,
                         seed + 2000, name=f"random_bases_{num_qubits}q")


def dyadic_basis_problem(num_qubits: int, seed: int = 1200, num_chains: int = 256, num_steps: int = 200,
                         shots_per_setting: int = 1000, beta0: float = 0.05) -> Problem:
    """Entangled (non-Pauli) measurements whose packed projectors are exact in bf16: every
    setting is a Kronecker product of the two-qubit bases above over qubit pairs (0,1), (2,3),
    ..., times the Z or X basis on a last odd qubit -- 3^(Q/2) settings for even Q.  Ginibre
    truth of rank 2 mixed with I/D at weight 0.05."""
    if num_qubits < 2:
        raise ValueError("dyadic entangled bases need at least two qubits")
    d = 1 << num_qubits
    rng = np.random.default_rng(seed)
    truth = depolarise(ginibre_state(d, min(2, d), rng), 0.05)
    factors = [list(_TWO_QUBIT_BASES)] * (num_qubits // 2)
    if num_qubits % 2:
        factors.append([np.eye(2, dtype=np.complex128), np.array([[_B, _B], [_B, -_B]], dtype=np.complex128)])
    bases = [np.ones((1, 1), dtype=np.complex128)]
    for opts in factors:
        bases = [np.kron(b, f) for b in bases for f in opts]
    return basis_problem(num_qubits, np.stack(bases), truth, shots_per_setting, num_chains, num_steps, beta0,
                         seed + 1000, seed + 2000, name=f"dyadic_bases_{num_qubits}q", dyadic=True)


def latent_batch(num: int, num_qubits: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Standard-normal latent vectors ``x`` of length ``4 D^2`` (float64, ``[num, 4D^2]``)."""
    d = 1 << num_qubits
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((num, 4 * d * d))


# ---- a non-multinomial likelihood: Poisson counts through lossy detectors ----------------------

def lossy_pauli_problem(num_qubits: int, num_chains: int = 256, num_steps: int = 200, trials: float = 1000.0,
                        seed: int = 1300, beta0: float = 0.05) -> Problem:
    """Pauli settings measured through detectors of efficiency eta_kl in {8/16, ..., 16/16}: the
    elements are Lambda'_kl = eta_kl Lambda_kl, whose sum over a setting falls short of the
    identity, and the counts are independent Poisson variables of mean mu_k Tr(Lambda'_kl rho),
    mu_k = `trials` (the expected number of trials of every setting).  The efficiencies keep
    every packed entry exact in bf16, so the tensor-core forms apply.  Truth: a rank-2 Ginibre
    state mixed 0.05 with I / D."""
    rng = np.random.default_rng(seed)
    D = 1 << num_qubits
    truth = 0.95 * ginibre_state(D, 2, rng) + 0.05 * np.eye(D) / D
    re, im = pauli_povms(num_qubits)
    eta = rng.integers(8, 17, size=re.shape[0]).astype(np.float64) / 16.0
    re = re * eta[:, None, None]
    im = im * eta[:, None, None]
    p = np.einsum("mab,ba->m", re + 1j * im, truth).real
    K = re.shape[0] // D
    mu = np.full(K, float(trials))
    counts = rng.poisson(np.repeat(mu, D) * np.clip(p, 0.0, None)).astype(np.int32)
    return Problem(num_qubits, re, im, counts, truth, int(num_chains), int(num_steps), float(beta0),
                   int(rng.integers(1 << 31)), f"lossy_pauli_q{num_qubits}", likelihood=1, trials=mu)
