"""FP64 CPU oracle of the pooled-chain pCN Bayesian QST sampler (arXiv:2501.17334).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark.  The product path never imports it; it
shares no code with the CUDA implementation.

The C core (``qst_oracle.c``) follows Algorithms 1 and 2 and Eq. likelihood; the
numpy helpers here follow Eq. ACFrho / Eq. IACT (mixing diagnostics), Eq. fid
(Uhlmann fidelity), Eq. fro (Frobenius error) and Eq. BME2 (pooled mean).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qst_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP over chains).  Returns the library path."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OracleCfg(ctypes.Structure):
    _fields_ = [
        ("D", ctypes.c_int32), ("KD", ctypes.c_int32),
        ("povm_re", ctypes.c_void_p), ("povm_im", ctypes.c_void_p), ("counts", ctypes.c_void_p),
        ("seed", ctypes.c_uint64), ("chain_begin", ctypes.c_int64), ("num_chains", ctypes.c_int64),
        ("num_steps", ctypes.c_int64), ("beta0", ctypes.c_double), ("adapt_interval", ctypes.c_int32),
        ("acc_lo", ctypes.c_double), ("acc_hi", ctypes.c_double), ("adapt_factor", ctypes.c_double),
        ("beta_max", ctypes.c_double), ("thin", ctypes.c_int32), ("burn_in", ctypes.c_int32),
        ("trace_steps", ctypes.c_int32), ("traj_chains", ctypes.c_int32), ("traj_capacity", ctypes.c_int32),
        ("prior", ctypes.c_int32), ("likelihood", ctypes.c_int32), ("mu", ctypes.c_void_p),
    ]


class OracleOut(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in (
        "pool_re", "pool_im", "num_pooled", "chain_pool_re", "chain_pool_im", "final_y", "final_logl",
        "final_beta", "accepts", "trace_accept", "trace_logl_prop", "trace_log_alpha", "trace_logl_cur",
        "traj_re", "traj_im")]


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        L.oracle_philox4x32_10.argtypes = [P, P, P]
        L.oracle_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_int64, P]
        L.oracle_alpha.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
        L.oracle_alpha.restype = ctypes.c_double
        L.oracle_philox_blocks.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_uint32, ctypes.c_int64, P]
        L.oracle_qr_unitary_split.argtypes = [ctypes.c_int, P, P, P, P, P, P]
        L.oracle_probabilities_split.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, P]
        L.oracle_loglik.argtypes = [ctypes.c_int, P, P]
        L.oracle_loglik.restype = ctypes.c_double
        L.oracle_loglik_poisson.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P]
        L.oracle_loglik_poisson.restype = ctypes.c_double
        L.oracle_evaluate_batch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P, P, P,
                                            ctypes.c_int64, P, P, P, P, P]
        L.oracle_run.argtypes = [ctypes.POINTER(OracleCfg), ctypes.POINTER(OracleOut)]
        L.oracle_run.restype = ctypes.c_int
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------- primitives

def philox(counter, key) -> np.ndarray:
    """One Philox4x32-10 block for a 4-word counter and 2-word key (uint32 array of 4)."""
    c = _c(counter, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox_blocks(seed: int, step: int, chain: int, tag: int, block0: int, nblocks: int) -> np.ndarray:
    """Blocks ``block0..block0+nblocks-1`` of one (step, chain, tag) stream, ``[nblocks, 4]`` uint32."""
    out = np.zeros((nblocks, 4), np.uint32)
    lib().oracle_philox_blocks(seed, step, chain, tag, block0, nblocks, _ptr(out))
    return out


def normals(seed: int, step: int, chain: int, tag: int, n: int) -> np.ndarray:
    out = np.zeros(n, np.float64)
    lib().oracle_normals(seed, step, chain, tag, n, _ptr(out))
    return out


def alpha(seed: int, step: int, chain: int) -> float:
    return lib().oracle_alpha(seed, step, chain)


def qr_unitary(H: np.ndarray):
    """Algorithm 1 steps 4-5 on a complex ``D x D`` matrix: ``(U, diag R before the phase fix)``."""
    D = H.shape[0]
    hr = _c(H.real.T, np.float64)  # column-major
    hi = _c(H.imag.T, np.float64)
    ur = np.zeros((D, D)); ui = np.zeros((D, D)); rr = np.zeros(D); ri = np.zeros(D)
    lib().oracle_qr_unitary_split(D, _ptr(hr), _ptr(hi), _ptr(ur), _ptr(ui), _ptr(rr), _ptr(ri))
    return (ur + 1j * ui).T, rr + 1j * ri


PRIOR_BURES, PRIOR_HS = 0, 1   # Algorithm 1; Hilbert-Schmidt (rho = G G^dag / Tr)
LIK_MULTINOMIAL, LIK_POISSON = 0, 1   # Eq. likelihood; Poisson counts of mean mu_k p_kl


def _likelihood(problem):
    """(likelihood, mu as a contiguous FP64 array or None) of a problem (multinomial by default)."""
    lik = int(getattr(problem, "likelihood", LIK_MULTINOMIAL))
    mu = getattr(problem, "trials", None)
    if lik == LIK_POISSON and mu is None:
        raise ValueError("a Poisson problem needs its expected trials per setting")
    return lik, _c(mu, np.float64)


def evaluate(problem, x: np.ndarray, want_rho=True, want_p=True, prior=PRIOR_BURES):
    """rho(x), p(x) and log L(x) for rows of ``x`` (``[n, 4D^2]``), all FP64."""
    D, KD = problem.dim, problem.num_povms * problem.dim
    x = _c(np.atleast_2d(x), np.float64)
    n = x.shape[0]
    rr = np.zeros((n, D, D)) if want_rho else None
    ri = np.zeros((n, D, D)) if want_rho else None
    p = np.zeros((n, KD)) if want_p else None
    ll = np.zeros(n)
    pr = _c(problem.povm_re, np.float64); pi = _c(problem.povm_im, np.float64)
    cnt = _c(problem.counts, np.int32)
    lik, mu = _likelihood(problem)
    lib().oracle_evaluate_batch(D, int(prior), lik, _ptr(mu), KD, _ptr(pr), _ptr(pi), _ptr(cnt), n, _ptr(x), _ptr(rr),
                                _ptr(ri), _ptr(p), _ptr(ll))
    rho = (rr + 1j * ri) if want_rho else None
    return rho, p, ll


def probabilities(problem, rho: np.ndarray) -> np.ndarray:
    D, KD = problem.dim, problem.num_povms * problem.dim
    rr = _c(rho.real, np.float64); ri = _c(rho.imag, np.float64)
    p = np.zeros(KD)
    pr = _c(problem.povm_re, np.float64); pi = _c(problem.povm_im, np.float64)
    lib().oracle_probabilities_split(D, KD, _ptr(pr), _ptr(pi), _ptr(rr), _ptr(ri), _ptr(p))
    return p


def loglik(counts: np.ndarray, p: np.ndarray) -> float:
    c = _c(counts, np.int32); pp = _c(p, np.float64)
    return lib().oracle_loglik(len(c), _ptr(c), _ptr(pp))


def loglik_poisson(counts: np.ndarray, p: np.ndarray, mu: np.ndarray) -> float:
    """Poisson log-likelihood of counts of mean mu_k p_kl (D = len(counts) / len(mu) outcomes
    per setting), without - log c!."""
    c = _c(counts, np.int32); pp = _c(p, np.float64); m = _c(mu, np.float64)
    return lib().oracle_loglik_poisson(len(c) // len(m), len(c), _ptr(c), _ptr(m), _ptr(pp))


# --------------------------------------------------------------------------- the sampler

DEFAULTS = dict(beta0=0.1, adapt_interval=500, acc_lo=0.2, acc_hi=0.6, adapt_factor=1.1, beta_max=1.0,
                thin=1, burn_in=0)


def run(problem, num_chains=None, num_steps=None, chain_begin=0, trace_steps=0, traj_chains=0,
        traj_capacity=0, want_final=False, want_chain_pool=False, prior=PRIOR_BURES, **overrides):
    """Algorithm 2 on every chain of ``problem`` (or the given counts), pooled as Eq. BME2.

    Returns a dict with the pooled sum and mean, the sample count and any requested traces.
    """
    D, KD = problem.dim, problem.num_povms * problem.dim
    R = problem.num_chains if num_chains is None else int(num_chains)
    S = problem.num_steps if num_steps is None else int(num_steps)
    opts = dict(DEFAULTS)
    opts["beta0"] = problem.beta0
    opts.update(overrides)
    keep = []
    pr = _c(problem.povm_re, np.float64); pi = _c(problem.povm_im, np.float64)
    cnt = _c(problem.counts, np.int32)
    keep += [pr, pi, cnt]
    # no POVM arrays: the Pauli projectors, each entry built from the single-qubit ones
    cfg = OracleCfg(D=D, KD=KD, povm_re=None if pr is None else pr.ctypes.data,
                    povm_im=None if pi is None else pi.ctypes.data, counts=cnt.ctypes.data,
                    seed=int(problem.seed), chain_begin=int(chain_begin), num_chains=R, num_steps=S,
                    beta0=float(opts["beta0"]), adapt_interval=int(opts["adapt_interval"]),
                    acc_lo=float(opts["acc_lo"]), acc_hi=float(opts["acc_hi"]),
                    adapt_factor=float(opts["adapt_factor"]), beta_max=float(opts["beta_max"]),
                    thin=int(opts["thin"]), burn_in=int(opts["burn_in"]), trace_steps=int(trace_steps),
                    traj_chains=int(traj_chains), traj_capacity=int(traj_capacity), prior=int(prior))
    lik, mu = _likelihood(problem)
    keep.append(mu)
    cfg.likelihood = lik
    cfg.mu = None if mu is None else mu.ctypes.data
    res = {}

    def buf(name, shape, dtype):
        a = np.zeros(shape, dtype)
        res[name] = a
        return a.ctypes.data

    out = OracleOut()
    out.pool_re = buf("pool_re", (D, D), np.float64)
    out.pool_im = buf("pool_im", (D, D), np.float64)
    out.num_pooled = buf("num_pooled", 1, np.int64)
    if want_chain_pool:
        out.chain_pool_re = buf("chain_pool_re", (R, D, D), np.float64)
        out.chain_pool_im = buf("chain_pool_im", (R, D, D), np.float64)
    if want_final:
        out.final_y = buf("final_y", (R, 4 * D * D), np.float64)
        out.final_logl = buf("final_logl", R, np.float64)
        out.final_beta = buf("final_beta", R, np.float64)
        out.accepts = buf("accepts", R, np.int64)
    if trace_steps:
        out.trace_accept = buf("trace_accept", (R, trace_steps), np.uint8)
        out.trace_logl_prop = buf("trace_logl_prop", (R, trace_steps), np.float64)
        out.trace_log_alpha = buf("trace_log_alpha", (R, trace_steps), np.float64)
        out.trace_logl_cur = buf("trace_logl_cur", (R, trace_steps), np.float64)
    if traj_chains:
        out.traj_re = buf("traj_re", (traj_chains, traj_capacity, D, D), np.float64)
        out.traj_im = buf("traj_im", (traj_chains, traj_capacity, D, D), np.float64)
    t0 = time.perf_counter()
    rc = lib().oracle_run(ctypes.byref(cfg), ctypes.byref(out))
    res["seconds"] = time.perf_counter() - t0
    if rc != 0:
        raise ValueError(f"oracle_run rejected its configuration (code {rc})")
    n = int(res["num_pooled"][0])
    res["num_pooled"] = n
    res["pool"] = res.pop("pool_re") + 1j * res.pop("pool_im")
    res["mean"] = res["pool"] / n if n > 0 else None
    if want_chain_pool:
        res["chain_pool"] = res.pop("chain_pool_re") + 1j * res.pop("chain_pool_im")
    if traj_chains:
        res["traj"] = res.pop("traj_re") + 1j * res.pop("traj_im")
    res["threads"] = num_threads()
    return res


def num_threads() -> int:
    return int(lib().oracle_num_threads())


# --------------------------------------------------------------------------- diagnostics (numpy)

def acf(traj: np.ndarray, lmax: int = 200) -> np.ndarray:
    """Eq. ACFrho: c[l], l = 0..lmax, of one chain's kept states ``traj`` (``[N, D, D]`` complex).

    c~[l] = sum_{n=1}^{N-lmax} Re Tr[(rho_n - m)^dag (rho_{n+l} - m)], m the chain's own mean
    (Eq. BME1); c = c~ / c~[0].
    """
    traj = np.asarray(traj)
    N = traj.shape[0]
    if N <= lmax:
        raise ValueError("the ACF needs more kept samples than lmax")
    dev = (traj - traj.mean(axis=0)).reshape(N, -1)
    m = N - lmax
    raw = np.array([np.sum((dev[:m].conj() * dev[l:l + m]).real) for l in range(lmax + 1)])
    return raw / raw[0]


def iact(c: np.ndarray) -> float:
    """Eq. IACT: tau = 1 + 2 sum_{l=1}^{lmax} c[l]."""
    return float(1.0 + 2.0 * np.sum(c[1:]))


def _clip_spectrum(w: np.ndarray) -> np.ndarray:
    """Eigenvalues of a PSD matrix with round-off below 1e-13 of the largest set to zero."""
    floor = 1e-13 * max(float(np.max(np.abs(w))), 1e-300)
    return np.where(w > floor, w, 0.0)


def _psd_sqrt(a: np.ndarray) -> np.ndarray:
    w, v = np.linalg.eigh((a + a.conj().T) / 2)
    return (v * np.sqrt(_clip_spectrum(w))) @ v.conj().T


def fidelity(sigma: np.ndarray, rho: np.ndarray) -> float:
    """Eq. fid: (Tr sqrt(sqrt(sigma) rho sqrt(sigma)))^2."""
    s = _psd_sqrt(sigma)
    m = s @ rho @ s
    w = np.linalg.eigvalsh((m + m.conj().T) / 2)
    return float(np.sum(np.sqrt(_clip_spectrum(w))) ** 2)


def frobenius_sq(a: np.ndarray, b: np.ndarray) -> float:
    """Eq. fro: ||a - b||_F^2."""
    return float(np.sum(np.abs(a - b) ** 2))
