"""Python binding of the C ABI in include/qst.h (argument marshalling only).

Every step of the sampler runs in libqst.so's CUDA kernels; this module converts
arguments, allocates the device workspace with PyTorch and passes raw pointers and
the current CUDA stream.  It never computes anything itself and there is no CPU
fallback: if the library cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import _build

QST_OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of memory", 4: "timeout",
                5: "numeric", 6: "invalid state", 7: "unsupported"}
PREC_FP32 = 0
PREC_BF16X3 = 1
PREC_TF32 = 2
PREC_TF32X2 = 3
PREC_PAULI = 4   # structured FP32 form, Pauli POVMs only
PREC_AUTO = 5    # per problem the faster of the forms that apply (timed at creation)
PRIOR_BURES = 0  # Algorithm 1
PRIOR_HS = 1     # Hilbert-Schmidt: rho = G G^dag / Tr
LIKELIHOOD_MULTINOMIAL = 0  # Eq. likelihood
LIKELIHOOD_POISSON = 1      # Poisson counts of mean mu_k p_kl (Problem.trials = mu)
KERNEL_PROPOSE, KERNEL_PROJECT, KERNEL_ACCEPT, KERNEL_DIAG = range(4)
KERNEL_NAMES = {KERNEL_PROPOSE: "propose", KERNEL_PROJECT: "project", KERNEL_ACCEPT: "accept", KERNEL_DIAG: "diag"}


class QstError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ProblemDesc(ctypes.Structure):
    _fields_ = [("num_qubits", ctypes.c_int32), ("num_povms", ctypes.c_int32), ("counts", ctypes.c_void_p),
                ("povm_re", ctypes.c_void_p), ("povm_im", ctypes.c_void_p), ("num_chains", ctypes.c_int64),
                ("chain_offset", ctypes.c_int64), ("seed", ctypes.c_uint64), ("beta0", ctypes.c_double),
                ("likelihood", ctypes.c_int32), ("trials", ctypes.c_void_p)]


class SamplerCfg(ctypes.Structure):
    _fields_ = [("beta0", ctypes.c_double), ("adapt_interval", ctypes.c_int32), ("acc_lo", ctypes.c_double),
                ("acc_hi", ctypes.c_double), ("adapt_factor", ctypes.c_double), ("beta_max", ctypes.c_double),
                ("thin", ctypes.c_int32), ("burn_in", ctypes.c_int32), ("diag_chains", ctypes.c_int32),
                ("traj_capacity", ctypes.c_int32), ("acf_lmax", ctypes.c_int32), ("trace_steps", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("qr_passes", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("prior", ctypes.c_int32), ("propose_threads", ctypes.c_int32)]


class Diag(ctypes.Structure):
    _fields_ = [("steps_done", ctypes.c_int64), ("num_pooled", ctypes.c_int64), ("num_kept", ctypes.c_int64),
                ("accept_rate", ctypes.c_double), ("beta_min", ctypes.c_double), ("beta_mean", ctypes.c_double),
                ("beta_max", ctypes.c_double), ("num_nonfinite", ctypes.c_int64), ("diag_chains", ctypes.c_int32),
                ("acf_lmax", ctypes.c_int32), ("tau_mean", ctypes.c_double), ("tau_max", ctypes.c_double),
                ("n_eff", ctypes.c_double), ("device_status", ctypes.c_uint32), ("column_groups", ctypes.c_uint32),
                ("propose_chains_per_cta", ctypes.c_uint32), ("accept_chains_per_cta", ctypes.c_uint32),
                ("projection_form", ctypes.c_int32), ("qr_passes", ctypes.c_int32)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "reserved"}


_lib = None

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "qst_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "qst_last_error": (ctypes.c_char_p, []),
    "qst_default_config": (None, [ctypes.POINTER(SamplerCfg)]),
    "qst_workspace_size": (ctypes.c_int, [ctypes.POINTER(ProblemDesc), ctypes.c_int32, ctypes.POINTER(SamplerCfg),
                                          ctypes.POINTER(ctypes.c_size_t)]),
    "qst_create": (ctypes.c_int, [ctypes.POINTER(ProblemDesc), ctypes.c_int32, ctypes.POINTER(SamplerCfg), _P,
                                  ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    "qst_run_chains": (ctypes.c_int, [_P, ctypes.c_int64]),
    "qst_posterior_mean": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.POINTER(ctypes.c_int64)]),
    "qst_posterior_sum": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_int64)]),
    "qst_diagnostics": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(Diag), _P, _P]),
    "qst_synchronize": (ctypes.c_int, [_P]),
    "qst_destroy": (None, [_P]),
    "qst_get_state": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P]),
    "qst_get_trace": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "qst_checkpoint_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "qst_checkpoint": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "qst_restore": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "qst_evaluate": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, _P, _P]),
    "qst_set_profiling": (ctypes.c_int, [_P, ctypes.c_int32]),
    "qst_kernel_time": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int64)]),
    "qst_launch_count": (ctypes.c_int64, [_P]),
    "qst_philox_blocks": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_int64, ctypes.c_uint32, ctypes.c_int32, _P, _P]),
    "qst_pack_projectors": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
    "qst_inject_nan": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64]),
    "qst_probe_wait_timeout": (ctypes.c_int, [_P, ctypes.c_int32]),
    "qst_pauli_povms": (ctypes.c_int, [ctypes.c_int32, _P, _P]),
    "qst_loglik_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, _P, _P, ctypes.c_int64, _P, _P]),
}

NOALLOC_MAX_ROWS = 4096


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libqst.so (building it if it is missing or stale).  Raises if that fails."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libqst.so is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int):
    if status != QST_OK:
        raise QstError(status, load().qst_last_error().decode())


def default_config(**overrides) -> SamplerCfg:
    cfg = SamplerCfg()
    load().qst_default_config(ctypes.byref(cfg))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class _Descs:
    """Keeps host arrays alive while qst_create reads them."""

    def __init__(self, problems, chain_offsets=None):
        self.arrays = []
        self.descs = (ProblemDesc * len(problems))()
        for i, p in enumerate(problems):
            counts = np.ascontiguousarray(p.counts, dtype=np.int32)
            self.arrays.append(counts)
            d = self.descs[i]
            d.num_qubits = p.num_qubits
            d.num_povms = p.num_povms
            d.counts = counts.ctypes.data
            if p.povm_re is None and p.povm_im is None:   # the built-in Pauli POVMs
                d.povm_re = None
                d.povm_im = None
            else:
                re = np.ascontiguousarray(p.povm_re, dtype=np.float64)
                im = np.ascontiguousarray(p.povm_im, dtype=np.float64)
                self.arrays += [re, im]
                d.povm_re = re.ctypes.data
                d.povm_im = im.ctypes.data
            d.num_chains = p.num_chains
            d.chain_offset = 0 if chain_offsets is None else int(chain_offsets[i])
            d.seed = p.seed
            d.beta0 = float(getattr(p, "beta0", 0.0) or 0.0)
            d.likelihood = int(getattr(p, "likelihood", LIKELIHOOD_MULTINOMIAL))
            trials = getattr(p, "trials", None)
            if trials is None:
                d.trials = None
            else:
                t = np.ascontiguousarray(trials, dtype=np.float64)
                self.arrays.append(t)
                d.trials = t.ctypes.data


def workspace_size(problems: Sequence, cfg: SamplerCfg, chain_offsets=None) -> int:
    descs = _Descs(problems, chain_offsets)
    n = ctypes.c_size_t()
    _check(load().qst_workspace_size(descs.descs, len(problems), ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


class Sampler:
    """A handle over one or more problems (objects with the fields of ``workload.Problem``).

    The workspace is a torch uint8 CUDA tensor owned by this object; the stream is
    torch's current stream at creation (or ``stream``).
    """

    def __init__(self, problems, cfg: Optional[SamplerCfg] = None, stream=None, chain_offsets=None,
                 workspace=None, **cfg_overrides):
        import torch
        if not isinstance(problems, (list, tuple)):
            problems = [problems]
        self.problems = list(problems)
        self.cfg = cfg if cfg is not None else default_config(**cfg_overrides)
        if cfg is not None:
            for k, v in cfg_overrides.items():
                setattr(self.cfg, k, v)
        self.lib = load()
        descs = _Descs(self.problems, chain_offsets)
        n = ctypes.c_size_t()
        _check(self.lib.qst_workspace_size(descs.descs, len(self.problems), ctypes.byref(self.cfg), ctypes.byref(n)))
        self.workspace_bytes = n.value
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        if workspace is None:
            workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device="cuda")
        self.workspace = workspace
        base = workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        h = ctypes.c_void_p()
        _check(self.lib.qst_create(descs.descs, len(self.problems), ctypes.byref(self.cfg), ctypes.c_void_p(aligned),
                                   ctypes.c_size_t(self.workspace_bytes), _stream_ptr(self.stream), ctypes.byref(h)))
        self.handle = h

    # -- lifecycle
    def close(self):
        if getattr(self, "handle", None):
            self.lib.qst_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the ABI, same names
    def run_chains(self, num_steps: int):
        _check(self.lib.qst_run_chains(self.handle, int(num_steps)))

    def posterior_mean(self, problem: int = 0):
        D = self.problems[problem].dim
        re = np.zeros((D, D))
        im = np.zeros((D, D))
        n = ctypes.c_int64()
        _check(self.lib.qst_posterior_mean(self.handle, problem, re.ctypes.data, im.ctypes.data, ctypes.byref(n)))
        return re + 1j * im, n.value

    def posterior_sum(self, problem: int = 0):
        """qst_posterior_sum: the FP64 sum of the kept packed states ([D*D], packed layout) and
        their count."""
        D = self.problems[problem].dim
        out = np.zeros(D * D)
        n = ctypes.c_int64()
        _check(self.lib.qst_posterior_sum(self.handle, problem, out.ctypes.data, ctypes.byref(n)))
        return out, n.value

    def diagnostics(self, problem: int = 0):
        d = Diag()
        lmax = self.cfg.acf_lmax
        acf = np.zeros(lmax + 1)
        ndiag = min(self.cfg.diag_chains, self.problems[problem].num_chains)
        tau = np.zeros(max(ndiag, 1))
        _check(self.lib.qst_diagnostics(self.handle, problem, ctypes.byref(d), acf.ctypes.data, tau.ctypes.data))
        out = d.as_dict()
        out["acf"] = acf if d.diag_chains > 0 else None
        out["tau"] = tau[:ndiag] if d.diag_chains > 0 else None
        return out

    def synchronize(self):
        _check(self.lib.qst_synchronize(self.handle))

    def get_state(self, problem: int = 0):
        p = self.problems[problem]
        R, nx = p.num_chains, 4 * p.dim * p.dim
        y = np.zeros((R, nx), np.float32)
        logl = np.zeros(R)
        beta = np.zeros(R)
        acc = np.zeros(R, np.int64)
        _check(self.lib.qst_get_state(self.handle, problem, y.ctypes.data, logl.ctypes.data, beta.ctypes.data,
                                      acc.ctypes.data))
        return {"y": y, "logl": logl, "beta": beta, "accepts": acc}

    def get_trace(self, problem: int = 0):
        R, T = self.problems[problem].num_chains, self.cfg.trace_steps
        acc = np.zeros((T, R), np.uint8)
        ll = np.zeros((T, R))
        _check(self.lib.qst_get_trace(self.handle, problem, acc.ctypes.data, ll.ctypes.data))
        return acc, ll

    def checkpoint(self) -> bytes:
        n = ctypes.c_size_t()
        _check(self.lib.qst_checkpoint_size(self.handle, ctypes.byref(n)))
        buf = np.zeros(n.value, np.uint8)
        _check(self.lib.qst_checkpoint(self.handle, buf.ctypes.data, n.value))
        return buf

    def restore(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(self.lib.qst_restore(self.handle, buf.ctypes.data, buf.size))

    def evaluate(self, x, problem: int = 0, want_rho=True, want_p=True):
        """rho (packed), p and log L for latent rows x (torch CUDA float32 [n, 4D^2])."""
        import torch
        p = self.problems[problem]
        n = x.shape[0]
        x = x.contiguous().to(torch.float32)
        rho = torch.empty((n, p.dim * p.dim), dtype=torch.float32, device=x.device) if want_rho else None
        pp = torch.empty((n, p.num_povms * p.dim), dtype=torch.float32, device=x.device) if want_p else None
        ll = torch.empty(n, dtype=torch.float64, device=x.device)
        _check(self.lib.qst_evaluate(self.handle, problem, _ptr(x), n, _ptr(rho), _ptr(pp), _ptr(ll)))
        return rho, pp, ll

    def set_profiling(self, enabled: bool):
        _check(self.lib.qst_set_profiling(self.handle, 1 if enabled else 0))

    def kernel_time(self, kind: int, reset: bool = False):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(self.lib.qst_kernel_time(self.handle, kind, 1 if reset else 0, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def launch_count(self) -> int:
        return int(self.lib.qst_launch_count(self.handle))

    def inject_nan(self, chain: int, problem: int = 0):
        _check(self.lib.qst_inject_nan(self.handle, problem, chain))

    def probe_wait_timeout(self, wait_ms: int = 50):
        """Failure-path probe: a bounded device wait that runs out (raises QstError with
        status QST_ERR_TIMEOUT); the handle stays usable afterwards."""
        _check(self.lib.qst_probe_wait_timeout(self.handle, int(wait_ms)))


# ---- free functions with the ABI's names

def philox_blocks(seed, step, tag, chain0, nchains, block0, nblocks, stream=None):
    import torch
    out = torch.empty((nchains, nblocks, 4), dtype=torch.int32, device="cuda")
    _check(load().qst_philox_blocks(seed, step, tag, chain0, nchains, block0, nblocks, out.data_ptr(),
                                    _stream_ptr(stream)))
    return out


def loglik_noalloc(num_qubits: int, num_povms: int, P, counts, x, logl, stream=None):
    """qst_loglik_noalloc: log L of the rows of ``x`` into ``logl`` without any device allocation
    by the library (P, x, logl: torch CUDA tensors owned by the caller; counts: host int32)."""
    c = np.ascontiguousarray(counts, dtype=np.int32)
    _check(load().qst_loglik_noalloc(num_qubits, num_povms, _ptr(P), c.ctypes.data, _ptr(x), int(x.shape[0]),
                                     _ptr(logl), _stream_ptr(stream)))


def pauli_povms(num_qubits: int):
    """The library's built-in Pauli POVMs (what NULL POVM arrays select): real and imaginary
    [3^Q 2^Q, 2^Q, 2^Q] float64 arrays."""
    D = 1 << num_qubits
    re = np.empty((3 ** num_qubits * D, D, D))
    im = np.empty_like(re)
    _check(load().qst_pauli_povms(num_qubits, re.ctypes.data, im.ctypes.data))
    return re, im


def pack_projectors(num_qubits: int, povm_re: np.ndarray, povm_im: np.ndarray) -> np.ndarray:
    D = 1 << num_qubits
    re = np.ascontiguousarray(povm_re, dtype=np.float64)
    im = np.ascontiguousarray(povm_im, dtype=np.float64)
    KD = re.shape[0]
    out = np.zeros((D * D, KD), np.float32)
    _check(load().qst_pack_projectors(num_qubits, KD // D, re.ctypes.data, im.ctypes.data, out.ctypes.data))
    return out

