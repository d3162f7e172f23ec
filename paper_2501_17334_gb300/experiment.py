"""The paper's simulated study on the GPU sampler (Sec. IV), written as CSV.

For Q qubits the ground truth is one density matrix drawn from the Bures distribution
(Algorithm 1 of a standard-normal latent vector, mapped by the CUDA path itself), the data
are all 3^Q Pauli settings with P = 25 2^Q shots each, and every chain keeps N states at
thinning T (N T steps).  One handle per thinning runs every (Q, R) pair as its own
problem; problems with the same data and seed start their chains at global id 0, so the
R-chain problem's chains are the first R chains of every larger one (nested pools).

Outputs, one row per point:
  acf.csv            Q, T, lag, c[lag]                         Eq. ACFrho, chain-averaged (Fig. 2)
  tau.csv            Q, T, tau_mean, tau_max, accept_rate       Eq. IACT
  frob.csv           Q, T, R, N_eff = N R / tau, eps_F^2        Eq. fro against the (T_max, R_max) pool (Fig. 3)
  fidelity.csv       Q, T, R, gpu_seconds, 1 - F                 Eq. fid against the same pool (Fig. 4)

gpu_seconds is the CUDA-event time of the whole handle at that thinning (all Q and R run
concurrently on the GPU); chains of every R take the same time, which is the point of the
method.  The analysis (Frobenius norm, fidelity) runs on the host in FP64.

Usage: python -m paper_2501_17334_gb300.experiment --out DIR [--qubits 1 2 3 4]
       [--log2-thinning 0 2 4 6 8 10 12] [--chains 1 4 16 64 256 1024] [--keep 1024]
"""
from __future__ import annotations

import argparse
import csv
import os
from typing import Dict, List, Sequence

import numpy as np

from . import qst
from . import workload as W


# ---- host analysis (FP64) -----------------------------------------------------------------

def frobenius_sq(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b||_F^2 (Eq. fro)."""
    d = np.asarray(a) - np.asarray(b)
    return float(np.real(np.vdot(d, d)))


def _psd_eigenvalues(w: np.ndarray) -> np.ndarray:
    """Eigenvalues of a PSD matrix with those below 1e-12 of the largest (round-off, whose
    square roots would otherwise add ~1e-9 to a trace) set to zero."""
    return np.where(w > 1e-12 * max(float(np.max(np.abs(w))), 1e-300), w, 0.0)


def _sqrtm_psd(a: np.ndarray) -> np.ndarray:
    w, v = np.linalg.eigh((a + a.conj().T) / 2)
    return (v * np.sqrt(_psd_eigenvalues(w))) @ v.conj().T


def fidelity(sigma: np.ndarray, rho: np.ndarray) -> float:
    """(Tr sqrt(sqrt(sigma) rho sqrt(sigma)))^2 (Eq. fid), both arguments PSD."""
    s = _sqrtm_psd(np.asarray(sigma, dtype=np.complex128))
    m = s @ np.asarray(rho, dtype=np.complex128) @ s
    w = _psd_eigenvalues(np.linalg.eigvalsh((m + m.conj().T) / 2))
    return float(np.sum(np.sqrt(w)) ** 2)


# ---- the simulated data ---------------------------------------------------------------------

def bures_truth(num_qubits: int, seed: int) -> np.ndarray:
    """A density matrix drawn from the Bures distribution: Algorithm 1 applied, on the GPU, to a
    seeded standard-normal latent vector of length 4 D^2."""
    import torch
    D = 1 << num_qubits
    x = np.random.default_rng(seed).standard_normal((1, 4 * D * D)).astype(np.float32)
    re, im = W.pauli_povms(num_qubits)
    probe = W.Problem(num_qubits, re, im, np.zeros(3 ** num_qubits * D, np.int32), None, 1, 1, 0.1, seed)
    s = qst.Sampler(probe, precision=qst.PREC_FP32, diag_chains=0)
    try:
        rho_p, _, _ = s.evaluate(torch.from_numpy(x).cuda(), want_p=False)
        torch.cuda.synchronize()
        packed = rho_p.cpu().numpy().astype(np.float64)[0].reshape(D, D)
    finally:
        s.close()
    # packed layout: Re rho_ii on the diagonal, Re rho_ij above it, Im rho_ij below it
    upper = np.triu(np.ones((D, D), bool), 1)
    re_part = np.where(upper, packed, 0.0) + np.where(upper.T, packed.T, 0.0) + np.diag(np.diag(packed))
    im_up = np.where(upper, -packed.T, 0.0)
    rho = re_part + 1j * (im_up - im_up.T)
    return rho / np.trace(rho).real


def paper_problem(num_qubits: int, num_chains: int, seed: int = 0) -> W.Problem:
    """Sec. IV data for Q qubits: Bures truth, all 3^Q Pauli settings, P = 25 2^Q shots each."""
    truth = bures_truth(num_qubits, 7000 + 10 * seed + num_qubits)
    shots = 25 * (1 << num_qubits)
    return W.make_problem(num_qubits, truth, shots, num_chains, 1, 0.1,
                          8000 + 10 * seed + num_qubits, 9000 + 10 * seed + num_qubits,
                          name=f"sec4_q{num_qubits}")


# ---- one thinning ----------------------------------------------------------------------------

def run_thinning(problems: Dict[int, W.Problem], chains: Sequence[int], thin: int, keep: int,
                 diag_chains: int = 64, precision: int = qst.PREC_BF16X3) -> dict:
    """All (Q, R) pairs at thinning T in one handle: N T steps, pooled means per (Q, R), the
    chain-averaged ACF and tau of the largest R for every Q, and the handle's GPU time."""
    import copy
    import torch
    keys, probs = [], []
    for q, base in problems.items():
        for r in chains:
            p = copy.copy(base)
            p.num_chains = int(r)
            probs.append(p)
            keys.append((q, int(r)))
    cfg = qst.default_config(precision=precision, thin=thin, diag_chains=diag_chains, traj_capacity=keep,
                             acf_lmax=200)
    s = qst.Sampler(probs, cfg=cfg)
    try:
        stream = torch.cuda.current_stream()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        s.run_chains(keep * thin)
        t1.record(stream)
        torch.cuda.synchronize()
        gpu_s = t0.elapsed_time(t1) / 1000.0
        means, diags = {}, {}
        for i, k in enumerate(keys):
            means[k], _ = s.posterior_mean(i)
            if k[1] == max(chains):
                diags[k[0]] = s.diagnostics(i)
    finally:
        s.close()
    return {"means": means, "diags": diags, "gpu_seconds": gpu_s}


def sweep(qubits: Sequence[int], log2_thinning: Sequence[int], chains: Sequence[int], keep: int, out_dir: str,
          precision: int = qst.PREC_BF16X3) -> dict:
    """The study of Sec. IV; returns the rows it writes."""
    if keep <= 200:
        raise ValueError("keep (N) must exceed l_max = 200 for Eq. ACFrho")
    os.makedirs(out_dir, exist_ok=True)
    problems = {q: paper_problem(q, max(chains)) for q in qubits}
    runs = {}
    for lt in sorted(log2_thinning):
        runs[1 << lt] = run_thinning(problems, chains, 1 << lt, keep, precision=precision)
    t_max, r_max = max(runs), max(chains)
    rows = {"acf": [], "tau": [], "frob": [], "fidelity": []}
    for q in qubits:
        ref = runs[t_max]["means"][(q, r_max)]
        for t, run in sorted(runs.items()):
            dg = run["diags"][q]
            tau = dg["tau_mean"] if dg["diag_chains"] > 0 else float("nan")
            if dg["acf"] is not None:
                rows["acf"] += [(q, t, l, float(c)) for l, c in enumerate(dg["acf"])]
            rows["tau"].append((q, t, tau, dg["tau_max"], dg["accept_rate"]))
            for r in chains:
                m = run["means"][(q, r)]
                # N_eff = N R / tau (Sec. IV); the unwindowed sum of Eq. IACT can fall to or below
                # zero for short chains, where N_eff is undefined
                n_eff = keep * r / tau if tau > 0 else float("nan")
                rows["frob"].append((q, t, r, n_eff, frobenius_sq(m, ref)))
                rows["fidelity"].append((q, t, r, run["gpu_seconds"], 1.0 - fidelity(ref, m)))
    heads = {"acf": ("Q", "T", "lag", "acf"), "tau": ("Q", "T", "tau_mean", "tau_max", "accept_rate"),
             "frob": ("Q", "T", "R", "N_eff", "eps_F2"), "fidelity": ("Q", "T", "R", "gpu_seconds", "one_minus_F")}
    for name, rs in rows.items():
        with open(os.path.join(out_dir, f"{name}.csv"), "w", newline="") as f:
            w = csv.writer(f)
            w.writerow(heads[name])
            w.writerows(rs)
    return rows


def main(argv: List[str] = None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--qubits", type=int, nargs="+", default=[1, 2, 3, 4])
    ap.add_argument("--log2-thinning", type=int, nargs="+", default=[0, 2, 4, 6, 8, 10, 12])
    ap.add_argument("--chains", type=int, nargs="+", default=[1, 4, 16, 64, 256, 1024])
    ap.add_argument("--keep", type=int, default=1024, help="N, kept states per chain")
    args = ap.parse_args(argv)
    qst.load()
    sweep(args.qubits, args.log2_thinning, args.chains, args.keep, args.out)


if __name__ == "__main__":
    main()
