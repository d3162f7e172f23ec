#!/usr/bin/env python3
"""Throughput of the pooled-chain pCN sampler (4-qubit Pauli tomography, 65536 chains).

One "step" is one pass of the whole hot path over every chain: Philox proposal,
Algorithm 1 assembly, projector contraction, log-likelihood, accept/adapt, pooling
and trajectory store (65536 chain-steps).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own 65536 chains with a disjoint global
chain-id range (weak scaling; chains never communicate), timed between barriers and
reported as the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "4-qubit pCN chain-steps/s, mixed vs plain FP32 form, at logL err ≤1e-3"
UNIT = "chain-steps/s"
CONFIG_INDEX = 4
CHAINS = 65536


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons in the background."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            for name, v in zip(names, s[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _l2_flush_buffer():
    import torch
    return torch.empty(256 << 20, dtype=torch.uint8, device="cuda")


def time_form(qst, prob, precision, steps, warmup, world, chain_offset, profile=True):
    """Device-timed steps of one form (inputs resident in HBM)."""
    import torch
    s = qst.Sampler(prob, precision=precision, chain_offsets=[chain_offset])
    s.run_chains(warmup)
    torch.cuda.synchronize()
    s.set_profiling(profile)
    for k in range(4):
        s.kernel_time(k, reset=True)
    launches0 = s.launch_count()
    stream = torch.cuda.current_stream()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _barrier(world)
    torch.cuda.synchronize()
    start.record(stream)
    s.run_chains(steps)
    stop.record(stream)
    torch.cuda.synchronize()
    _barrier(world)
    ms = start.elapsed_time(stop)
    launches = s.launch_count() - launches0
    kernel_ms = {qst.KERNEL_NAMES[k]: s.kernel_time(k) for k in range(4)}
    return s, ms, launches, kernel_ms


def logl_error(qst, oracle, s, prob, nsample=1024):
    """max |log L_gpu - log L_oracle| on the current states of nsample chains."""
    import torch
    st = s.get_state()
    idx = np.linspace(0, prob.num_chains - 1, nsample).astype(np.int64)
    y = st["y"][idx]
    _, _, ll = s.evaluate(torch.from_numpy(y).cuda(), want_rho=False, want_p=False)
    torch.cuda.synchronize()
    _, _, ll_ref = oracle.evaluate(prob, y.astype(np.float64), want_rho=False, want_p=False)
    d = np.abs(ll.cpu().numpy() - ll_ref)
    return float(np.max(d)), float(np.median(d))


def cpu_baseline(oracle, prob, seconds_target=15.0):
    """The FP64 oracle (as it stands) on a bounded sample of the workload."""
    nthreads = oracle.num_threads()
    chains = max(16, 16 * nthreads)
    t0 = time.perf_counter()
    oracle.run(prob, num_chains=chains, num_steps=0)
    init = time.perf_counter() - t0
    steps = 1
    t1 = time.perf_counter()
    oracle.run(prob, num_chains=chains, num_steps=steps)
    one = time.perf_counter() - t1 - init
    per_step = max(one, 1e-6)
    steps = int(max(1, min(50, (seconds_target - init) / per_step)))
    t2 = time.perf_counter()
    oracle.run(prob, num_chains=chains, num_steps=steps)
    total = time.perf_counter() - t2 - init
    return {"value": chains * steps / total, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"config 4 problem, {chains} chains x {steps} steps (FP64 C oracle, OpenMP over chains); "
                      f"init of y0 subtracted"}


def run_reference(args):
    """Reference arm: the FP64 oracle timed on the host cores (rank 0 only)."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_2501_17334_gb300 import workload as W
    prob = W.config_problem(CONFIG_INDEX)
    oracle.lib()
    nthreads = oracle.num_threads()
    chains = max(16, 8 * nthreads)
    t0 = time.perf_counter()
    oracle.run(prob, num_chains=chains, num_steps=0)
    init = time.perf_counter() - t0
    oracle.run(prob, num_chains=chains, num_steps=args.warmup)
    t1 = time.perf_counter()
    oracle.run(prob, num_chains=chains, num_steps=args.steps)
    total = time.perf_counter() - t1 - init
    value = chains * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "config 4: 4-qubit Pauli QST, 1296 projectors, 81000 shots, Haar pure truth "
                                   "depolarised 0.02, beta0 0.02; each step a bounded sample of "
                                   f"{chains} chains (65536 in the GPU arm)", "chains": chains},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": f"{chains} chains x {args.steps} steps of config 4 per timed run"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2501_17334_gb300 import qst, workload as W
    qst.load()
    prob = W.config_problem(CONFIG_INDEX)
    offset = rank * CHAINS
    peaks, peak_src = _peaks()

    # the mixed form if this build has it, else the plain form is the headline
    forms = []
    try:
        qst.Sampler(W.config_problem(CONFIG_INDEX, num_chains=128, num_steps=1), precision=qst.PREC_BF16X3).close()
        forms.append(("bf16x3", qst.PREC_BF16X3))
    except qst.QstError:
        pass
    if not args.no_plain or not forms:
        forms.append(("fp32", qst.PREC_FP32))

    clocks = Clocks(local)
    results = {}
    clocks.start()
    for name, prec in forms:
        s, ms, launches, kms = time_form(qst, prob, prec, args.steps, args.warmup, world, offset)
        ms = _max_over_ranks(ms, world)
        results[name] = {"ms": ms, "launches": launches, "kernels": kms, "sampler": s}
    clocks.stop()
    head_name = forms[0][0]
    head = results[head_name]
    total_chain_steps = CHAINS * args.steps * world
    value = total_chain_steps / (head["ms"] / 1000.0)

    # dominant kernel of the headline form and its roofline
    kms = head["kernels"]
    dom = max(kms, key=lambda k: kms[k][0])
    dom_ms, dom_n = kms[dom]
    avg_s = dom_ms / 1000.0 / max(dom_n, 1)
    D = 16
    if dom == "project" and head_name == "bf16x3":
        flops = 3 * 2.0 * D * D * 1296 * CHAINS
        achieved = flops / avg_s / 1e12
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": dom, "peak_source": f"{peak_src} bf16 sustained"}
    elif dom == "project":
        flops = 2.0 * D * D * 1296 * CHAINS
        achieved = flops / avg_s / 1e12
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": dom, "peak_source": "FP32 FFMA: 152 SMs x 128 lanes x 2 x max SM clock"}
    else:
        # propose: FP32 FFMA work of Algorithm 1 per chain-step
        flops_chain = 8 * D * D * (D - 1) / 2 * 2 + 8 * D ** 3 + 8 * D * D * (D + 2) / 2
        achieved = flops_chain * CHAINS / avg_s / 1e12
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": dom, "peak_source": "FP32 FFMA: 152 SMs x 128 lanes x 2 x max SM clock"}

    # logL error of the headline form on identical states (sampled chains)
    import oracle
    err_max, err_med = logl_error(qst, oracle, head["sampler"], prob)

    # end to end through the C ABI with host buffers: create (H2D of counts and projectors),
    # run, read the posterior mean back (D2H)
    e2e = None
    if rank == 0 or world > 1:
        e2e_steps = args.steps
        for r in results.values():
            r["sampler"].close()
        torch.cuda.synchronize()
        _barrier(world)
        t0 = time.perf_counter()
        s = qst.Sampler(prob, precision=forms[0][1], chain_offsets=[offset])
        s.run_chains(e2e_steps)
        mean, npool = s.posterior_mean()
        t1 = time.perf_counter()
        s.close()
        e2e_s = _max_over_ranks(t1 - t0, world)
        h2d = prob.counts.nbytes + prob.povm_re.nbytes + prob.povm_im.nbytes
        e2e = {"value": CHAINS * e2e_steps * world / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": 2 * 8 * D * D / e2e_steps,
               "includes": "qst_create (validation, packing, upload, y0 init) + run + posterior mean read-back"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+bf16x3" if head_name == "bf16x3" else "f32",
        "data": "synthetic",
        "config": {"workload": "config 4: 4-qubit Pauli QST (D=16, 81 bases x 16 outcomes = 1296 projectors, "
                               "1000 shots/basis), Haar pure truth depolarised 0.02, 65536 chains/GPU, beta0 0.02",
                   "chains_per_gpu": CHAINS, "form": head_name,
                   "l2": "chain state 0.6 GB/GPU > 129 MB L2: every step streams it from HBM"},
        "logl_err": {"max_abs": err_max, "median_abs": err_med, "sample": "1024 chains' current states",
                     "form": head_name},
        "forms": {n: {"value": total_chain_steps / (r["ms"] / 1000.0), "ms_per_step": r["ms"] / args.steps,
                      "kernel_ms_per_step": {k: v[0] / args.steps for k, v in r["kernels"].items()}}
                  for n, r in results.items()},
        "roofline": roof,
        "clocks": clocks.summary(),
        "gpu_launches": head["launches"],
        "e2e": e2e,
    }
    if "fp32" in results and head_name != "fp32":
        line["speedup_vs_plain_fp32"] = results["fp32"]["ms"] / head["ms"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(oracle, prob)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
