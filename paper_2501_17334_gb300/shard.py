"""Chain sharding across processes (one per GPU) and the final merge of the pooled sums.

Chains never communicate (Algorithm 2 runs each chain on its own), and the Philox counter of
every random draw holds the chain's global id, so a chain gives the same trajectory on any
rank. A run over R chains on N processes gives each rank one contiguous range of global
chain ids (``chain_range``). The pooled estimate of Eq. BME2 is a sum over chains and kept
steps divided by the number of kept states. It is merged once, at the end, by
``merge_posterior_mean``: every rank's FP64 sum and count are gathered and added on the host
in rank order. The result is the same on every rank and independent of the reduction
schedule. Nothing is exchanged while the chains run.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np


def chain_range(rank: int, world: int, num_chains: int) -> Tuple[int, int]:
    """(first global chain id, chain count) of ``rank`` when ``num_chains`` chains are split
    over ``world`` ranks: contiguous ranges, sizes differing by at most one, in rank order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of size {world}")
    if num_chains < 0:
        raise ValueError("num_chains must be >= 0")
    base, extra = divmod(num_chains, world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def merge_posterior_mean(mean: np.ndarray, num_pooled: int, group=None):
    """Merge per-rank posterior means into the mean over every rank's kept states.

    ``mean`` is this rank's complex D x D mean of ``num_pooled`` kept states (what
    ``Sampler.posterior_mean`` returns). The sums mean * n are gathered from all ranks of
    the default process group (or ``group``) and added in rank order in FP64. Returns
    ``(merged mean, total count)`` on every rank. A rank with no kept states contributes
    zero. Works with the gloo backend (host tensors) and with NCCL (device tensors).
    """
    import torch
    import torch.distributed as dist

    mean = np.asarray(mean, dtype=np.complex128)
    D = mean.shape[0]
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    device = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    local = np.zeros(2 * D * D + 1, dtype=np.float64)
    if num_pooled > 0:
        s = mean * float(num_pooled)
        local[:D * D] = s.real.ravel()
        local[D * D:2 * D * D] = s.imag.ravel()
    local[-1] = float(num_pooled)
    send = torch.from_numpy(local).to(device)
    parts = [torch.empty_like(send) for _ in range(world)]
    dist.all_gather(parts, send, group=group)
    total = np.zeros_like(local)
    for p in parts:                      # fixed rank order: deterministic
        total += p.cpu().numpy()
    n = int(round(total[-1]))
    if n == 0:
        return None, 0
    merged = (total[:D * D] + 1j * total[D * D:2 * D * D]).reshape(D, D) / n
    return merged, n
