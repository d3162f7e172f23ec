"""Chain sharding across processes (one per GPU) and the final merge of the pooled sums.

Chains never communicate (Algorithm 2 runs each chain on its own), and the Philox counter of
every random draw holds the chain's global id, so a chain gives the same trajectory on any
rank. A run over R chains on N processes gives each rank one contiguous range of global
chain ids (``chain_range``). The pooled estimate of Eq. BME2 is a sum over chains and kept
steps divided by the number of kept states. It is merged once, at the end, by
``merge_posterior_sum``: every rank's raw FP64 sum (``Sampler.posterior_sum``, the C ABI's
``qst_posterior_sum``) and count are gathered, added on the host in rank order and divided
once. The result is the same on every rank and independent of the reduction schedule.
Nothing is exchanged while the chains run.
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


def packed_to_matrix(packed: np.ndarray, D: int) -> np.ndarray:
    """The Hermitian D x D matrix of a packed vec_h array: Re rho_ii on the diagonal, Re rho_ij
    above it (i < j), Im rho_ij below it (i > j), as include/qst.h lays it out."""
    v = np.asarray(packed, dtype=np.float64).reshape(D, D)
    m = np.zeros((D, D), dtype=np.complex128)
    iu = np.triu_indices(D, 1)
    m[np.diag_indices(D)] = np.diag(v)
    m[iu] = v[iu] - 1j * v.T[iu]          # Im rho_ij = -Im rho_ji, stored at [j, i]
    m[(iu[1], iu[0])] = np.conj(m[iu])
    return m


def merge_posterior_sum(sum_packed: np.ndarray, num_pooled: int, group=None):
    """Merge per-rank pooled sums into the posterior mean over every rank's kept states.

    ``sum_packed`` is this rank's FP64 sum of its kept packed states and ``num_pooled`` their
    count (what ``Sampler.posterior_sum`` returns). The sums and counts of all ranks of the
    default process group (or ``group``) are gathered and added in rank order in FP64, and
    the total is divided once. Returns ``(merged mean as a complex D x D matrix, total
    count)`` on every rank, or ``(None, 0)`` when nothing was kept. A rank with no kept
    states contributes zero. Works with the gloo backend (host tensors) and with NCCL
    (device tensors).
    """
    import torch
    import torch.distributed as dist

    s = np.asarray(sum_packed, dtype=np.float64).ravel()
    d = s.size
    D = int(round(np.sqrt(d)))
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    device = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    local = np.zeros(d + 1, dtype=np.float64)
    if num_pooled > 0:
        local[:d] = s
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
    return packed_to_matrix(total[:d] / n, D), n
