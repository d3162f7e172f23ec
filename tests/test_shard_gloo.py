"""Multi-process path on the CPU: chain ranges per rank and the final merge of Eq. BME2.

Two gloo ranks each run their own contiguous range of global chain ids (the oracle
stands in for the GPU sampler, which computes the same chains) and merge their raw FP64
pooled sums with ``shard.merge_posterior_sum``.  The merged mean must equal a single run
over all chains up to FP64 summation order, and every rank must hold the same result.
"""
import os
import socket
import sys

import numpy as np
import pytest

from paper_2501_17334_gb300 import shard
from paper_2501_17334_gb300 import workload as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("num_chains", [0, 1, 7, 64, 65536, 65537])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_chain_ranges_partition_the_chain_ids(num_chains, world):
    nxt = 0
    sizes = []
    for r in range(world):
        b, n = shard.chain_range(r, world, num_chains)
        assert b == nxt
        nxt = b + n
        sizes.append(n)
    assert nxt == num_chains
    assert max(sizes) - min(sizes) <= 1


def test_chain_range_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard.chain_range(2, 2, 10)
    with pytest.raises(ValueError):
        shard.chain_range(0, 0, 10)


@pytest.mark.parametrize("D", [1, 2, 4, 16])
def test_packed_to_matrix_inverts_the_packed_layout(D):
    from tests._helpers import pack_rho
    rng = np.random.default_rng(D)
    g = rng.normal(size=(D, D)) + 1j * rng.normal(size=(D, D))
    rho = g @ g.conj().T
    assert np.array_equal(shard.packed_to_matrix(pack_rho(rho), D), rho - 1j * np.diag(np.diag(rho).imag))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, num_chains, num_steps, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    from paper_2501_17334_gb300 import shard as S, workload as WL
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = WL.config_problem(1, num_chains=num_chains, num_steps=num_steps)
        begin, count = S.chain_range(rank, world, num_chains)
        res = oracle.run(prob, num_chains=count, num_steps=num_steps, chain_begin=begin)
        from tests._helpers import pack_rho
        merged, n = S.merge_posterior_sum(pack_rho(res["pool"]), res["num_pooled"])
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.concatenate([merged.ravel(), [n]]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,num_chains", [(2, 64), (2, 33), (3, 20)])
def test_gloo_ranks_merge_to_the_single_run(oracle_mod, tmp_path, world, num_chains):
    import torch.multiprocessing as mp
    num_steps = 150
    mp.start_processes(_rank_main, args=(world, _free_port(), num_chains, num_steps, str(tmp_path)),
                       nprocs=world, join=True, start_method="spawn")
    prob = W.config_problem(1, num_chains=num_chains, num_steps=num_steps)
    full = oracle_mod.run(prob, num_chains=num_chains, num_steps=num_steps)
    got = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    for g in got[1:]:
        assert np.array_equal(g, got[0])           # every rank holds the same merge
    n = int(got[0][-1].real)
    assert n == full["num_pooled"] == num_chains * num_steps
    merged = got[0][:-1].reshape(2, 2)
    assert np.abs(merged - full["mean"]).max() < 1e-13
