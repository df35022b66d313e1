"""Multi-rank state sharding on CPU: two gloo ranks each propagate their shard
of random states with the oracle, average the correlations across ranks, and
must reproduce the single-process average over all states."""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2509_26309_gb300.replicas import shard_states

NSTATES = 5
STEPS = 24
DT = math.pi / 9


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    import tbpm_inputs as ti
    import oracle
    from paper_2509_26309_gb300.replicas import average_over_ranks, shard_states
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    h = ti.graphene_csr(8, 6, onsite=ti.anderson_onsite(96, 1.0, 1))
    acc = torch.zeros(STEPS + 1, dtype=torch.complex128)
    for j in shard_states(NSTATES, rank, world):
        acc += torch.from_numpy(oracle.dos_corr(h, 9.0, ti.random_phase_state(h.n, j), DT, STEPS))
    avg = average_over_ranks(acc, NSTATES)
    if rank == 0:
        np.save(out_path, avg.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_shards_cover_states_once():
    for world in (1, 2, 3, 8):
        got = sorted(j for r in range(world) for j in shard_states(11, r, world))
        assert got == list(range(11))
    with pytest.raises(ValueError):
        shard_states(4, 2, 2)


def test_two_gloo_ranks_average(tmp_path):
    import tbpm_inputs as ti
    import oracle
    out = str(tmp_path / "avg.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    h = ti.graphene_csr(8, 6, onsite=ti.anderson_onsite(96, 1.0, 1))
    ref = sum(oracle.dos_corr(h, 9.0, ti.random_phase_state(h.n, j), DT, STEPS) for j in range(NSTATES))
    ref = ref / NSTATES
    assert np.max(np.abs(got - ref)) < 1e-14
