"""The multi-rank path of bench.py on the CPU (gloo, world size 2): every
rank runs its own replica with its own seed (weak scaling, no collective on
the data path) and rank 0 reports the events of all ranks over the slowest
rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ev, N = bench.workload("c1", seed=rank)
    times = [10.0 + 5.0 * rank, 3.0 - rank]  # rank 1 slower on the first, faster on the second
    (t_max, e_max), n_total = bench.reduce_over_ranks(times, ev.n_events, torch.device("cpu"))
    out[rank] = (t_max, e_max, n_total, float(ev.logp[5]), ev.n_events, N)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_report_all_events_over_the_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 15.0 and r0[1] == r1[1] == 3.0  # max over ranks
    assert r0[2] == r1[2] == r0[4] + r1[4]                   # events of both ranks
    assert r0[3] != r1[3]                                     # seeds differ per rank
    assert r0[5] == r1[5] == 500


def test_single_rank_is_identity():
    import torch
    import bench
    assert bench.reduce_over_ranks([2.5, 7.0], 1234, torch.device("cpu")) == ([2.5, 7.0], 1234.0)
