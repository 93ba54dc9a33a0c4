"""The bench's path for N > 1 ranks, on CPU with the gloo backend (world size
2): every rank runs an independent replica of the workload with its own
particle draw (weak scaling, no data-path collective), and the job's time is
the slowest rank's."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + 0.5 * rank, dist, device="cpu")
    w = bench.make_workload("laser_foil_2d", rank, sample=8)
    e = w.species[0]
    np.save(os.path.join(out, f"rank{rank}.npy"), np.array([t, e.n, e.x[0], e.ux[0]]))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_time_is_the_slowest_rank_and_draws_differ(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"rank{i}.npy") for i in range(world)]
    assert r[0][0] == r[1][0] == 1.5  # both ranks see the slowest time
    assert r[0][1] == r[1][1]  # the same workload shape on every rank
    assert r[0][2] != r[1][2] and r[0][3] != r[1][3]  # independent particle draws


def test_single_rank_time_is_its_own():
    assert bench.max_over_ranks(2.5, None) == 2.5
