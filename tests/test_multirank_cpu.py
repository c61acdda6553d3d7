"""The N > 1 benchmark path on CPU: two gloo ranks run independent tubes (the
CPU oracle stands in for the GPU work) and combine work and time the way
bench.py does -- no collective touches the data path, only the totals."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    import time
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle as orc
    from paper_1011_6330_gb300 import synth
    nz, L = 64, 2.0
    t = orc.Tube(nz, L, 0.4 * L / nz, -np.ones(nz + 1), -1e-3, precision="f32",
                 accumulate="fixed")
    z, u = synth.random_particles(500, L, seed=bench.rank_seed(rank))
    t.add_particles(z, u)
    bench.barrier(world)                                 # as around bench.py's timed region
    t0 = time.perf_counter()
    work = 0
    for _ in range(20):
        work += t.xi.size + t.injection_count()
        t.step()
    secs = time.perf_counter() - t0 + 0.01 * rank       # ranks differ in time
    bench.barrier(world)
    total, slowest = bench.combine_ranks(work, secs)
    out[rank] = (work, secs, total, slowest, t.total_injected, float(t.ez.sum()))
    dist.destroy_process_group()


def test_two_ranks_run_independent_tubes_and_combine_totals():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    (w0, s0, tot0, max0, inj0, ez0), (w1, s1, tot1, max1, inj1, ez1) = out[0], out[1]
    assert tot0 == tot1 == w0 + w1
    assert max0 == max1 == max(s0, s1)
    assert ez0 != ez1                     # different seeds: independent tubes


def test_single_process_combine_is_identity():
    import bench
    assert bench.combine_ranks(123.0, 4.5) == (123.0, 4.5)
    bench.barrier(1)                                     # no process group needed on one GPU
    assert bench.gr_workload_name(10 ** 8) == "gr_tube_P0.5s_B1e12G_Nz65536_1e+08_particles_fix32"
    assert bench.gr_workload_name(10 ** 8, 65536, "f32") == \
        "gr_tube_P0.5s_B1e12G_Nz65536_1e+08_particles_fp32"
    assert len({bench.rank_seed(r) for r in range(8)}) == 8
