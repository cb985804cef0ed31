"""Multi-process (gloo, world_size 2, CPU) checks of the N > 1 logic.

The bench runs one independent replica per rank and reports the slowest rank's time; the
sketch itself is linear in A (Sec. 4, linear updates), so row blocks of A sketched on
different ranks sum to the sketch of the whole matrix (W by a reduction, Y by
concatenation).  Both are checked here with the FP64 oracle on CPU ranks.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle as O
        import workloads as WL
        # slowest rank's time
        out[rank * 4 + 0] = bench.max_over_ranks(10.0 + rank, world)
        # row-partitioned sketch: rank r holds rows [r*m/2, (r+1)*m/2) of A
        m, n, s, l = 40, 30, 5, 11
        A = WL.make_gaussian(m, n, seed=7)
        Om = O.draw_embedding(n, s, O.EMB_GAUSSIAN, O.STREAM_OMEGA, 3)
        Psi = O.draw_embedding(l, m, O.EMB_GAUSSIAN, O.STREAM_PSI, 3)
        r0, r1 = rank * m // world, (rank + 1) * m // world
        Yp = O.qmatmul(A[:, r0:r1], Om)
        Wp = torch.as_tensor(O.qmatmul(Psi[:, :, r0:r1], A[:, r0:r1]))
        dist.all_reduce(Wp)
        ys = [torch.zeros((4, m // world, s), dtype=torch.float64) for _ in range(world)]
        dist.all_gather(ys, torch.as_tensor(Yp))
        Y = torch.cat(ys, dim=1).numpy()
        Yref, Wref = O.sketch(A, Om, Psi)
        out[rank * 4 + 1] = float(np.abs(Y - Yref).max())
        out[rank * 4 + 2] = float(np.abs(Wp.numpy() - Wref).max())
        out[rank * 4 + 3] = 1.0
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    out = torch.zeros(world * 4, dtype=torch.float64).share_memory_()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn",
                       join=True)
    res = out.view(world, 4).numpy()
    assert np.all(res[:, 3] == 1.0)
    assert np.all(res[:, 0] == 11.0)          # both ranks see the max
    assert np.all(res[:, 1] < 1e-12) and np.all(res[:, 2] < 1e-12)
