"""Helpers run in spawned processes by tests/test_multirank.py (CPU, gloo backend)."""
import os

import numpy as np


def slab_rank(rank, world, port, p, nsub, out_dir):
    """r*-slab decomposition of one problem over `world` CPU ranks: rank r owns a contiguous
    range of rows, holds one halo row on each side, and before every Lax-Wendroff iteration
    receives the neighbours' edge rows (level n) by point-to-point messages."""
    import torch
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n_r = p["n_r"]
    bounds = np.linspace(0, n_r, world + 1).astype(int)
    a, b = int(bounds[rank]), int(bounds[rank + 1]) - 1        # owned rows [a, b]
    wlo, whi = max(0, a - 1), min(n_r - 1, b + 1)              # window with halos
    o = oracle.Oracle(**p, row_lo=wlo, row_hi=whi, bits=53)
    o.pulse(8.0, 3.0, 0.8, 0.6, 2)
    for _ in range(nsub):
        st = o.get_state(1)                                    # [4, 1, rows, nth]
        reqs = []
        if rank > 0:      # my first owned row -> left neighbour's right halo
            reqs.append(dist.isend(torch.from_numpy(st[:, :, a - wlo].copy()), rank - 1))
        if rank < world - 1:
            reqs.append(dist.isend(torch.from_numpy(st[:, :, b - wlo].copy()), rank + 1))
        if rank > 0:
            left = torch.empty((4, 1, p["n_theta"]), dtype=torch.float64)
            dist.recv(left, rank - 1)
            o.set_row(0, left.numpy())
        if rank < world - 1:
            right = torch.empty((4, 1, p["n_theta"]), dtype=torch.float64)
            dist.recv(right, rank + 1)
            o.set_row(whi - wlo, right.numpy())
        for r in reqs:
            r.wait()
        o.step(1)
    st = o.get_state(1)
    np.save(os.path.join(out_dir, f"slab_{rank}.npy"), st[:, :, a - wlo:b - wlo + 1])
    dist.barrier()
    dist.destroy_process_group()


def replica_rank(rank, world, port, t_ms, out_dir):
    """The benchmark's replica aggregation on gloo ranks with fake per-rank times."""
    import sys

    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_max, value = bench.aggregate_ranks(t_ms[rank], 1_000_000, world, dist, torch, "cpu")
    np.save(os.path.join(out_dir, f"rep_{rank}.npy"), np.array([t_max, value]))
    dist.destroy_process_group()
