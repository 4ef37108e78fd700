"""Helpers run in spawned processes by tests/test_multirank.py (CPU, gloo backend)."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


class _OracleSlab:
    """The slab interface of the library's handles (get_halo_rows, set_halo_rows, substep) on a
    window of the CPU oracle: rows [wlo, whi] with the owned rows [a, b] inside."""

    def __init__(self, o, a, b, wlo, whi, torch):
        self.o, self.a, self.b, self.wlo, self.whi, self.torch = o, a, b, wlo, whi, torch
        self.words, self.n_theta = 1, o.nth

    def get_halo_rows(self, lo, hi):
        if lo is not None:
            lo.copy_(self.torch.from_numpy(self.o.get_row(self.a - self.wlo)))
        if hi is not None:
            hi.copy_(self.torch.from_numpy(self.o.get_row(self.b - self.wlo)))

    def set_halo_rows(self, lo, hi):
        if lo is not None:
            self.o.set_row(0, lo.numpy())
        if hi is not None:
            self.o.set_row(self.whi - self.wlo, hi.numpy())

    def substep(self, n):
        self.o.step(n)


def slab_rank(rank, world, port, p, nsub, out_dir):
    """r*-slab decomposition of one problem over `world` CPU ranks: rank r owns a contiguous
    range of rows (paper_1006_0663_gb300.slab.split_rows), holds one halo row on each side, and
    before every Lax-Wendroff iteration exchanges edge rows with its neighbours through the
    library's rank driver (slab.RankSlab: point-to-point messages), here on oracle windows."""
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1006_0663_gb300 import slab

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n_r = p["n_r"]
    a, b = slab.split_rows(n_r, world)[rank]                    # owned rows [a, b]
    wlo, whi = max(0, a - 1), min(n_r - 1, b + 1)              # window with halos
    o = oracle.Oracle(**p, row_lo=wlo, row_hi=whi, bits=53)
    o.pulse(8.0, 3.0, 0.8, 0.6, 2)
    run = slab.RankSlab(_OracleSlab(o, a, b, wlo, whi, torch), rank, world, dist, torch, "cpu")
    run.iterate(nsub)
    st = o.get_state(1)
    np.save(os.path.join(out_dir, f"slab_{rank}.npy"), st[:, :, a - wlo:b - wlo + 1])
    dist.barrier()
    dist.destroy_process_group()


def replica_rank(rank, world, port, t_ms, out_dir):
    """The benchmark's replica aggregation on gloo ranks with fake per-rank times."""

    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_max, value = bench.aggregate_ranks(t_ms[rank], 1_000_000, world, dist, torch, "cpu")
    np.save(os.path.join(out_dir, f"rep_{rank}.npy"), np.array([t_max, value]))
    dist.destroy_process_group()
