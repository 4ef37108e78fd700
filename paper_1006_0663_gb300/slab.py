"""r*-slab decomposition of one problem: the halo exchange around the C ABI's slab calls.

The paper decomposes the (r*, theta) grid over processing elements (Sec. 4). Here one problem
is split along r* into slabs (teuk_create_slab); each Lax-Wendroff iteration (Eqs. lw1, lw2)
reaches one row beyond a slab's owned rows, so before every iteration each slab needs one
halo row from each neighbour: the neighbour's edge row of the same level. This module does
that exchange, either between slab handles of this process (device-to-device copies queued
on the handles' stream) or between ranks (point-to-point messages of torch.distributed:
NCCL between GPUs, gloo between host processes). No rank ever reads another's memory
directly: every remote row is first copied into a local buffer.
"""
from __future__ import annotations


def split_rows(n_r: int, parts: int):
    """Owned rows (own_lo, own_hi) of `parts` contiguous slabs covering rows 0 .. n_r - 1."""
    if parts < 1 or parts > n_r:
        raise ValueError("need 1 <= parts <= n_r")
    bounds = [(n_r * k) // parts for k in range(parts + 1)]
    return [(bounds[k], bounds[k + 1] - 1) for k in range(parts)]


def _ptr(x):
    return 0 if x is None else int(x.data_ptr())


class LocalSlabs:
    """Slab handles of one problem in this process, ordered by r*, on one CUDA stream (the
    exchange copies are queued in stream order between the slabs' iterations)."""

    def __init__(self, slabs, torch):
        self.slabs = list(slabs)
        shape = (4, self.slabs[0].words, self.slabs[0].n_theta)
        dev = torch.device("cuda", torch.cuda.current_device())
        # each slab's outgoing edge rows: lo (to the slab below), hi (to the slab above)
        self.lo = [torch.empty(shape, dtype=torch.float64, device=dev) for _ in self.slabs]
        self.hi = [torch.empty(shape, dtype=torch.float64, device=dev) for _ in self.slabs]

    def exchange(self):
        n = len(self.slabs)
        for s, g in enumerate(self.slabs):
            g.get_halo_rows(self.lo[s] if s > 0 else None, self.hi[s] if s < n - 1 else None)
        for s, g in enumerate(self.slabs):
            g.set_halo_rows(self.hi[s - 1] if s > 0 else None, self.lo[s + 1] if s < n - 1 else None)

    def iterate(self, n_iterations: int = 1):
        for _ in range(n_iterations):
            self.exchange()
            for g in self.slabs:
                g.substep(1)


class RankSlab:
    """One slab per rank of a torch.distributed group (rank r holds the r-th slab of r*).

    `slab` is anything with get_halo_rows(lo, hi), set_halo_rows(lo, hi) (buffers or None)
    and substep(1); buffers are tensors of shape (4, words, n_theta) on `device`."""

    def __init__(self, slab, rank: int, world: int, dist, torch, device):
        self.slab, self.rank, self.world, self.dist = slab, rank, world, dist
        shape = (4, slab.words, slab.n_theta)
        mk = lambda: torch.empty(shape, dtype=torch.float64, device=device)  # noqa: E731
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = mk(), mk(), mk(), mk()
        self.below = rank > 0
        self.above = rank < world - 1

    def exchange(self):
        d = self.dist
        self.slab.get_halo_rows(self.send_lo if self.below else None, self.send_hi if self.above else None)
        reqs = []
        if self.below:
            reqs.append(d.isend(self.send_lo, self.rank - 1))
        if self.above:
            reqs.append(d.isend(self.send_hi, self.rank + 1))
        if self.below:
            d.recv(self.recv_lo, self.rank - 1)
        if self.above:
            d.recv(self.recv_hi, self.rank + 1)
        for r in reqs:
            r.wait()
        self.slab.set_halo_rows(self.recv_lo if self.below else None, self.recv_hi if self.above else None)

    def iterate(self, n_iterations: int = 1):
        for _ in range(n_iterations):
            self.exchange()
            self.slab.substep(1)
