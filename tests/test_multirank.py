"""Multi-rank paths on CPU ranks (gloo), no GPU.

* r*-slab decomposition (the multi-GPU form of one problem): slabs of rows with one halo row
  exchanged per Lax-Wendroff iteration reproduce the undecomposed solution bit for bit.
* Replicas (what `bench.py --gpus N` runs): the job time is the slowest rank's and the value
  counts every rank's updates.
"""
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

from tests import slab_ranks  # noqa: E402


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


P = dict(M=1.0, a=0.7, s=-2, m=2, rstar_min=-20.0, rstar_max=40.0, n_r=46, n_theta=12, dt=0.25,
         substeps=4)


@pytest.mark.parametrize("world", [2, 3])
def test_slab_decomposition_matches_single_domain(oracle_mod, tmp_path, world):
    nsub = 9
    mp.start_processes(slab_ranks.slab_rank, args=(world, _port(), P, nsub, str(tmp_path)),
                       nprocs=world, start_method="spawn")
    parts = [np.load(tmp_path / f"slab_{r}.npy") for r in range(world)]
    got = np.concatenate(parts, axis=2)
    o = oracle_mod.Oracle(**P, bits=53)
    o.pulse(8.0, 3.0, 0.8, 0.6, 2)
    o.step(nsub)
    want = o.get_state(1)
    assert got.shape == want.shape
    np.testing.assert_array_equal(got, want)


def test_replica_aggregation(tmp_path):
    t_ms = [100.0, 125.0]
    mp.start_processes(slab_ranks.replica_rank, args=(2, _port(), t_ms, str(tmp_path)), nprocs=2,
                       start_method="spawn")
    for r in range(2):
        t_max, value = np.load(tmp_path / f"rep_{r}.npy")
        assert t_max == 125.0
        assert value == pytest.approx(2 * 1_000_000 / 0.125)
