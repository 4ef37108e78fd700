"""r*-slab handles (teuk_create_slab) with one halo row exchanged per iteration.

Slabs of one problem on one GPU, exchanging their edge rows device to device through the
C ABI's halo calls (paper_1006_0663_gb300.slab.LocalSlabs), reproduce the whole-grid handle
bit for bit on their owned rows, and the 256-bit oracle within the parity tolerances. The
multi-GPU form runs the same calls with torch.distributed messages between ranks (RankSlab,
driven on CPU ranks in tests/test_multirank.py)."""
import ctypes

import numpy as np
import pytest

from paper_1006_0663_gb300 import slab, teuk, workloads

pytestmark = pytest.mark.gpu

TOL = {1: 1e-12, 2: 1e-26, 4: 1e-55}
P = dict(M=1.0, a=0.9, s=-2, m=2, rstar_min=-30.0, rstar_max=50.0, n_r=61, n_theta=24, dt=0.0,
         substeps=3, theta_order=10, parity=0)


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_split_rows():
    parts = slab.split_rows(61, 3)
    assert parts[0][0] == 0 and parts[-1][1] == 60
    assert all(b[0] == a[1] + 1 for a, b in zip(parts, parts[1:]))


@pytest.mark.parametrize("W,engine", [(1, 0), (2, 0), (2, 1), (4, 0), (4, 1)])
@pytest.mark.parametrize("parts", [2, 3])
def test_slabs_match_whole_grid_and_oracle(oracle_mod, W, engine, parts):
    torch = _torch()
    nit = 7
    whole = teuk.Teuk(precision=W, **P)
    slabs = [teuk.Teuk(precision=W, own_rows=rows, **P) for rows in slab.split_rows(P["n_r"], parts)]
    for g in [whole] + slabs:
        if engine:
            g.set_engine(engine)
        g.set_initial_pulse(8.0, 4.0, 0.8, 0.6, 2)
    whole.substep(nit)
    run = slab.LocalSlabs(slabs, torch)
    run.iterate(nit)
    want = whole.get_state()
    got = np.concatenate([g.get_state()[:, :, g.own_lo - g.row0:g.own_hi - g.row0 + 1] for g in slabs],
                         axis=2)
    np.testing.assert_array_equal(got, want)
    o = oracle_mod.Oracle(M=P["M"], a=P["a"], s=P["s"], m=P["m"], rstar_min=P["rstar_min"],
                          rstar_max=P["rstar_max"], n_r=P["n_r"], n_theta=P["n_theta"], dt=0.0,
                          substeps=P["substeps"], parity=workloads.parity_of(P["m"], P["s"]), bits=256)
    o.pulse(8.0, 4.0, 0.8, 0.6, 2)
    o.step(nit)
    err, umax = o.max_rel_err(got)
    assert umax > 0.05 and err < TOL[W], err


def test_slab_refusals_and_observer():
    _torch()
    lo_rows, hi_rows = slab.split_rows(P["n_r"], 2)
    g = teuk.Teuk(precision=1, own_rows=lo_rows, **P)
    assert g.row0 == 0 and g.n_r == lo_rows[1] + 2
    g.set_initial_pulse(8.0, 4.0, 0.8, 0.6, 2)
    with pytest.raises(teuk.TeukError):
        g.step(1)                       # outer steps need the exchange between iterations
    with pytest.raises(teuk.TeukError):
        g.substep(2)
    with pytest.raises(teuk.TeukError):
        g.set_dissipation(1.0)
    torch = _torch()
    buf = torch.zeros((4, 1, P["n_theta"]), dtype=torch.float64, device="cuda")
    with pytest.raises(teuk.TeukError):
        g.set_halo_rows(buf, None)      # no halo below global row 0
    g.set_halo_rows(None, buf)
    dr = (P["rstar_max"] - P["rstar_min"]) / (P["n_r"] - 1)
    with pytest.raises(teuk.TeukError):
        g.set_observer(P["rstar_min"] + (hi_rows[0] + 2) * dr, 4)  # owned by the other slab
    obs, used = g.observe(P["rstar_min"] + 5 * dr)
    assert abs(used - (P["rstar_min"] + 5 * dr)) < 1e-12
    pitch = (P["n_theta"] + 15) // 16 * 16
    state = torch.zeros((4, 1, g.n_r, pitch), dtype=torch.float64, device="cuda")
    L = teuk.lib()
    rc = L.teuk_substep_noalloc(g._h, ctypes.c_void_p(state.data_ptr()), ctypes.c_void_p(state.data_ptr()), 2)
    assert rc == teuk.ERR_INVALID_ARG       # several iterations need halo exchanges between them
    whole = teuk.Teuk(precision=1, **P)
    with pytest.raises(teuk.TeukError):
        whole.set_halo_rows(None, buf)  # not a slab
    with pytest.raises(teuk.TeukError):
        teuk.Teuk(precision=1, own_rows=(0, 0), **P)  # fewer than three local rows
