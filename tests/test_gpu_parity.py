"""GPU parity: the CUDA library against the CPU oracle (256-bit MPFR unless stated).

Tolerances (max-norm relative error over all compared points and the four components):
FP64 1e-12, double-double 1e-26, quad-double 1e-55. Grids span several thread blocks and a
ragged theta tail (n_theta not a multiple of the warp width or of the 16-double pitch).
"""
import ctypes

import numpy as np
import pytest

from paper_1006_0663_gb300 import teuk, workloads

pytestmark = pytest.mark.gpu

TOL = {1: 1e-12, 2: 1e-26, 4: 1e-55}
COEF_TOL = {1: 1e-13, 2: 1e-28, 4: 1e-57}


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    _cuda()


def small(**kw):
    base = dict(M=1.0, a=0.9, s=-2, m=2, rstar_min=-30.0, rstar_max=50.0, n_r=41, n_theta=24,
                dt=0.0, substeps=4, theta_order=10, parity=0)
    base.update(kw)
    return base


def make_pair(oracle_mod, p, W, bits=256, row_lo=0, row_hi=None):
    g = teuk.Teuk(precision=W, **p)
    par = p["parity"] or workloads.parity_of(p["m"], p["s"])
    o = oracle_mod.Oracle(M=p["M"], a=p["a"], s=p["s"], m=p["m"], rstar_min=p["rstar_min"],
                          rstar_max=p["rstar_max"], n_r=p["n_r"], n_theta=p["n_theta"], dt=p["dt"],
                          substeps=p["substeps"], theta_order=p["theta_order"], parity=par,
                          row_lo=row_lo, row_hi=row_hi, bits=bits)
    return g, o


def word_diff(gw, ow):
    """(sum of gw words) - (sum of ow words), summed from the smallest words up."""
    diff = 0.0
    for k in reversed(range(max(gw.shape[0], ow.shape[0]))):
        a = gw[k] if k < gw.shape[0] else 0.0
        b = ow[k] if k < ow.shape[0] else 0.0
        diff = diff + (a - b)
    return diff


def coef_err(gc, oc, W):
    """max over components of max|gpu - oracle| / max|oracle| (exact word sums in mpmath-free
    form: the difference of the leading words plus the difference of the tails)."""
    worst = 0.0
    for c in range(gc.shape[0]):
        diff = np.zeros(gc.shape[2:])
        # sum word differences from the smallest: exact enough for a tolerance check
        for k in reversed(range(max(W, oc.shape[1]))):
            gw = gc[c, k] if k < W else 0.0
            ow = oc[c, k] if k < oc.shape[1] else 0.0
            diff = diff + (gw - ow)
        scale = np.abs(oc[c, 0]).max()
        if scale > 0:
            worst = max(worst, np.abs(diff).max() / scale)
    return worst


@pytest.mark.parametrize("W", [1, 2, 4])
def test_mw_device_matches_host(W):
    rng = np.random.default_rng(3)
    n = 1000
    a = np.zeros((W, n)); b = np.zeros((W, n))
    a[0] = rng.uniform(0.5, 2, n) * 2.0 ** rng.integers(-20, 20, n)
    b[0] = rng.uniform(-2, 2, n) * 2.0 ** rng.integers(-20, 20, n)
    for k in range(1, W):
        a[k] = a[k - 1] * rng.uniform(-1, 1, n) * 2.0 ** -53
        b[k] = b[k - 1] * rng.uniform(-1, 1, n) * 2.0 ** -53
    for op in (0, 1, 2, 3, 4, 7):
        c = np.zeros_like(a); c[0] = rng.uniform(-1, 1, n)
        h = teuk.mw_eval(op, W, a, b, out=c, device=False)
        d = teuk.mw_eval(op, W, a, b, out=c, device=True)
        np.testing.assert_array_equal(h, d, err_msg=f"op {op}")


@pytest.mark.parametrize("W", [1, 2, 4])
def test_tortoise_and_coefficients(oracle_mod, W):
    p = small(n_r=37, n_theta=20, rstar_min=-120.0, rstar_max=300.0)
    g, o = make_pair(oracle_mod, p, W)
    grid = o.grid(words=5)
    for which, key in ((0, "x_node"), (1, "x_half")):
        xg = g.tortoise_x(which)
        xo = grid[key]
        rel = np.abs(word_diff(xg, xo)) / np.abs(xo[0])
        assert rel.max() < COEF_TOL[W], (which, rel.max())
    for which in (0, 1):
        err = coef_err(g.coeffs(which), o.coeffs(which, words=5), W)
        assert err < COEF_TOL[W], (which, err)


@pytest.mark.parametrize("W", [1, 2, 4])
def test_initial_pulse(oracle_mod, W):
    p = small()
    g, o = make_pair(oracle_mod, p, W)
    g.set_initial_pulse(10.0, 4.0, 0.7, 0.6, 2)
    o.pulse(10.0, 4.0, 0.7, 0.6, 2)
    err, umax = o.max_rel_err(g.get_state())
    assert umax > 0.1 and err < TOL[W] / 10, err


CASES = [
    dict(),                                                    # s=-2, m=2, parity +1
    dict(a=0.6, s=-1, m=2, n_theta=40, n_r=53),                # odd parity (m+s odd)
    dict(a=0.99, s=0, m=0, n_theta=17, n_r=35, substeps=2),    # scalar field, tiny ragged theta
    dict(a=0.5, s=-2, m=1, theta_order=2, n_theta=30),         # 2nd-order theta operator
    dict(a=0.7, s=0, m=1, n_theta=6, n_r=31),                  # narrowest rows: both pole images
]


@pytest.mark.parametrize("W", [1, 2, 4])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_evolution_parity(oracle_mod, W, case):
    p = small(**CASES[case])
    g, o = make_pair(oracle_mod, p, W)
    ell = max(abs(p["m"]), abs(p["s"]))
    g.set_initial_pulse(12.0, 4.0, 0.8, 0.55, ell)
    o.pulse(12.0, 4.0, 0.8, 0.55, ell)
    outer = 3
    g.step(outer)
    g.sync()
    o.step(outer * p["substeps"])
    err, umax = o.max_rel_err(g.get_state())
    assert umax > 0.05
    assert err < TOL[W], err


@pytest.mark.parametrize("W,name,nsub", [(2, "c2", 12), (4, "c3", 8), (1, "c5", 40), (2, "c5", 12),
                                        (1, "c1", 60), (4, "tails", 8)])
def test_full_size_sampled_parity(oracle_mod, W, name, nsub):
    """Workload at its full size in the benchmark's launch configuration (autotuned shape, FP64
    error-free transforms for dd and qd); the 256-bit oracle computes a window of rows, exact
    in its interior after nsub iterations (one row per iteration of domain of dependence)."""
    prob = workloads.CONFIGS[name]
    p = dict(M=prob.M, a=prob.a, s=prob.s, m=prob.m, rstar_min=prob.rstar_min,
             rstar_max=prob.rstar_max, n_r=prob.n_r, n_theta=prob.n_theta, dt=0.0,
             substeps=prob.substeps, theta_order=10, parity=0)
    # sample where the pulse is, and a window that contains the inner boundary row
    ic = int(round((prob.center - prob.rstar_min) / prob.dr))
    windows = [(ic - 12, ic + 12), (0, 16)]
    bits = 256
    g = teuk.Teuk(precision=W, **p)
    g.tune()
    ar, ai = prob.amps
    g.set_initial_pulse(prob.center, prob.width, ar, ai, prob.ell)
    g.substep(nsub)
    g.sync()
    full = g.get_state()
    # the error is relative to the field's maximum (the pulse window's), as over the whole
    # grid: the inner-boundary window holds Gaussian tails 1e-160 and smaller
    scale = None
    for lo, hi in windows:
        wlo, whi = max(0, lo - nsub - 1), min(prob.n_r - 1, hi + nsub + 1)
        o = oracle_mod.Oracle(M=prob.M, a=prob.a, s=prob.s, m=prob.m, rstar_min=prob.rstar_min,
                              rstar_max=prob.rstar_max, n_r=prob.n_r, n_theta=prob.n_theta, dt=0.0,
                              substeps=prob.substeps, parity=prob.parity, row_lo=wlo, row_hi=whi,
                              bits=bits)
        o.pulse(prob.center, prob.width, ar, ai, prob.ell)
        o.step(nsub)
        planes = np.ascontiguousarray(full[:, :, wlo:whi + 1])
        err, umax = o.max_rel_err(planes, lo - wlo, hi - wlo)
        if scale is None:
            scale = umax
            assert umax > 0
        assert err * umax / scale < TOL[W], (lo, hi, err, umax, scale)


def test_waveform_ring_matches_observe():
    p = small(n_r=61, n_theta=32)
    g = teuk.Teuk(precision=2, **p)
    g.set_initial_pulse(5.0, 4.0, 0.7, 0.6, 2)
    g.set_observer(20.0, capacity=4)
    outs = []
    for _ in range(6):
        g.step(1)
        obs, used = g.observe(20.0)
        outs.append(obs)
    wf = g.read_waveform()
    assert wf.shape == (4, 2, 2, 32)
    for t in range(4):
        np.testing.assert_array_equal(wf[t], outs[2 + t])
    assert abs(used - 20.0) <= 1.0


@pytest.mark.parametrize("W", [1, 2, 4])
def test_conjugation_symmetry_bitwise(W):
    p = small()
    g1 = teuk.Teuk(precision=W, **p)
    g2 = teuk.Teuk(precision=W, **dict(p, a=-p["a"]))
    g1.set_initial_pulse(10.0, 4.0, 0.8, 0.6, 2)
    g2.set_initial_pulse(10.0, 4.0, 0.8, -0.6, 2)
    g1.step(2)
    g2.step(2)
    u1, u2 = g1.get_state(), g2.get_state()
    np.testing.assert_array_equal(u1[0], u2[0])
    np.testing.assert_array_equal(u1[1], -u2[1])
    np.testing.assert_array_equal(u1[2], u2[2])
    np.testing.assert_array_equal(u1[3], -u2[3])


@pytest.mark.parametrize("W", [1, 2])
def test_checkpoint_resume_bitwise(W):
    p = small()
    g1 = teuk.Teuk(precision=W, **p)
    g1.set_initial_pulse(10.0, 4.0, 0.8, 0.6, 2)
    g1.step(4)
    ref = g1.get_state()
    g2 = teuk.Teuk(precision=W, **p)
    g2.set_initial_pulse(10.0, 4.0, 0.8, 0.6, 2)
    g2.step(2)
    snap = g2.get_state()
    g3 = teuk.Teuk(precision=W, **p)
    g3.set_state(snap, 8)
    g3.step(2)
    np.testing.assert_array_equal(g3.get_state(), ref)


def test_nonfinite_guard_reports_error():
    p = small()
    g = teuk.Teuk(precision=1, **p)
    g.set_initial_pulse(10.0, 4.0, 0.8, 0.6, 2)
    u = g.get_state()
    u[2, 0, 20, 5] = np.nan  # a corrupted state made on the host
    g.set_state(u)
    g.step(1)
    with pytest.raises(teuk.TeukError) as e:
        g.sync()
    assert e.value.code == teuk.ERR_NONFINITE


@pytest.mark.parametrize("W", [1, 2])
def test_autotuner_keeps_state_and_results(W):
    """teuk_tune times launch shapes on a copy of the state: the state is unchanged and the
    results of any launch shape are identical bit for bit (same arithmetic per point)."""
    p = small(n_r=61, n_theta=40)
    g1 = teuk.Teuk(precision=W, **p)
    g2 = teuk.Teuk(precision=W, **p)
    for g in (g1, g2):
        g.set_initial_pulse(10.0, 4.0, 0.8, 0.6, 2)
    before = g2.get_state()
    rows = g2.tune()
    assert rows in (0, 1, 2, 3, 4, 7, 8)  # 0: the one-warp-per-32-columns kernels won
    np.testing.assert_array_equal(g2.get_state(), before)
    g1.step(2)
    g2.step(2)
    np.testing.assert_array_equal(g1.get_state(), g2.get_state())
    shape = g2.launch_shape()
    if shape["variant"] == 9:  # persistent launches won: one per 1 or 8 outer steps
        assert g2.kernel_launches in (1, 2)
    elif shape["variant"] == 10:  # fused iterations: one launch each
        assert g2.kernel_launches == 2 * p["substeps"]
    else:
        assert g2.kernel_launches == 2 * 2 * p["substeps"]


@pytest.mark.parametrize("W", [2, 4])
def test_mw_dot11_device_matches_host(W):
    rng = np.random.default_rng(9)
    n = 4096
    a = np.zeros((W, n)); b = np.zeros((W, n))
    a[0] = rng.uniform(-2, 2, n) * 1e3
    b[0] = rng.uniform(-1, 1, n)
    for k in range(1, W):
        a[k] = a[k - 1] * rng.uniform(-1, 1, n) * 2.0 ** -53
        b[k] = b[k - 1] * rng.uniform(-1, 1, n) * 2.0 ** -53
    c = np.zeros_like(a)
    h = teuk.mw_eval(8, W, a, b, out=c, device=False)
    d = teuk.mw_eval(8, W, a, b, out=c, device=True)
    np.testing.assert_array_equal(h, d)


BATCH_MEMBERS = [
    dict(a=0.9, s=-2, m=2, n_r=41, n_theta=24, substeps=4),
    dict(a=0.3, s=0, m=1, n_r=77, n_theta=64, substeps=2, rstar_max=90.0),
    dict(a=0.7, s=-1, m=-3, n_r=33, n_theta=32, substeps=7),
    dict(a=0.5, s=-2, m=0, n_r=129, n_theta=128, substeps=16, rstar_min=-60.0),
    dict(a=0.99, s=0, m=0, n_r=50, n_theta=40, substeps=3, theta_order=2),
]


def _member(W, kw):
    p = small(**kw)
    g = teuk.Teuk(precision=W, **p)
    ell = max(abs(p["m"]), abs(p["s"]))
    g.set_initial_pulse(8.0, 4.0, 0.8, 0.6, ell)
    g.set_observer(15.0, capacity=16)
    return g


@pytest.mark.parametrize("W", [1, 2, 4])
def test_batch_matches_individual_bitwise(W):
    """Uneven members (sizes, theta resolutions, spins, substeps) advanced in one cooperative
    launch give exactly the states and waveforms of advancing each member alone."""
    alone = [_member(W, kw) for kw in BATCH_MEMBERS]
    batched = [_member(W, kw) for kw in BATCH_MEMBERS]
    n = 5
    for g in alone:
        g.step(n)
        g.sync()
    b = teuk.Batch(batched)
    b.step(n)
    b.sync()
    info = b.info()
    assert info["k_max"] == 16 and info["launches"] == 1
    for ga, gb in zip(alone, batched):
        np.testing.assert_array_equal(ga.get_state(), gb.get_state())
        np.testing.assert_array_equal(ga.read_waveform(), gb.read_waveform())
    b.close()
    _batch_members_vs_oracle(batched, n, W)


def _batch_members_vs_oracle(members, n_outer, W):
    """Each batched member's state against the 256-bit oracle after n_outer outer steps."""
    import oracle
    for g, kw in zip(members, BATCH_MEMBERS):
        p = small(**kw)
        par = p["parity"] or workloads.parity_of(p["m"], p["s"])
        o = oracle.Oracle(M=p["M"], a=p["a"], s=p["s"], m=p["m"], rstar_min=p["rstar_min"],
                          rstar_max=p["rstar_max"], n_r=p["n_r"], n_theta=p["n_theta"], dt=p["dt"],
                          substeps=p["substeps"], theta_order=p["theta_order"], parity=par, bits=256)
        ell = max(abs(p["m"]), abs(p["s"]))
        o.pulse(8.0, 4.0, 0.8, 0.6, ell)
        o.step(n_outer * p["substeps"])
        err, umax = o.max_rel_err(g.get_state())
        assert umax > 0.01 and err < TOL[W], (kw, err)


@pytest.mark.parametrize("W", [2, 4])
def test_batch_engine_matches_individual_bitwise(W):
    """Members on the integer engine advanced in one cooperative launch (batch_ix_kernel) give
    exactly the states and waveforms of advancing each alone on the engine; a batch refuses to
    step once a member changed engine, and members of different engines make no batch."""
    alone = [_member(W, kw) for kw in BATCH_MEMBERS]
    batched = [_member(W, kw) for kw in BATCH_MEMBERS]
    for g in alone + batched:
        g.set_engine(1)
    n = 5
    for g in alone:
        g.step(n)
        g.sync()
    b = teuk.Batch(batched)
    b.step(n)
    b.sync()
    assert b.info()["launches"] == 1
    for ga, gb in zip(alone, batched):
        np.testing.assert_array_equal(ga.get_state(), gb.get_state())
        np.testing.assert_array_equal(ga.read_waveform(), gb.read_waveform())
    _batch_members_vs_oracle(batched, n, W)
    batched[0].set_engine(0)
    with pytest.raises(teuk.TeukError):
        b.step(1)
    b.close()
    other = _member(W, BATCH_MEMBERS[1])
    with pytest.raises(teuk.TeukError):
        teuk.Batch([alone[0], other])
    for g in alone + batched + [other]:
        g.close()


def test_engine_wide_rows_shapes():
    """Integer-engine rows of 512 theta cells: shapes whose rows exceed one block's shared
    memory are refused by teuk_set_launch_shape and skipped by the autotuner, and the tuned
    handle steps to the same bits as the default shape."""
    p = small(n_r=41, n_theta=512, substeps=2)
    g1 = teuk.Teuk(precision=2, **p)
    g2 = teuk.Teuk(precision=2, **p)
    for g in (g1, g2):
        g.set_engine(1)
        g.set_initial_pulse(8.0, 4.0, 0.8, 0.6, max(abs(p["m"]), abs(p["s"])))
    with pytest.raises(teuk.TeukError):
        g1.set_launch_shape(32, 8, 0)
    g1.tune()
    sh = g1.launch_shape()
    assert sh["variant"] in (0, 1, 2) and sh["threads_theta"] * sh["rows_per_block"] <= 256
    g1.step(3)
    g2.step(3)
    g1.sync()
    g2.sync()
    np.testing.assert_array_equal(g1.get_state(), g2.get_state())
    g1.close()
    g2.close()


@pytest.mark.parametrize("W,engine", [(1, 0), (2, 1)])
def test_kernel_timing_inside_graphs(W, engine):
    """Per-kernel timing keeps graph replay: the events are nodes of the captured outer step
    around its last iteration, and one drain reports the last replay's half-step and full-step
    launch; without graphs every launch is timed. Timing does not change the results."""
    import torch
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p = small(n_r=57, n_theta=40, substeps=3)
        states = []
        for graphs, timing in [(True, True), (False, True), (True, False)]:
            g = teuk.Teuk(precision=W, **p)
            if engine:
                g.set_engine(1)
            g.use_graphs(graphs)
            g.set_initial_pulse(10.0, 4.0, 0.8, 0.6, 2)
            g.set_observer(12.0, capacity=8)
            g.timing(timing)
            g.step(4)
            g.sync()
            ms_h, ms_f, n_h, n_f = g.kernel_times()
            if timing:
                expect = 1 if graphs else 4 * p["substeps"]
                assert (n_h, n_f) == (expect, expect), (graphs, n_h, n_f)
                assert ms_h > 0 and ms_f > 0
            else:
                assert (n_h, n_f) == (0, 0)
            states.append((g.get_state(), g.read_waveform()))
            g.close()
        for st, wf in states[1:]:
            np.testing.assert_array_equal(st, states[0][0])
            np.testing.assert_array_equal(wf, states[0][1])


def test_batch_chunks_of_200_steps():
    alone = [_member(1, kw) for kw in BATCH_MEMBERS[:2]]
    batched = [_member(1, kw) for kw in BATCH_MEMBERS[:2]]
    for g in alone:
        g.step(203)
    b = teuk.Batch(batched)
    b.step(203)
    b.sync()
    assert b.info()["launches"] == 2
    for ga, gb in zip(alone, batched):
        np.testing.assert_array_equal(ga.get_state(), gb.get_state())
        np.testing.assert_array_equal(ga.read_waveform(), gb.read_waveform())


@pytest.mark.parametrize("W", [1, 2])
def test_graph_replay_matches_direct_launches(W):
    """teuk_step replays one captured outer step as a CUDA graph on a non-default stream;
    states and observer samples equal those of launching the kernels one by one."""
    import torch
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p = small(n_r=57, n_theta=40)
        g1 = teuk.Teuk(precision=W, **p)
        g2 = teuk.Teuk(precision=W, **p)
        g2.use_graphs(False)
        for g in (g1, g2):
            g.set_initial_pulse(10.0, 4.0, 0.8, 0.6, 2)
            g.set_observer(12.0, capacity=3)
        g1.step(2)
        g2.step(2)
        g1.step(3)   # reuses the captured graph
        g2.step(3)
        g1.sync()
        g2.sync()
        np.testing.assert_array_equal(g1.get_state(), g2.get_state())
        np.testing.assert_array_equal(g1.read_waveform(), g2.read_waveform())
        assert g1.kernel_launches == g2.kernel_launches == 5 * 2 * p["substeps"]
        g1.tune()    # invalidates the graph; the next step recaptures
        g1.step(1)
        g2.step(1)
        g1.sync()
        np.testing.assert_array_equal(g1.get_state(), g2.get_state())
    torch.cuda.synchronize()


@pytest.mark.parametrize("W", [1, 2, 4])
@pytest.mark.parametrize("n_theta,parity_m", [(24, 2), (70, 1), (128, 2)])
def test_launch_shapes_bitwise_identical(W, n_theta, parity_m):
    """Every launch shape (rows per block, threads per row with several columns per thread,
    register budgets, one warp per 32 columns with recomputed halos, balanced blocks that
    share rows) gives the same bits, state and observer samples."""
    p = small(n_r=37, n_theta=n_theta, m=parity_m)
    shapes = [(32, 1, 0), (64, 2, 1), (32, 8, 2), (0, 0, 3), (0, 0, 4), (0, 0, 5),
              (32, 1, 6), (64, 1, 7), (128, 1, 8), (256, 1, 7)]
    ref = None
    for tx, ty, v in shapes:
        g = teuk.Teuk(precision=W, **p)
        g.set_launch_shape(tx or 32, ty or 1, v)
        g.set_initial_pulse(10.0, 4.0, 0.8, 0.6, 2)
        g.set_observer(5.0, capacity=4)
        g.step(2)
        g.sync()
        st = (g.get_state(), g.read_waveform())
        if ref is None:
            ref = st
        else:
            np.testing.assert_array_equal(st[0], ref[0], err_msg=f"shape {(tx, ty, v)}")
            np.testing.assert_array_equal(st[1], ref[1], err_msg=f"shape {(tx, ty, v)} waveform")
        g.close()


MULTIPOLE_CASES = [
    dict(a=0.9, s=0, m=0, n_theta=24, ell0=0),                  # scalar, l = 0 data (Fig. 1 set-up)
    dict(a=0.7, s=-2, m=2, n_theta=33, ell0=2),                 # ragged theta, even parity
    dict(a=0.6, s=-1, m=2, n_theta=20, n_r=45, ell0=2),         # odd parity (m + s odd)
]


@pytest.mark.parametrize("W", [1, 2, 4])
@pytest.mark.parametrize("case", range(len(MULTIPOLE_CASES)))
def test_multipole_parity(oracle_mod, W, case):
    """Device multipoles c_l(t) of the recorded waveform against the oracle's projection of its
    own evolution (same problem, 256-bit), l = l_min .. l_min + 7."""
    c = dict(MULTIPOLE_CASES[case])
    ell0 = c.pop("ell0")
    p = small(**c)
    g, o = make_pair(oracle_mod, p, W)
    g.set_initial_pulse(12.0, 4.0, 0.8, 0.55, ell0)
    o.pulse(12.0, 4.0, 0.8, 0.55, ell0)
    robs = 20.0
    outer = 5
    g.set_observer(robs, capacity=outer)
    _, used = g.observe(robs)
    dr = (p["rstar_max"] - p["rstar_min"]) / (p["n_r"] - 1)
    i_obs = int(round((used - p["rstar_min"]) / dr))
    lo = max(abs(p["m"]), abs(p["s"]))
    hi = lo + 7
    samples = []
    for _ in range(outer):
        g.step(1)
        o.step(p["substeps"])
        samples.append(o.get_row(i_obs, words=5)[:2])  # Phi_R, Phi_I: [2][5][n_theta]
    g.sync()
    cg = g.read_multipoles(lo, hi)                       # [n][n_ell][2][W]
    co = oracle_mod.project(p["s"], p["m"], lo, hi, np.array(samples), bits=256, out_words=5)
    assert cg.shape == (outer, hi - lo + 1, 2, W)
    scale = max(np.abs(np.array(samples)[:, :, 0]).max(), 1e-300)
    diff = np.zeros(cg.shape[:3])
    for k in reversed(range(5)):
        diff = diff + ((cg[..., k] if k < W else 0.0) - co[..., k])
    err = np.abs(diff).max() / scale
    assert np.abs(co[:, 0, :, 0]).max() > 1e-3 * scale
    assert err < TOL[W], err


def test_multipoles_of_waveform_ring_wraparound():
    """With more outer steps than ring slots, the multipoles follow the kept samples (oldest
    first), identical to projecting the same samples recorded in a larger ring."""
    p = small(s=0, m=0, a=0.9, n_theta=24)
    g1 = teuk.Teuk(precision=2, **p)
    g2 = teuk.Teuk(precision=2, **p)
    for g, cap in ((g1, 3), (g2, 16)):
        g.set_initial_pulse(12.0, 4.0, 0.8, 0.55, 0)
        g.set_observer(20.0, capacity=cap)
        g.step(7)
    m1 = g1.read_multipoles(0, 6)
    m2 = g2.read_multipoles(0, 6)
    assert m1.shape[0] == 3 and m2.shape[0] == 7
    np.testing.assert_array_equal(m1, m2[4:])
    with pytest.raises(teuk.TeukError):
        g1.read_multipoles(0, 24)   # l_max >= n_theta


@pytest.mark.parametrize("W", [1, 2, 4])
def test_host_state_iterations_match_resident_bitwise(W):
    """The host-resident data flow (state copied in and out every iteration) runs the same
    kernels on the same values: bit-identical to iterations on the resident state."""
    p = small()
    g1 = teuk.Teuk(precision=W, **p)
    g1.set_initial_pulse(10.0, 4.0, 0.8, 0.6, 2)
    host = g1.get_state()
    g1.substep_host_state(host, 5)
    g2 = teuk.Teuk(precision=W, **p)
    g2.set_initial_pulse(10.0, 4.0, 0.8, 0.6, 2)
    g2.substep(5)
    g2.sync()
    np.testing.assert_array_equal(host, g2.get_state())
    np.testing.assert_array_equal(g1.get_state(), host)
    import oracle
    o = oracle.Oracle(M=p["M"], a=p["a"], s=p["s"], m=p["m"], rstar_min=p["rstar_min"],
                      rstar_max=p["rstar_max"], n_r=p["n_r"], n_theta=p["n_theta"], dt=p["dt"],
                      substeps=p["substeps"], theta_order=p["theta_order"],
                      parity=workloads.parity_of(p["m"], p["s"]), bits=256)
    o.pulse(10.0, 4.0, 0.8, 0.6, 2)
    o.step(5)
    err, umax = o.max_rel_err(host)
    assert umax > 0.05 and err < TOL[W], err


def _paper_parity(m):
    """Sec. 3.B's axis rule: d_theta Phi = 0 (even reflection) for even |m|, Phi = 0 (odd) for odd |m|."""
    return 1 if abs(m) % 2 == 0 else -1


@pytest.mark.parametrize("W,engine", [(1, 0), (2, 0), (4, 0), (2, 1), (4, 1)])
@pytest.mark.parametrize("order", [2, 10])
@pytest.mark.parametrize("rule", ["regular", "paper"])
@pytest.mark.parametrize("sm", [(-1, 2), (0, 1), (-2, 3)])
def test_theta_order_and_parity_rule_matrix(oracle_mod, W, engine, order, rule, sm):
    """Regression matrix of the angular options: 2nd-order (Sec. 3.B) and 10th-order (Sec. 3.D)
    theta differences x the regular (-1)^(m+s) reflection and the paper's |m| rule, which
    differ for s = -1, m = 2 and agree for the other two modes; both multi-word engines."""
    s, m = sm
    parity = workloads.parity_of(m, s) if rule == "regular" else _paper_parity(m)
    p = small(a=0.8, s=s, m=m, n_theta=26, n_r=37, substeps=3, theta_order=order, parity=parity)
    g, o = make_pair(oracle_mod, p, W)
    if engine:
        g.set_engine(1)
    ell = max(abs(m), abs(s))
    g.set_initial_pulse(8.0, 4.0, 0.75, 0.5, ell)
    o.pulse(8.0, 4.0, 0.75, 0.5, ell)
    g.step(3)
    g.sync()
    o.step(9)
    err, umax = o.max_rel_err(g.get_state())
    assert umax > 0.01
    assert err < TOL[W], err


@pytest.mark.parametrize("W", [1, 2, 4])
def test_dissipation_parity(oracle_mod, W):
    """r* dissipation step (not part of the paper's scheme) against the oracle's: 4 outer steps
    and 2 extra iterations (the step comes first in each outer step), graphs and direct
    launches, sigma = 1.5."""
    p = small(s=0, m=0, a=0.9, n_r=45, n_theta=20, substeps=3)
    g, _ = make_pair(oracle_mod, p, W)
    o = oracle_mod.Oracle(M=p["M"], a=p["a"], s=p["s"], m=p["m"], rstar_min=p["rstar_min"],
                          rstar_max=p["rstar_max"], n_r=p["n_r"], n_theta=p["n_theta"], dt=p["dt"],
                          substeps=p["substeps"], theta_order=p["theta_order"], parity=1, bits=256,
                          ko_sigma=1.5)
    g.set_dissipation(1.5)
    g.set_initial_pulse(5.0, 3.0, 0.8, 0.55, 0)
    o.pulse(5.0, 3.0, 0.8, 0.55, 0)
    g.step(4)
    g.substep(2)
    g.sync()
    o.step(4 * 3 + 2)
    err, umax = o.max_rel_err(g.get_state())
    assert umax > 0.05
    assert err < TOL[W], err
    # sigma = 0 is the paper's scheme: bit-identical to a handle that never enabled it
    g0 = teuk.Teuk(precision=W, **p)
    g1 = teuk.Teuk(precision=W, **p)
    g1.set_dissipation(0.7)
    g1.set_dissipation(0.0)
    for h in (g0, g1):
        h.set_initial_pulse(5.0, 3.0, 0.8, 0.55, 0)
        h.step(3)
    np.testing.assert_array_equal(g0.get_state(), g1.get_state())
    with pytest.raises(teuk.TeukError):
        g1.set_dissipation(-1.0)


@pytest.mark.parametrize("W,engine", [(1, 0), (2, 0), (2, 1), (4, 0), (4, 1)])
@pytest.mark.parametrize("s,m", [(0, 0), (-1, 2)])
def test_theta_dissipation_parity(oracle_mod, W, engine, s, m):
    """theta and r* dissipation together (not part of the paper's scheme) against the oracle:
    3 outer steps and 2 extra iterations, even (s = m = 0) and odd (s = -1, m = 2) axis
    parity, both multi-word engines; a sigma beyond the step's stability limit is refused."""
    p = small(s=s, m=m, a=0.9, n_r=45, n_theta=21, substeps=3)
    g = teuk.Teuk(precision=W, **p)
    if engine:
        g.set_engine(engine)
    o = oracle_mod.Oracle(M=p["M"], a=p["a"], s=p["s"], m=p["m"], rstar_min=p["rstar_min"],
                          rstar_max=p["rstar_max"], n_r=p["n_r"], n_theta=p["n_theta"], dt=p["dt"],
                          substeps=p["substeps"], theta_order=p["theta_order"],
                          parity=workloads.parity_of(m, s), bits=256, ko_sigma=1.0, ko_theta=0.6)
    g.set_dissipation(1.0)
    g.set_theta_dissipation(0.6)
    assert g.theta_dissipation == 0.6
    ell = max(abs(m), abs(s))
    g.set_initial_pulse(5.0, 3.0, 0.8, 0.55, ell)
    o.pulse(5.0, 3.0, 0.8, 0.55, ell)
    g.step(3)
    g.substep(2)
    g.sync()
    o.step(3 * 3 + 2)
    err, umax = o.max_rel_err(g.get_state())
    assert umax > 0.05
    assert err < TOL[W], err
    with pytest.raises(teuk.TeukError):
        g.set_theta_dissipation(4.0)  # sigma c_th dt / dtheta > 2 on this grid
    assert g.theta_dissipation == 0.6


@pytest.mark.parametrize("W", [2, 4])
def test_integer_engine_ops_device_matches_host(W):
    rng = np.random.default_rng(21 + W)
    n = 2048
    a = np.zeros((W, n)); b = np.zeros((W, n)); o = np.zeros((W, n))
    for x in (a, b, o):
        x[0] = rng.uniform(-2, 2, n) * 2.0 ** rng.integers(-60, 60, n)
        for k in range(1, W):
            x[k] = x[k - 1] * rng.uniform(-1, 1, n) * 2.0 ** -54
    a[:, ::17] = 0.0
    b[:, 5::13] = a[:, 5::13]
    for op in (9, 10, 11, 12):
        h = teuk.mw_eval(op, W, a, b, out=o, device=False)
        d = teuk.mw_eval(op, W, a, b, out=o, device=True)
        np.testing.assert_array_equal(h, d, err_msg=f"op {op}")


@pytest.mark.parametrize("W", [2, 4])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_integer_engine_evolution_parity(oracle_mod, W, case):
    """Double-double and quad-double through the integer engine (every dot product in fixed
    point on the integer pipe, rounded once) against the 256-bit oracle, the same cases as the FP64-transform
    engine."""
    p = small(**CASES[case])
    g, o = make_pair(oracle_mod, p, W)
    g.set_engine(1)
    assert g.engine == 1
    ell = max(abs(p["m"]), abs(p["s"]))
    g.set_initial_pulse(12.0, 4.0, 0.8, 0.55, ell)
    o.pulse(12.0, 4.0, 0.8, 0.55, ell)
    g.step(3)
    g.sync()
    o.step(3 * p["substeps"])
    err, umax = o.max_rel_err(g.get_state())
    assert umax > 0.05
    assert err < TOL[W], err


def _member_problem(name):
    return workloads.batch_member(int(name[3:-1])) if name.startswith("c4[") else workloads.CONFIGS[name]


@pytest.mark.parametrize("W,name,nsub", [(2, "c2", 12), (4, "c3", 8), (2, "c5", 12), (2, "c4[27]", 12),
                                        (2, "c4[40]", 12), (2, "c4[54]", 12), (2, "c4[60]", 12)])
def test_integer_engine_full_size_window(oracle_mod, W, name, nsub):
    """Full-size workloads on the integer engine, in the benchmark's launch configuration (tuned),
    against a 256-bit oracle window around the pulse (domain of dependence). The c4 members are
    the batch's largest (4075 x 256, s = -1), two others with 256 theta cells and s = -1 / -2,
    and the one with the most iterations per outer step (454)."""
    prob = _member_problem(name)
    p = dict(M=prob.M, a=prob.a, s=prob.s, m=prob.m, rstar_min=prob.rstar_min, rstar_max=prob.rstar_max,
             n_r=prob.n_r, n_theta=prob.n_theta, dt=0.0, substeps=prob.substeps, theta_order=10, parity=0)
    g = teuk.Teuk(precision=W, **p)
    g.set_engine(1)
    g.tune()
    ar, ai = prob.amps
    g.set_initial_pulse(prob.center, prob.width, ar, ai, prob.ell)
    g.substep(nsub)
    g.sync()
    full = g.get_state()
    ic = int(round((prob.center - prob.rstar_min) / prob.dr))
    lo, hi = ic - 12, ic + 12
    wlo, whi = lo - nsub - 1, hi + nsub + 1
    o = oracle_mod.Oracle(M=prob.M, a=prob.a, s=prob.s, m=prob.m, rstar_min=prob.rstar_min,
                          rstar_max=prob.rstar_max, n_r=prob.n_r, n_theta=prob.n_theta, dt=0.0,
                          substeps=prob.substeps, parity=prob.parity, row_lo=wlo, row_hi=whi, bits=256)
    o.pulse(prob.center, prob.width, ar, ai, prob.ell)
    o.step(nsub)
    err, umax = o.max_rel_err(np.ascontiguousarray(full[:, :, wlo:whi + 1]), lo - wlo, hi - wlo)
    assert umax > 0 and err < TOL[W], err


@pytest.mark.parametrize("W", [2, 4])
@pytest.mark.parametrize("n_theta", [24, 70])
def test_integer_engine_launch_shapes_and_graphs_bitwise(W, n_theta):
    """Within the integer engine every launch shape and register budget, and graph replay,
    give the same bits (integer arithmetic per point does not depend on the launch)."""
    p = small(n_r=37, n_theta=n_theta)
    ref = None
    for tx, ty, v, graphs in [(32, 1, 0, True), (64, 2, 1, False), (32, 4, 2, True), (128, 1, 1, True)]:
        g = teuk.Teuk(precision=W, **p)
        g.set_engine(1)
        g.set_launch_shape(tx, ty, v)
        g.use_graphs(graphs)
        g.set_initial_pulse(10.0, 4.0, 0.8, 0.6, 2)
        g.set_observer(5.0, capacity=4)
        g.step(2)
        g.sync()
        st = (g.get_state(), g.read_waveform())
        if ref is None:
            ref = st
        else:
            np.testing.assert_array_equal(st[0], ref[0], err_msg=str((tx, ty, v)))
            np.testing.assert_array_equal(st[1], ref[1], err_msg=str((tx, ty, v)))
        g.close()


@pytest.mark.parametrize("W,engine", [(1, 0), (2, 0), (2, 1), (4, 0), (4, 1)])
@pytest.mark.parametrize("scale", [-400, 400])
def test_power_of_two_scale_covariance_bitwise(W, engine, scale):
    """The scheme is linear in the state and both engines' arithmetic commutes with scaling by
    a power of two (exponents shift, mantissas do not change, no value leaves the normal
    range here): the evolved state and waveform of 2^scale u0 are 2^scale times those of u0,
    bit for bit. Pins the exponent bookkeeping (block-floating rows, accumulator bases) far
    from exponent 0."""
    p = small(a=0.7, s=-1, m=1, n_theta=40, n_r=45, substeps=3)
    runs = []
    for k in (0, scale):
        g = teuk.Teuk(precision=W, **p)
        if engine:
            g.set_engine(1)
        g.set_initial_pulse(8.0, 4.0, 0.8, 0.6, 1)
        g.set_state(g.get_state() * 2.0 ** k)
        g.set_observer(12.0, capacity=4)
        g.step(3)
        g.sync()
        runs.append((g.get_state(), g.read_waveform()))
        g.close()
    (s0, w0), (s1, w1) = runs
    assert np.abs(s0).max() > 0
    np.testing.assert_array_equal(s1, s0 * 2.0 ** scale)
    np.testing.assert_array_equal(w1, w0 * 2.0 ** scale)


@pytest.mark.parametrize("W", [2, 4])
def test_engine_switch_mid_run_parity(oracle_mod, W):
    """The state stays in multi-word doubles whichever engine steps it: a run that alternates
    engines (integer, FP64 transforms, integer) between outer steps stays within the
    precision's tolerance of the 256-bit oracle, and its observer ring keeps its samples."""
    p = small(a=0.6, s=-1, m=2, n_theta=40, n_r=53)
    g, o = make_pair(oracle_mod, p, W)
    ell = max(abs(p["m"]), abs(p["s"]))
    g.set_initial_pulse(12.0, 4.0, 0.8, 0.55, ell)
    o.pulse(12.0, 4.0, 0.8, 0.55, ell)
    g.set_observer(15.0, capacity=8)
    for engine in (1, 0, 1):
        g.set_engine(engine)
        g.step(1)
    g.sync()
    assert g.engine == 1
    o.step(3 * p["substeps"])
    err, umax = o.max_rel_err(g.get_state())
    assert umax > 0.05
    assert err < TOL[W], err
    assert g.read_waveform().shape[0] == 3


@pytest.mark.parametrize("W", [2, 4])
def test_integer_engine_reports_nonfinite_and_rejects_fp64(W):
    p = small()
    g = teuk.Teuk(precision=W, **p)
    g.set_engine(1)
    g.set_initial_pulse(10.0, 4.0, 0.8, 0.6, 2)
    st = g.get_state()
    st[0, 0, 20, 5] = np.inf
    g.set_state(st)
    g.step(1)
    with pytest.raises(teuk.TeukError) as e:
        g.sync()
    assert e.value.code == teuk.ERR_NONFINITE
    h = teuk.Teuk(precision=1, **p)
    with pytest.raises(teuk.TeukError):
        h.set_engine(1)
    assert h.engine == 0


@pytest.mark.parametrize("W", [2, 4])
def test_engine_copy_wait_gives_up_and_reports_timeout(oracle_mod, W):
    """The integer engine's bounded wait for its bulk copies into shared memory: with the test
    hook, one block arms its barrier without issuing any copy (nothing in flight), gives up
    after 2^10 tries, skips its rows and sets the status bit that teuk_sync reports as
    TEUK_ERR_TIMEOUT. After the hook is cleared and the state replaced, the same handle steps
    correctly again (256-bit oracle)."""
    p = small(n_r=45, n_theta=24)
    g = teuk.Teuk(precision=W, **p)
    g.set_engine(1)
    L = teuk.lib()
    g.set_initial_pulse(8.0, 4.0, 0.8, 0.6, 2)
    assert L.teuk_test_stall_copies(g._h, 1, 10) == teuk.OK
    g.substep(2)
    assert L.teuk_sync(g._h) == teuk.ERR_TIMEOUT
    assert L.teuk_sync(g._h) == teuk.ERR_TIMEOUT  # kept until the state is replaced
    assert L.teuk_test_stall_copies(g._h, 0, 9) == teuk.ERR_INVALID_ARG
    assert L.teuk_test_stall_copies(g._h, -1, 20) == teuk.OK
    g.set_initial_pulse(8.0, 4.0, 0.8, 0.6, 2)
    g.substep(6)
    g.sync()
    o = oracle_mod.Oracle(M=p["M"], a=p["a"], s=p["s"], m=p["m"], rstar_min=p["rstar_min"],
                          rstar_max=p["rstar_max"], n_r=p["n_r"], n_theta=p["n_theta"], dt=p["dt"],
                          substeps=p["substeps"], parity=workloads.parity_of(p["m"], p["s"]), bits=256)
    o.pulse(8.0, 4.0, 0.8, 0.6, 2)
    o.step(6)
    err, umax = o.max_rel_err(g.get_state())
    assert umax > 0.05 and err < TOL[W], err
    g2 = teuk.Teuk(precision=W, **p)  # FP64-transform engine: no such wait
    assert L.teuk_test_stall_copies(g2._h, 1, 10) == teuk.ERR_INVALID_ARG


@pytest.mark.parametrize("W", [1, 2, 4])
@pytest.mark.parametrize("rows,steps_per_launch", [(1, 1), (2, 8), (4, 3), (8, 1)])
def test_persistent_launches_bitwise_and_oracle(oracle_mod, W, rows, steps_per_launch):
    """Outer steps in persistent cooperative launches (neighbour progress counters instead of
    launch boundaries) give exactly the states and waveform samples of the graph-replayed
    row kernels, with several launches in a row, and agree with the 256-bit oracle."""
    p = small(n_r=53)
    ref = teuk.Teuk(precision=W, **p)
    per = teuk.Teuk(precision=W, **p)
    per.set_persistent(rows_per_block=rows, steps_per_launch=steps_per_launch)
    assert per.launch_shape()["variant"] == 9
    for g in (ref, per):
        g.set_initial_pulse(8.0, 4.0, 0.8, 0.6, 2)
        g.set_observer(20.0, capacity=32)
        g.step(7)
        g.step(4)
        g.sync()
    np.testing.assert_array_equal(ref.get_state(), per.get_state())
    np.testing.assert_array_equal(ref.read_waveform(), per.read_waveform())
    launches = -(-7 // steps_per_launch) + -(-4 // steps_per_launch)
    assert per.kernel_launches == launches
    o = oracle_mod.Oracle(M=p["M"], a=p["a"], s=p["s"], m=p["m"], rstar_min=p["rstar_min"],
                          rstar_max=p["rstar_max"], n_r=p["n_r"], n_theta=p["n_theta"], dt=p["dt"],
                          substeps=p["substeps"], parity=workloads.parity_of(p["m"], p["s"]), bits=256)
    o.pulse(8.0, 4.0, 0.8, 0.6, 2)
    o.step(11 * p["substeps"])
    err, umax = o.max_rel_err(per.get_state())
    assert umax > 0.01 and err < TOL[W], err


def test_persistent_c1_and_refusals():
    """The FP64 benchmark grid (256 x 64) through persistent launches and the tuner: bit-identical
    to graph replay; a grid whose blocks cannot all be resident is refused, not launched."""
    prob = workloads.CONFIGS["c1"].with_(ko_sigma=0.0)  # persistent launches take no dissipation
    ref = teuk.Teuk.from_problem(prob)
    per = teuk.Teuk.from_problem(prob)
    per.set_persistent(rows_per_block=2, steps_per_launch=4)
    ar, ai = prob.amps
    for g in (ref, per):
        g.set_initial_pulse(prob.center, prob.width, ar, ai, prob.ell)
        g.set_observer(prob.rstar_obs, capacity=16)
        g.step(5)
        g.sync()
    np.testing.assert_array_equal(ref.get_state(), per.get_state())
    np.testing.assert_array_equal(ref.read_waveform(), per.read_waveform())
    before = per.get_state()
    per.tune()  # tries persistent shapes too; keeps the state
    np.testing.assert_array_equal(before, per.get_state())
    ref.step(2)
    per.step(2)
    per.sync()
    np.testing.assert_array_equal(ref.get_state(), per.get_state())
    big = teuk.Teuk(precision=1, M=1.0, a=0.5, s=0, m=0, rstar_min=-50.0, rstar_max=150.0,
                    n_r=40001, n_theta=32, substeps=1)
    big.set_persistent(rows_per_block=1)
    with pytest.raises(teuk.TeukError) as e:
        big.step(1)
    assert e.value.code == teuk.ERR_INVALID_ARG
    g = teuk.Teuk(precision=2, **small())
    g.set_engine(1)
    with pytest.raises(teuk.TeukError):
        g.set_persistent(rows_per_block=2)


def test_persistent_wait_gives_up_and_reports_timeout(oracle_mod):
    """The persistent kernel's bounded waits: with the test hook one block never publishes its
    progress counters, its neighbours give up after 2^10 polls, the abort word ends every
    other wait, and teuk_sync reports TEUK_ERR_TIMEOUT; with the hook cleared and the state
    replaced, the handle steps correctly again (bit-identical to graph replay)."""
    p = small(n_r=53)
    g = teuk.Teuk(precision=1, **p)
    g.set_persistent(rows_per_block=2, steps_per_launch=2)
    L = teuk.lib()
    g.set_initial_pulse(8.0, 4.0, 0.8, 0.6, 2)
    assert L.teuk_test_stall_copies(g._h, 3, 10) == teuk.OK
    g.step(2)
    assert L.teuk_sync(g._h) == teuk.ERR_TIMEOUT
    assert L.teuk_test_stall_copies(g._h, -1, 20) == teuk.OK
    ref = teuk.Teuk(precision=1, **p)
    for h in (g, ref):
        h.set_initial_pulse(8.0, 4.0, 0.8, 0.6, 2)
        h.step(3)
        h.sync()
    np.testing.assert_array_equal(g.get_state(), ref.get_state())


@pytest.mark.parametrize("W", [1, 2])
def test_grid_fields_parity_rule_and_dissipation(W):
    """teuk_grid.parity = 2 is the paper's |m| rule (bitwise equal to the explicit sign), and
    ko_sigma / ko_theta given in the grid are the setters' dissipation (bitwise equal)."""
    for m, s_, sign in ((1, -1, -1), (2, -1, 1), (3, 0, -1)):
        p = small(m=m, s=s_)
        a = teuk.Teuk(precision=W, **dict(p, parity=2))
        b = teuk.Teuk(precision=W, **dict(p, parity=sign))
        for g in (a, b):
            g.set_initial_pulse(8.0, 4.0, 0.8, 0.6, max(abs(m), abs(s_)))
            g.step(2)
        np.testing.assert_array_equal(a.get_state(), b.get_state())
    p = small(s=0, m=0, n_theta=21)
    a = teuk.Teuk(precision=W, ko_sigma=1.0, ko_theta=0.5, **p)
    b = teuk.Teuk(precision=W, **p)
    b.set_dissipation(1.0)
    b.set_theta_dissipation(0.5)
    assert a.theta_dissipation == 0.5
    for g in (a, b):
        g.set_initial_pulse(5.0, 3.0, 0.8, 0.55, 0)
        g.step(3)
    np.testing.assert_array_equal(a.get_state(), b.get_state())
    with pytest.raises(teuk.TeukError):
        teuk.Teuk(precision=W, ko_sigma=-1.0, **p)


def _rich_state(p, W, seed):
    """Random theta content (all multipoles the grid holds) under a Gaussian in r*, zero
    boundary rows: the filter then has something to remove."""
    rng = np.random.default_rng(seed)
    rs = np.linspace(p["rstar_min"], p["rstar_max"], p["n_r"])
    env = np.exp(-((rs - 5.0) / 6.0) ** 2)
    u = np.zeros((4, W, p["n_r"], p["n_theta"]))
    u[:, 0] = rng.standard_normal((4, p["n_r"], p["n_theta"])) * env[None, :, None]
    u[:, 0, 0] = 0.0
    u[:, 0, -1] = 0.0
    return u


@pytest.mark.parametrize("W,engine", [(1, 0), (2, 0), (2, 1), (4, 0), (4, 1)])
@pytest.mark.parametrize("s,m,ko,period", [(0, 0, 0.0, 1), (-1, 2, 1.0, 2), (-2, 2, 1.0, 1), (0, 0, 0.0, 2)])
def test_theta_filter_parity(oracle_mod, W, engine, s, m, ko, period):
    """theta filter (not part of the paper's scheme), alone and after the r* dissipation,
    every outer step or every second one, against the 256-bit oracle (which solves the Gram
    system of its own profiles instead of using orthonormal tables): random theta content, 3
    outer steps and 2 iterations."""
    p = small(s=s, m=m, a=0.9, n_r=45, n_theta=24, substeps=3)
    l_cut = max(abs(s), abs(m)) + 5
    g = teuk.Teuk(precision=W, **p)
    if engine:
        g.set_engine(engine)
    g.set_dissipation(ko)
    g.set_theta_filter(l_cut, period)
    assert g.theta_filter == l_cut and g.theta_filter_period == period
    o = oracle_mod.Oracle(M=p["M"], a=p["a"], s=s, m=m, rstar_min=p["rstar_min"], rstar_max=p["rstar_max"],
                          n_r=p["n_r"], n_theta=p["n_theta"], dt=p["dt"], substeps=p["substeps"],
                          theta_order=p["theta_order"], parity=workloads.parity_of(m, s), bits=256,
                          ko_sigma=ko, theta_filter=l_cut, theta_filter_period=period)
    u0 = _rich_state(p, W, 40 + 3 * abs(s) + m)
    g.set_state(u0)
    o.set_state(u0[:, :1])
    g.step(3)
    g.substep(2)
    g.sync()
    o.step(3 * 3 + 2)
    err, umax = o.max_rel_err(g.get_state())
    assert umax > 0.05
    assert err < TOL[W], err
    # the filter removed the high multipoles: the state differs from the unfiltered run
    g2 = teuk.Teuk(precision=W, **p)
    if engine:
        g2.set_engine(engine)
    g2.set_dissipation(ko)
    g2.set_state(u0)
    g2.step(3)
    g2.substep(2)
    assert np.abs(g2.get_state()[:, 0] - g.get_state()[:, 0]).max() > 1e-3 * umax


@pytest.mark.parametrize("W", [1, 4])
def test_theta_filter_rules(W):
    """Grid field = setter (bit for bit); refused values keep the filter in use; l_cut = 0
    switches it off (bit for bit the unfiltered run); slabs, batches and the no-allocation
    entry point refuse filtered handles."""
    p = small(s=-1, m=2, n_r=41, n_theta=24, substeps=3)
    a = teuk.Teuk(precision=W, theta_filter=6, theta_filter_period=2, **p)
    b = teuk.Teuk(precision=W, **p)
    b.set_theta_filter(6, 2)
    assert a.theta_filter == 6 and b.theta_filter == 6 and a.theta_filter_period == b.theta_filter_period == 2
    u0 = _rich_state(p, W, 7)
    for h in (a, b):
        h.set_state(u0)
        h.step(2)
    np.testing.assert_array_equal(a.get_state(), b.get_state())
    for bad, per in ((-1, 1), (2, 1), (13, 1), (42, 1), (6, -1), (6, 1025)):
        with pytest.raises(teuk.TeukError):  # l_cut <= max(|s|, |m|), 2 (l_cut - 1) >= n_theta, > 41; period
            b.set_theta_filter(bad, per)
        assert b.theta_filter == 6 and b.theta_filter_period == 2
    # the outer-step count restarts from the state's iteration count: from outer step 1 with
    # period 2 the first outer step does not project (bit for bit the unfiltered step)
    e, f = teuk.Teuk(precision=W, theta_filter=6, theta_filter_period=2, **p), teuk.Teuk(precision=W, **p)
    for h in (e, f):
        h.set_state(u0, substeps_done=p["substeps"])
        h.step(1)
    np.testing.assert_array_equal(e.get_state(), f.get_state())
    e.step(1)  # outer step 2 projects
    f.step(1)
    assert np.abs(e.get_state() - f.get_state()).max() > 0
    # resumed in the middle of an outer step, the count goes on as in the uninterrupted run
    whole = teuk.Teuk(precision=W, theta_filter=6, theta_filter_period=2, **p)
    part = teuk.Teuk(precision=W, theta_filter=6, theta_filter_period=2, **p)
    whole.set_state(u0)
    whole.substep(p["substeps"] + 1)
    part.set_state(whole.get_state(), substeps_done=p["substeps"] + 1)
    for h in (whole, part):
        h.substep(3 * p["substeps"])
    np.testing.assert_array_equal(whole.get_state(), part.get_state())
    with pytest.raises(teuk.TeukError):
        teuk.Teuk(precision=W, theta_filter=2, **p)
    with pytest.raises(teuk.TeukError):
        teuk.Teuk(precision=W, own_rows=(0, 20), theta_filter=6, **p)
    c, d = teuk.Teuk(precision=W, **p), teuk.Teuk(precision=W, **p)
    c.set_theta_filter(6)
    c.set_theta_filter(0)
    assert c.theta_filter == 0
    for h in (c, d):
        h.set_state(u0)
        h.step(2)
    np.testing.assert_array_equal(c.get_state(), d.get_state())
    with pytest.raises(teuk.TeukError):
        teuk.Batch([a, b])
    torch = pytest.importorskip("torch")
    pitch = (p["n_theta"] + 15) // 16 * 16
    buf = torch.zeros((4, W, p["n_r"], pitch), dtype=torch.float64, device="cuda")
    rc = teuk.lib().teuk_substep_noalloc(a._h, ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()), 1)
    assert rc == teuk.ERR_INVALID_ARG


@pytest.mark.parametrize("engine", [0, 1])
def test_c3_outer_step_operators_full_size(oracle_mod, engine):
    """c3 at full size in quad-double with its own outer-step operators (r* dissipation
    sigma = 2 and theta filter l_cut = 7, neither in the paper's scheme), tuned launch shape,
    2 k + 3 iterations (three dissipation and filter steps) against a 256-bit oracle window:
    each iteration reaches one row and each dissipation step two."""
    prob = workloads.CONFIGS["c3"]
    assert prob.theta_filter == 7 and prob.ko_sigma == 2.0
    g = teuk.Teuk.from_problem(prob, precision=4)
    if engine:
        g.set_engine(engine)
    g.tune()
    assert g.theta_filter == 7
    nsub = 2 * prob.substeps + 3
    reach = nsub + 2 * 3
    ar, ai = prob.amps
    g.set_initial_pulse(prob.center, prob.width, ar, ai, prob.ell)
    g.substep(nsub)
    g.sync()
    full = g.get_state()
    ic = int(round((prob.center - prob.rstar_min) / prob.dr))
    lo, hi = ic - 12, ic + 12
    wlo, whi = lo - reach - 1, hi + reach + 1
    o = oracle_mod.Oracle(M=prob.M, a=prob.a, s=prob.s, m=prob.m, rstar_min=prob.rstar_min,
                          rstar_max=prob.rstar_max, n_r=prob.n_r, n_theta=prob.n_theta, dt=0.0,
                          substeps=prob.substeps, parity=prob.parity, row_lo=wlo, row_hi=whi, bits=256,
                          ko_sigma=prob.ko_sigma, ko_theta=prob.ko_theta, theta_filter=prob.theta_filter,
                          theta_filter_period=prob.theta_filter_period)
    o.pulse(prob.center, prob.width, ar, ai, prob.ell)
    o.step(nsub)
    err, umax = o.max_rel_err(np.ascontiguousarray(full[:, :, wlo:whi + 1]), lo - wlo, hi - wlo)
    assert umax > 0.05
    assert err < TOL[4], err


def test_c3_bounded_over_its_stated_length():
    """c3 (a = 0.99, s = m = 0, 1024 x 64, 40,000 outer steps of k = 20) in FP64 with its
    outer-step operators stays bounded: the largest |u| of the last 10,000 steps is below that
    of the first 10,000 (the r^-3 amplification of the ingoing pulse near the hole), and the
    run ends without a non-finite value. Without the theta filter it overflows."""
    prob = workloads.CONFIGS["c3"]
    g = teuk.Teuk.from_problem(prob, precision=1)
    ar, ai = prob.amps
    g.set_initial_pulse(prob.center, prob.width, ar, ai, prob.ell)
    peaks = []
    for _ in range(8):
        g.step(prob.steps // 8)
        g.sync()
        peaks.append(float(np.abs(g.get_state()).max()))
    assert all(np.isfinite(peaks))
    assert max(peaks[6:]) < max(peaks[:2]), peaks


@pytest.mark.parametrize("W", [1, 2, 4])
@pytest.mark.parametrize("k,R", [(3, 1), (4, 3), (3, 7)])
def test_fused_iterations_bitwise(W, k, R):
    """Kernel family 4 (one launch per iteration, half rows recomputed per block, the state
    alternating between two buffers) gives the bits of the two-kernel form: odd and even
    iteration counts per outer step (the odd ones end with a copy back), with the observer
    ring, the r* dissipation and the theta filter, through graphs and direct launches."""
    p = small(s=-1, m=2, n_r=45, n_theta=24, substeps=k)
    runs = []
    for fused in (False, True):
        for graphs in (True, False):
            g = teuk.Teuk(precision=W, **p)
            g.set_dissipation(1.0)
            g.set_theta_filter(6, 2)
            if fused:
                g.set_launch_shape(32, R, 10)
                assert g.launch_shape() == {"threads_theta": 32, "rows_per_block": R, "variant": 10}
            g.use_graphs(graphs)
            g.set_observer(5.0, 16)
            g.set_initial_pulse(5.0, 3.0, 0.8, 0.55, 2)
            g.step(3)
            g.substep(2)
            g.step(2)
            g.sync()
            runs.append((g.get_state(), g.read_waveform()))
    for st, wf in runs[1:]:
        np.testing.assert_array_equal(st, runs[0][0])
        np.testing.assert_array_equal(wf, runs[0][1])


def test_fused_iterations_rules():
    """Variant 10 is refused on the integer engine, on slabs and for blocks over 256 threads;
    the tuner may choose it for small grids, with the same bits as the default shape."""
    p = small(s=-2, m=2, n_r=41, n_theta=24, substeps=4)
    g = teuk.Teuk(precision=2, **p)
    g.set_engine(1)
    with pytest.raises(teuk.TeukError):
        g.set_launch_shape(32, 1, 10)
    s = teuk.Teuk(precision=1, own_rows=(0, 20), **p)
    with pytest.raises(teuk.TeukError):
        s.set_launch_shape(32, 1, 10)
    f = teuk.Teuk(precision=1, **p)
    with pytest.raises(teuk.TeukError):
        f.set_launch_shape(128, 3, 10)  # 128 x 4 threads
    prob = workloads.CONFIGS["c1"]
    a = teuk.Teuk.from_problem(prob, precision=1)
    a.tune()
    b = teuk.Teuk.from_problem(prob, precision=1)
    ar, ai = prob.amps
    for h in (a, b):
        h.set_initial_pulse(prob.center, prob.width, ar, ai, prob.ell)
        h.step(5)
    np.testing.assert_array_equal(a.get_state(), b.get_state())
