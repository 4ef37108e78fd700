#!/usr/bin/env python
"""Benchmark of the GB300 Lax-Wendroff Teukolsky stepper: grid-point updates per second.

One benchmark step is one outer time step dt = 0.25 dr* of the large double-double workload
(M = 1, a = 0.9, s = -2, m = 2, r* in [-200, 1800] x 16384 nodes, theta x 512 cells), i.e.
81 Lax-Wendroff iterations (Eqs. lw1, lw2 of arXiv:1006.0663) on the integer engine plus the
waveform sample at r* = 1000. A grid-point update is one point advanced by one Lax-Wendroff
iteration. The same workload in FP64 is reported beside it with its own roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own replica of the workload (one problem
is not split across GPUs: replicas only), value = all ranks' updates / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point updates/sec (FP64, dd, qd) & % of FP64/HBM roofline at stated error"
UNIT = "grid-point updates/s"
WORKLOAD = "c5"
# words per real of each workload's main line (c5 is measured in double-double; FP64 beside it)
MAIN_WORDS = {"c5": 2}

# FP64 pipe operations (add, mul and fma count one each) per grid point for one launch of
# each kernel, from the operation list of the scheme in each arithmetic: dd accurate add 14,
# Dot2 term 9, finish 3; qd add 71, by-order dot term 70, renormalisation 38.
# half = Eq. lw1 kernel, full = Eq. lw2 kernel.
OPS_HALF = {1: 52, 2: 502, 4: 3742}
OPS_FULL = {1: 50, 2: 498, 4: 3734}
# Algorithmic DRAM bytes per grid point per launch: state rows read once, half rows written
# once (half kernel) / read once and state written once (full kernel), 8 folded coefficients.
BYTES_HALF = {w: (4 + 4 + 8) * 8 * w for w in (1, 2, 4)}
BYTES_FULL = {w: (4 + 4 + 4 + 8) * 8 * w for w in (1, 2, 4)}
# Integer engine: the tables are nine planes of a 16 kU4-byte mantissa and a 4-byte
# exponent-sign word per point (kU4 = 1 for dd, 2 for qd) instead of eight multi-word reals.
BYTES_HALF_IX = {w: (4 + 4) * 8 * w + 9 * (16 * (w // 2) + 4) for w in (2, 4)}
BYTES_FULL_IX = {w: (4 + 4 + 4) * 8 * w + 9 * (16 * (w // 2) + 4) for w in (2, 4)}
DTYPE = {1: "f64", 2: "f64x2 (double-double)", 4: "f64x4 (quad-double)"}
ENGINE_NAME = {0: "FP64 error-free transforms", 1: "integer engine"}
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of
# the kernel as it stands: (workload, kernel function) -> (bytes, launch shape captured, summary).
TRAFFIC = {("c2", "half_kernel<2, 1>"): (50.456e6 + 0.370e6, "128 x 1", "profiles/step_kernels_dd_c2.txt"),
           ("c2", "full_kernel<2, 1>"): (67.192e6 + 0.623e6, "128 x 1", "profiles/step_kernels_dd_c2.txt"),
           ("c5", "half_kernel<1, 0>"): (830.65e6 + 248.21e6, "64 x 1", "profiles/step_kernels_f64_c5.txt"),
           ("c5", "full_kernel<1, 0>"): (1085.83e6 + 247.52e6, "64 x 1", "profiles/step_kernels_f64_c5.txt"),
           ("c3", "half_kernel<4, 0>"): (25.95e6, "32 x 1", "profiles/step_kernels_qd_c3.txt"),
           ("c3", "full_kernel<4, 0>"): (34.35e6, "32 x 1", "profiles/step_kernels_qd_c3.txt"),
           ("c2", "half_ix_kernel<2, 2>"): (64.06e6 + 3.03e6, "128 x 1", "profiles/step_kernels_ix_dd_c2.txt"),
           ("c2", "full_ix_kernel<2, 2>"): (81.19e6 + 4.94e6, "128 x 1", "profiles/step_kernels_ix_dd_c2.txt"),
           ("c2", "half_ix_kernel<2, 1>"): (64.05e6 + 1.68e6, "128 x 2", "profiles/step_kernels_ix_dd_c2.txt"),
           ("c2", "full_ix_kernel<2, 1>"): (81.10e6 + 2.65e6, "128 x 2", "profiles/step_kernels_ix_dd_c2.txt"),
           ("c3", "half_ix_kernel<4, 1>"): (27.01e6 + 0.12e6, "64 x 4", "profiles/step_kernels_ix_qd_c3.txt"),
           ("c3", "full_ix_kernel<4, 1>"): (34.75e6 + 1.38e6, "64 x 4", "profiles/step_kernels_ix_qd_c3.txt"),
           # captured on the 2048-node case of c5, scaled to a full launch by the points
           ("c5", "full_ix_kernel<2, 1>"): (3.00e9, "256 x 1", "profiles/step_kernels_ix_dd_c5.txt")}


# Integer engine: algorithmic work per grid point of one launch (half or full kernel), in
# 32-bit limb multiply-add pairs (mad.lo / madc.hi with the carry, the product window's unit).
# Each of the two components of a point forms 11 products (Phi row: the table term and the
# h/4 or h/2 term, the 1/2 and 1 terms being shifts; Pi row: nine table terms), 10 partial
# products each in double-double (4 x 4 limbs, columns 3..6) and 36 in quad-double (8 x 8
# limbs, columns 7..14), and the theta stencil's 11 integer multiply-adds (6 for D2, 5 for D1)
# on a row of 6 (dd) / 10 (qd) limbs: 22 x 10 + 22 x 6 = 352 and 22 x 36 + 22 x 10 = 1012.
IX_PAIRS = {2: 22 * 10 + 22 * 6, 4: 22 * 36 + 22 * 10}


def kernel_name(dom, W, shape, engine=0):
    """The step kernel a launch shape selects (teuk_launch_shape variants 0..8)."""
    v = shape["variant"]
    if engine == 1:
        return f"{dom}_ix_kernel<{W}, {v % 3}>"
    fam = "" if v < 3 else ("seg_" if v < 6 else "bal_")
    return f"{dom}_{fam}kernel<{W}, {v % 3}>"


TOL = {1: 1e-12, 2: 1e-26, 4: 1e-55}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-variants", action="store_true", help="skip the FP64 / qd side figures")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-member batched workload")
    ap.add_argument("--workload", default=WORKLOAD, choices=["c1", "c2", "c3", "c5", "tails"],
                    help="workload of the main line (default c5 in double-double, the roofline "
                         "configuration)")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2, 4],
                    help="words per real (0: the workload's own precision)")
    ap.add_argument("--engine", type=int, default=-1, choices=[-1, 0, 1],
                    help="multi-word arithmetic: 0 FP64 error-free transforms, 1 integer engine "
                         "(default -1: the integer engine for double-double and quad-double)")
    ap.add_argument("--shape", default="",
                    help="pin the step kernels' launch shape 'threads_theta,rows,variant' "
                         "instead of autotuning (profiling)")
    ap.add_argument("--digits", action="store_true",
                    help="print the cost-per-digit table (errors vs the oracle and each other)")
    ap.add_argument("--digits-workloads", default="c1,c2,c3",
                    help="workloads of the cost-per-digit table (c5: FP64 against double-double)")
    ap.add_argument("--n-r", type=int, default=0,
                    help="profiling: the workload with this many r* nodes over the same r* range "
                         "(a smaller case of the same kernels)")
    ap.add_argument("--c4-steps", type=int, default=4,
                    help="outer steps of the 64-member batch timed in one cooperative launch")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------
def start_clock_sampler():
    path = os.path.join(tempfile.gettempdir(), f"teuk_clocks_{os.getpid()}.csv")
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                              "-lms", "200"], stdout=f, stderr=subprocess.DEVNULL)
        return p, f, path
    except Exception:
        return None, None, path


def stop_clock_sampler(p, f, path, device_index):
    if p is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    f.close()
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or parts[0] != str(device_index):
            continue
        try:
            sm.append(float(parts[1]))
            smax = float(parts[2])
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    os.unlink(path)
    sm.sort()
    med = sm[len(sm) // 2] if sm else None
    return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
def run_workload(prob, words, steps, warmup, torch, teuk, flush, with_timing=True, shape="", engine=0):
    """Device-resident timing of `steps` outer steps; returns a dict of measurements."""
    g = teuk.Teuk.from_problem(prob, precision=words)
    if engine:
        g.set_engine(engine)
    ar, ai = prob.amps
    g.set_initial_pulse(prob.center, prob.width, ar, ai, prob.ell)
    g.set_observer(prob.rstar_obs, capacity=steps + warmup + 1)
    if shape:
        tx, ty, v = (int(x) for x in shape.split(","))
        g.set_launch_shape(tx, ty, v)
    else:
        g.tune()  # launch-shape autotuner, untimed set-up
    rows_per_block = g.launch_shape()
    for _ in range(warmup):
        g.step(1)
    g.sync()
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    launches0 = g.kernel_launches
    if with_timing:
        g.timing(True)
    torch.cuda.synchronize()
    for t in range(steps):
        flush.zero_()  # L2 flush between timed steps (outside the timed interval)
        evs[t][0].record(stream)
        g.step(1)
        evs[t][1].record(stream)
    torch.cuda.synchronize()
    g.sync()
    ms = [a.elapsed_time(b) for a, b in evs]
    kt = g.kernel_times() if with_timing else (0, 0, 0, 0)
    out = dict(ms_total=sum(ms), ms=ms, launches=g.kernel_launches - launches0, kernel_times=kt,
               points=prob.n_r * prob.n_theta, substeps=prob.substeps,
               rows_per_block=rows_per_block)
    wf = g.read_waveform()
    out["waveform_samples"] = int(wf.shape[0])
    g.close()
    return out


def stated_error(prob, words, teuk, nsub=12, engine=0):
    """Error of this workload's GPU state against the 256-bit oracle after nsub Lax-Wendroff
    iterations, on a window of rows around the pulse, where the window
    interior is exact (domain of dependence)."""
    import oracle
    oracle.build()
    g = teuk.Teuk.from_problem(prob, precision=words)
    if engine:
        g.set_engine(engine)
    ar, ai = prob.amps
    g.set_initial_pulse(prob.center, prob.width, ar, ai, prob.ell)
    g.substep(nsub)
    g.sync()
    full = g.get_state()
    g.close()
    ic = int(round((prob.center - prob.rstar_min) / prob.dr))
    lo, hi = ic - 12, ic + 12
    wlo, whi = max(0, lo - nsub - 1), min(prob.n_r - 1, hi + nsub + 1)
    bits = 256
    o = oracle.Oracle(M=prob.M, a=prob.a, s=prob.s, m=prob.m, rstar_min=prob.rstar_min,
                      rstar_max=prob.rstar_max, n_r=prob.n_r, n_theta=prob.n_theta, dt=0.0,
                      substeps=prob.substeps, parity=prob.parity, row_lo=wlo, row_hi=whi, bits=bits,
                      ko_sigma=prob.ko_sigma, ko_theta=prob.ko_theta,
                      theta_filter=prob.theta_filter,
                      theta_filter_period=prob.theta_filter_period)
    o.pulse(prob.center, prob.width, ar, ai, prob.ell)
    o.step(nsub)
    err, _ = o.max_rel_err(full[:, :, wlo:whi + 1].copy(), lo - wlo, hi - wlo)
    return {"max_rel_err": err, "oracle_bits": bits, "iterations": nsub,
            "rows": f"{lo}..{hi} of {prob.n_r}", "tolerance": TOL[words], "engine": engine}


def run_batch1(prob, words, steps, torch, teuk):
    """One problem through the cooperative batched kernel (all iterations of `steps` outer
    steps in one launch): the launch-bound regime of small grids."""
    g = teuk.Teuk.from_problem(prob, precision=words)
    ar, ai = prob.amps
    g.set_initial_pulse(prob.center, prob.width, ar, ai, prob.ell)
    b = teuk.Batch([g])
    b.step(1)
    b.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(steps)
    b.sync()
    dt = time.perf_counter() - t0
    b.close()
    g.close()
    return prob.n_r * prob.n_theta * prob.substeps * steps / dt, dt / steps * 1e3


def run_c4(torch, teuk, workloads, engine=1, steps=4):
    """The 64-member double-double batch: `steps` outer steps in one cooperative launch against
    the same members stepped one at a time (CUDA graphs on) over the same window, CUDA events
    on the shared stream, equal arithmetic (bit-identical), on the given multi-word engine."""
    members = []
    for i in range(workloads.BATCH_SIZE):
        p = workloads.batch_member(i)
        g = teuk.Teuk.from_problem(p)
        if engine:
            g.set_engine(engine)
        ar, ai = p.amps
        g.set_initial_pulse(p.center, p.width, ar, ai, p.ell)
        g.set_observer(p.rstar_obs, capacity=2 * steps + 4)
        members.append(g)
    pts = sum(g.n_r * g.n_theta * g.substeps for g in members)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for g in members:
        g.step(1)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for g in members:
        g.step(steps)
    ev[1].record(stream)
    torch.cuda.synchronize()
    b = teuk.Batch(members)
    b.step(1)
    b.sync()
    launches0 = b.info()["launches"]
    ev[2].record(stream)
    b.step(steps)
    ev[3].record(stream)
    b.sync()
    torch.cuda.synchronize()
    t_seq = ev[0].elapsed_time(ev[1]) * 1e-3
    t_bat = ev[2].elapsed_time(ev[3]) * 1e-3
    info = b.info()
    b.close()
    for g in members:
        g.close()
    return {"workload": "c4: 64 double-double members, n_r U[512,4096], n_theta {32..256}, "
                        "m in [-4,4], s in {0,-1,-2}, a U[0,0.99], substeps 1..454 (seeds 1000+i)",
            "outer_steps_timed": steps, "cooperative_launches": info["launches"] - launches0,
            "updates_per_outer_step": pts,
            "batched_updates_per_s": pts * steps / t_bat, "one_at_a_time_updates_per_s": pts * steps / t_seq,
            "speedup": t_seq / t_bat, "batched_ms_per_step": t_bat * 1e3 / steps,
            "one_at_a_time_ms_per_step": t_seq * 1e3 / steps, "grid_blocks": info["grid"],
            "timing": "CUDA events on the shared stream", "arithmetic": ENGINE_NAME[engine]}


def run_e2e(prob, words, steps, torch, teuk, flush, engine=0):
    """Through the public API with host buffers: per step H2D of the state from pinned host
    memory, one outer step, D2H of the observer row. As in the device-timed loop, the 256 MiB
    L2 flush runs between steps outside the timed interval."""
    import numpy as np
    g = teuk.Teuk.from_problem(prob, precision=words)
    if engine:
        g.set_engine(engine)
    ar, ai = prob.amps
    g.set_initial_pulse(prob.center, prob.width, ar, ai, prob.ell)
    g.tune()
    state = g.get_state()
    pinned = torch.empty(state.shape, dtype=torch.float64, pin_memory=True)
    host = pinned.numpy()
    host[...] = state
    g.set_state(host)  # warm-up: the first copy from a newly pinned buffer is slow
    g.step(1)
    g.observe(prob.rstar_obs)
    torch.cuda.synchronize()
    total = 0.0
    for t in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # the iteration count continues as in one run (outer-step operators with a period,
        # such as c3's theta filter, then run where they would in the device-timed loop)
        g.set_state(host, substeps_done=(t + 1) * prob.substeps)
        g.step(1)
        obs, _ = g.observe(prob.rstar_obs)
        total += time.perf_counter() - t0
    g.close()
    upd = prob.n_r * prob.n_theta * prob.substeps * steps
    return dict(value=upd / total, unit=UNIT, h2d_bytes_per_step=int(state.nbytes),
                d2h_bytes_per_step=int(obs.nbytes),
                l2="flushed between steps outside the timed interval, as for value")


def run_design_a(prob, words, iters, torch, teuk, engine=0):
    """The data flow of the paper's first CUDA design (Sec. 4) on this machine's CPU-GPU link:
    the host keeps the state and every Lax-Wendroff iteration copies it to the device and
    back (page-locked host memory, one cudaMemcpy2DAsync each way, the host waits), with all
    arithmetic on the device. Against the same iterations with the state resident in HBM."""
    g = teuk.Teuk.from_problem(prob, precision=words)
    if engine:
        g.set_engine(engine)
    ar, ai = prob.amps
    g.set_initial_pulse(prob.center, prob.width, ar, ai, prob.ell)
    g.tune()
    state = g.get_state()
    pinned = torch.empty(state.shape, dtype=torch.float64, pin_memory=True)
    host = pinned.numpy()
    host[...] = state
    g.substep_host_state(host, 2)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.substep_host_state(host, iters)
    t_a = time.perf_counter() - t0
    g.set_state(host)
    g.substep(2)
    g.sync()
    t0 = time.perf_counter()
    g.substep(iters)
    g.sync()
    t_r = time.perf_counter() - t0
    g.close()
    upd = prob.n_r * prob.n_theta * iters
    link = 2 * state.nbytes
    return {"updates_per_s": upd / t_a, "resident_updates_per_s": upd / t_r, "slowdown": t_a / t_r,
            "iterations": iters, "link_bytes_per_iteration": link,
            "link_gbps_effective": link * iters / (t_a - t_r) / 1e9 if t_a > t_r else None}


def measured_hbm_peak():
    """HBM copy bandwidth of the GB300s (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


def roofline_for(res, prob, W, engine, clocks, sms, fp64_probe, int_probe, workload):
    """Roofline of the dominant step kernel of a run (live CUDA-event launch durations).

    FP64 error-free-transform kernels (and FP64): bound by the FP64 pipe, 2 operations per SM
    per cycle (ncu sm__sass_thread_inst_executed_op_dfma_pred_on.sum.peak_sustained = 304 per
    cycle for 152 SMs) at the SM clock sampled during the timed region, counted from the
    scheme's operation list (OPS_HALF / OPS_FULL). Integer-engine kernels: bound by the
    integer multiply-add pipe, counted as the product windows' and stencils' 32-bit limb
    multiply-add pairs the scheme needs per point (IX_PAIRS), against the measured throughput
    of the engine's own product window on every SM (teuk_int_peak). The HBM fraction of the
    kernel's algorithmic bytes is reported beside either."""
    ms_h, ms_f, n_h, n_f = res["kernel_times"]
    pts_h = (prob.n_r - 1) * prob.n_theta
    pts_f = (prob.n_r - 2) * prob.n_theta
    avg_h = ms_h / max(n_h, 1)
    avg_f = ms_f / max(n_f, 1)
    # the library times a sample of the launches inside the timed steps (with graph replay the
    # last iteration of the outer step); both kernels launch once per iteration
    dom = "half" if avg_h >= avg_f else "full"
    avg = avg_h if dom == "half" else avg_f
    pts = pts_h if dom == "half" else pts_f
    mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    kname = kernel_name(dom, W, res["rows_per_block"], engine)
    tr = TRAFFIC.get((workload, kname))
    fp64_peak = 2.0 * sms * mhz * 1e6
    fp64_ops = (OPS_HALF[W] if dom == "half" else OPS_FULL[W]) * pts / (avg * 1e-3)
    ix = engine == 1 and W > 1
    bpp = ((BYTES_HALF_IX if ix else BYTES_HALF)[W] if dom == "half" else (BYTES_FULL_IX if ix else BYTES_FULL)[W])
    hbm_peak, hbm_src = measured_hbm_peak()
    hbm = bpp * pts / (avg * 1e-3) / 1e9
    if ix:
        ops_pt = IX_PAIRS[W]
        peak = int_probe
        peak_source = ("measured product-window throughput of this GPU (teuk_int_peak: independent "
                       "windows on every SM, 10 partial products each)")
        op_unit = "32-bit limb multiply-add pairs (product windows and theta stencils) per point"
        unit = "T pairs/s"
    else:
        ops_pt = OPS_HALF[W] if dom == "half" else OPS_FULL[W]
        peak = fp64_peak
        peak_source = f"2 FP64 ops/SM/cycle x {sms} SMs x {mhz:.0f} MHz (SM clock sampled during the timed region)"
        op_unit = "FP64 pipe operations (add, mul, fma count one each)"
        unit = "Tops/s"
    achieved = ops_pt * pts / (avg * 1e-3)
    out = {
        "bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": unit,
        "frac": achieved / peak, "traffic": tr[0] if tr else None,
        "traffic_source": f"{tr[2]} (launch shape {tr[1]})" if tr else None,
        "kernel": kname, "avg_launch_ms": avg, "launch_shape": res["rows_per_block"],
        "points_per_launch": pts, "ops_per_point": ops_pt, "peak_source": peak_source, "op_unit": op_unit,
        "hbm": {"achieved_gbs": hbm, "peak_gbs": hbm_peak, "frac": hbm / hbm_peak,
                "bytes_per_point": bpp, "peak_source": hbm_src},
        "fma_chain_probe_tops": fp64_probe / 1e12,
        "fraction_of_step_in_dominant_kernel": avg * res["launches"] / 2 / max(res["ms_total"], 1e-9),
    }
    if ix:
        out["fp64_equivalent"] = {
            "method_fp64_ops_per_point": OPS_HALF[W] if dom == "half" else OPS_FULL[W],
            "x_fp64_pipe_peak": fp64_ops / fp64_peak,
            "note": "the same step in FP64 error-free transforms would need this multiple of the FP64 pipe"}
    return out


def cpu_model():
    """The host CPU's model name (lscpu / /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def cpu_baseline_others(prob, seconds_target=4.0):
    """Bounded samples of the same oracle window on one core (256-bit) and of the FP64 oracle
    on all cores, beside the main baseline (context for the cost of the arithmetic)."""
    import oracle
    n_all = oracle.max_threads()
    oracle.set_threads(1)
    one = cpu_baseline(prob, 2, seconds_target)
    oracle.set_threads(n_all)
    f64 = cpu_baseline(prob, 1, seconds_target)
    return {"bits256_one_core": {"value": one["value"], "cores": 1, "sample": one["sample"]},
            "fp64_all_cores": {"value": f64["value"], "cores": f64["cores"], "sample": f64["sample"]}}


def cpu_baseline(prob, words, seconds_target=15.0):
    """The oracle (256-bit MPFR for dd/qd workloads, FP64 for FP64) on all host cores, on a
    window of rows of the same workload for a bounded number of iterations."""
    import oracle
    oracle.build()
    bits = 53 if words == 1 else 256
    rows = 24 if words > 1 else 512
    ic = int(round((prob.center - prob.rstar_min) / prob.dr))
    lo = max(0, ic - rows // 2)
    o = oracle.Oracle(M=prob.M, a=prob.a, s=prob.s, m=prob.m, rstar_min=prob.rstar_min,
                      rstar_max=prob.rstar_max, n_r=prob.n_r, n_theta=prob.n_theta, dt=0.0,
                      substeps=prob.substeps, parity=prob.parity, row_lo=lo,
                      row_hi=min(prob.n_r - 1, lo + rows - 1), bits=bits, ko_sigma=prob.ko_sigma,
                      ko_theta=prob.ko_theta, theta_filter=prob.theta_filter,
                      theta_filter_period=prob.theta_filter_period)
    ar, ai = prob.amps
    o.pulse(prob.center, prob.width, ar, ai, prob.ell)
    done, t0 = 0, time.perf_counter()
    n = 1
    while time.perf_counter() - t0 < seconds_target:
        o.step(n)
        done += n
        n = min(n * 2, 64)
    dt = time.perf_counter() - t0
    upd = o.nrow * prob.n_theta * done
    return dict(value=upd / dt, unit=UNIT, cores=oracle.max_threads(), kind="oracle",
                sample=f"{o.nrow} r* rows x {prob.n_theta} theta of {prob.name}, {done} "
                       f"Lax-Wendroff iterations, {bits}-bit oracle, {dt:.1f} s")


# ---------------------------------------------------------------------------------------------
def reference_arm(args):
    from paper_1006_0663_gb300 import workloads
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    prob = workloads.CONFIGS[WORKLOAD]
    W = MAIN_WORDS.get(WORKLOAD, prob.words)
    per_step_s = 4.0
    # warm-up and K timed steps, each a bounded sample of the workload
    for _ in range(args.warmup):
        cpu_baseline(prob, W, seconds_target=0.5)
    vals = [cpu_baseline(prob, W, seconds_target=per_step_s) for _ in range(args.steps)]
    tot_upd = sum(v["value"] * per_step_s for v in vals)
    value = sum(v["value"] for v in vals) / len(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[W], "data": "synthetic",
        "config": {"workload": describe(prob, W)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                         "sample": vals[0]["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "note": f"{tot_upd:.3g} updates timed",
    }
    print(json.dumps(line))
    return 0


def aggregate_ranks(t_local_ms, updates_per_rank, world, dist, torch, device):
    """Whole-job throughput of independent replicas: every rank advances its own copy of the
    workload; the job time is the slowest rank's, value = all ranks' updates / that time."""
    if world > 1:
        t = torch.tensor([t_local_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
        dist.barrier()
    else:
        t_max = t_local_ms
    return t_max, world * updates_per_rank / (t_max * 1e-3)


def describe(prob, words=None):
    w = words or prob.words
    diss = ""
    if prob.ko_sigma or prob.ko_theta:
        diss = f", dissipation r* {prob.ko_sigma} theta {prob.ko_theta} (not in the paper)"
    if prob.theta_filter:
        diss += f", theta filter l < {prob.theta_filter} (not in the paper)"
    return (f"{prob.name}: {DTYPE[w]}, M={prob.M}, a={prob.a}, s={prob.s}, m={prob.m}, "
            f"r* in [{prob.rstar_min}, {prob.rstar_max}] x {prob.n_r} nodes, theta x {prob.n_theta} "
            f"cells, {prob.theta_order}th-order theta, dt=0.25 dr* with {prob.substeps} Lax-Wendroff "
            f"iterations per step, Gaussian pulse (center {prob.center}, width {prob.width}, seed "
            f"{prob.seed}), waveform at r*={prob.rstar_obs} every step{diss}")


def word_diff(a, b):
    """(sum of a's words) - (sum of b's words), summed from the smallest words up."""
    import numpy as np
    diff = np.zeros(a.shape[:1] + a.shape[2:])
    for k in reversed(range(max(a.shape[1], b.shape[1]))):
        x = a[:, k] if k < a.shape[1] else 0.0
        y = b[:, k] if k < b.shape[1] else 0.0
        diff = diff + (x - y)
    return diff


# Outer steps of the cost-per-digit runs: the stated length for c1 and c3 (bounded with their
# outer-step operators); for c2 a prefix (t = 244 M) well before the pulse, reflected by the
# zero-field row at r* = 400, returns to the hole (t ~ 760 M): from then on the s = -2 field of
# the problem as posed grows (so it does at a = 0 and on a twice finer r* grid, at a rate set
# by the boundary's distance), and a 40,000-step run in all three arithmetics would cost
# about 40 GPU-minutes.
DIGITS_STEPS = {"c1": 1000, "c2": 4000, "c3": 40000, "c5": 2000}
# Reference arithmetic of the long runs: quad-double, except c5, whose 2000-step quad-double run
# would take ~45 GPU-minutes; there double-double (within 1e-26 of the 256-bit oracle on every
# check) is the reference for FP64 and no dd figure is stated.
DIGITS_REF = {"c5": 2}
REF_NAME = {2: "dd", 4: "qd"}
# outer steps of the 256-bit check of each arithmetic (one for c5: its window is 512 columns wide)
REF_CHECK_STEPS = {"c5": 1}


def digits_table(names=("c1", "c2", "c3")):
    """Errors of FP64 / double-double / quad-double runs and their cost, on c1, c2 and c3.

    For each workload: the FP64, double-double and quad-double runs of DIGITS_STEPS outer steps
    on the GPU (dd and qd on the integer engine); quad-double is the reference for the other
    two (max over the grid of |u - u_qd| / max |u_qd|). The reference itself: a 3-outer-step
    prefix of each arithmetic against the 256-bit oracle (c1 whole grid; c2 and c3 a window
    of rows around the pulse). Cost: ns per update of each arithmetic on the workload's grid
    (CUDA events, tuned launch shape)."""
    import numpy as np
    import torch

    import oracle
    from paper_1006_0663_gb300 import teuk, workloads

    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {}
    for name in names:
        prob = workloads.CONFIGS[name]
        ref_w = DIGITS_REF.get(name, 4)
        arith = [w for w in (1, 2, 4) if w <= ref_w]
        ar, ai = prob.amps
        res = {"outer_steps": DIGITS_STEPS[name], "stated_steps": prob.steps, "reference_check": {},
               "run": {}, "cost": {}}
        # 256-bit check of a short prefix in every arithmetic
        n_check = REF_CHECK_STEPS.get(name, 3)
        nsub = n_check * prob.substeps
        if name == "c1":
            lo, hi, wlo, whi = 0, prob.n_r - 1, 0, prob.n_r - 1
        else:
            ic = int(round((prob.center - prob.rstar_min) / prob.dr))
            lo, hi = ic - 12, ic + 12
            wlo, whi = lo - nsub - 3, hi + nsub + 3
        o = oracle.Oracle(M=prob.M, a=prob.a, s=prob.s, m=prob.m, rstar_min=prob.rstar_min,
                          rstar_max=prob.rstar_max, n_r=prob.n_r, n_theta=prob.n_theta, dt=0.0,
                          substeps=prob.substeps, parity=prob.parity, row_lo=wlo, row_hi=whi, bits=256,
                          ko_sigma=prob.ko_sigma, ko_theta=prob.ko_theta,
                          theta_filter=prob.theta_filter,
                          theta_filter_period=prob.theta_filter_period)
        o.pulse(prob.center, prob.width, ar, ai, prob.ell)
        o.step(nsub)
        states, cost = {}, {}
        for W in arith:
            g = teuk.Teuk.from_problem(prob, precision=W)
            if W > 1:
                g.set_engine(1)
            g.tune()
            g.set_initial_pulse(prob.center, prob.width, ar, ai, prob.ell)
            g.step(n_check)
            g.sync()
            st = g.get_state()
            err, _ = o.max_rel_err(np.ascontiguousarray(st[:, :, wlo:whi + 1]), lo - wlo, hi - wlo)
            res["reference_check"][DTYPE[W]] = {"outer_steps": n_check, "max_rel_err_vs_256bit": err,
                                                "rows": f"{lo}..{hi}"}
            g.set_initial_pulse(prob.center, prob.width, ar, ai, prob.ell)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.step(DIGITS_STEPS[name])
            e1.record(stream)
            g.sync()
            ms = e0.elapsed_time(e1)
            states[W] = g.get_state()
            cost[W] = ms * 1e6 / (prob.points * prob.substeps * DIGITS_STEPS[name])
            g.close()
        ref = states[ref_w]
        scale = np.abs(ref[:, 0]).max()
        for W in [w for w in arith if w < ref_w]:
            err = float(np.abs(word_diff(states[W], ref)).max() / scale)
            d = -np.log10(err) if err > 0 else None
            res["run"][DTYPE[W]] = {f"max_rel_err_vs_{REF_NAME[ref_w]}": err, "digits": d,
                                    "ns_per_update": cost[W], "ns_per_update_per_digit": cost[W] / d if d else None}
        res["run"][DTYPE[ref_w]] = {"max_abs_field": float(scale), "ns_per_update": cost[ref_w], "reference": True}
        out[name] = res
    print(json.dumps({"digits_table": out}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.digits:
        return digits_table(tuple(args.digits_workloads.split(",")))
    import torch
    import torch.distributed as dist

    from paper_1006_0663_gb300 import teuk, workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prob = workloads.CONFIGS[args.workload]
    if args.n_r:
        prob = prob.with_(n_r=args.n_r)
        args.no_variants = args.no_batch = True
    W = args.precision or MAIN_WORDS.get(args.workload, prob.words)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)  # the library handles are created on this stream

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = start_clock_sampler()
    engine = (1 if W > 1 else 0) if args.engine < 0 else (args.engine if W > 1 else 0)
    res = run_workload(prob, W, args.steps, args.warmup, torch, teuk, flush, shape=args.shape, engine=engine)
    clocks = stop_clock_sampler(*sampler, device_index=local)
    torch.cuda.synchronize()
    updates_per_rank = res["points"] * res["substeps"] * args.steps
    t_max, value = aggregate_ranks(res["ms_total"], updates_per_rank, world, dist, torch, "cuda")

    out = None
    if rank == 0:
        describe_w = describe(prob, W)
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        fp64_probe, int_probe = teuk.fp64_peak(), teuk.int_peak()
        roofline = roofline_for(res, prob, W, engine, clocks, sms, fp64_probe, int_probe, args.workload)
        e2e = run_e2e(prob, W, max(3, args.steps // 4), torch, teuk, flush, engine)
        if args.workload != WORKLOAD or W != MAIN_WORDS.get(WORKLOAD):
            args.no_variants = args.no_batch = True
        variants = {}
        if not args.no_variants:
            # the same workload in FP64: its own roofline, end-to-end figure and oracle error
            r = run_workload(prob, 1, 3, 1, torch, teuk, flush)
            variants[f"{prob.name}/f64"] = {
                "updates_per_s": r["points"] * r["substeps"] * 3 / (r["ms_total"] * 1e-3),
                "ms_per_step": r["ms_total"] / 3, "launch": "CUDA graph per outer step",
                "roofline": roofline_for(r, prob, 1, 0, clocks, sms, fp64_probe, int_probe, args.workload),
                "e2e": run_e2e(prob, 1, 3, torch, teuk, flush, 0),
                "error_vs_oracle": None if args.no_cpu else stated_error(prob, 1, teuk)}
            # the main workload on the other multi-word engine
            other = 1 - engine
            r0 = run_workload(prob, W, 2, 1, torch, teuk, flush, engine=other)
            variants[f"{prob.name}/{DTYPE[W].split(' ')[0]} {ENGINE_NAME[other]}"] = {
                "updates_per_s": r0["points"] * r0["substeps"] * 2 / (r0["ms_total"] * 1e-3),
                "roofline": roofline_for(r0, prob, W, other, clocks, sms, fp64_probe, int_probe, args.workload)}
            for name, w, nst in (("c1", 1, 20), ("c2", 2, 4), ("c3", 4, 2)):
                p = workloads.CONFIGS[name]
                r = run_workload(p, w, nst, 1, torch, teuk, flush, engine=1 if w > 1 else 0)
                entry = {"updates_per_s": p.n_r * p.n_theta * p.substeps * nst / (r["ms_total"] * 1e-3),
                         "ms_per_step": r["ms_total"] / nst, "launch": "CUDA graph per outer step"}
                if w > 1:
                    entry["roofline"] = roofline_for(r, p, w, 1, clocks, sms, fp64_probe, int_probe, name)
                variants[f"{name}/{DTYPE[w].split(' ')[0]}"] = entry
            c1_plain = workloads.CONFIGS["c1"].with_(ko_sigma=0.0)  # batches take no dissipation
            ups, msps = run_batch1(c1_plain, 1, 20, torch, teuk)
            variants["c1/f64 batched kernel, no dissipation"] = {
                "updates_per_s": ups, "ms_per_step": msps, "launch": "one cooperative launch, 20 steps"}
            r = run_workload(c1_plain, 1, 20, 1, torch, teuk, flush, with_timing=False)
            variants["c1/f64 no dissipation"] = {
                "updates_per_s": c1_plain.points * c1_plain.substeps * 20 / (r["ms_total"] * 1e-3),
                "ms_per_step": r["ms_total"] / 20, "launch_shape": r["rows_per_block"],
                "launch": "tuned: CUDA graph per outer step or persistent launches (variant 9)"}
            c2 = workloads.CONFIGS["c2"]
            p2 = c2.with_(theta_order=2)
            r = run_workload(p2, 2, 2, 1, torch, teuk, flush, with_timing=False, engine=1)
            variants["c2/f64x2 2nd-order theta"] = {
                "updates_per_s": p2.points * p2.substeps * 2 / (r["ms_total"] * 1e-3),
                "ms_per_step": r["ms_total"] / 2, "launch": "CUDA graph per outer step"}
            variants["design_a_host_state"] = run_design_a(c2, 2, 2 * c2.substeps, torch, teuk, 1)
            variants["design_a_host_state"]["workload"] = "c2, double-double, integer engine"
        batched = None
        if not args.no_batch:
            batched = run_c4(torch, teuk, workloads, engine=1, steps=args.c4_steps)
            batched["other_engine"] = run_c4(torch, teuk, workloads, engine=0, steps=1)
        cpu = None if args.no_cpu else cpu_baseline(prob, W)
        if cpu is not None:
            cpu["cpu_model"] = cpu_model()
            if W > 1:
                cpu["other_runs"] = cpu_baseline_others(prob)
        parity = None if args.no_cpu else stated_error(prob, W, teuk, engine=engine)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[W], "data": "synthetic",
            "config": {"workload": describe_w,
                       "arithmetic": ENGINE_NAME[engine] if W > 1 else "FP64",
                       "l2": "256 MiB buffer written between timed steps (outside the timed "
                             "interval); the state and tables exceed L2",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": res["launches"],
            "clocks": clocks,
            "per_precision": variants,
            "batched": batched,
            "tolerance_vs_256bit_oracle": TOL[W],
            "error_vs_oracle": parity,
        }
        print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
