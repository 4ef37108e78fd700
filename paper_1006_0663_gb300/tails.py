"""Kerr late-time tails (arXiv:1006.0663, Sec. 3.C and Fig. 1).

An observer at fixed r* records the field of an initially pure l' multipole. At late times
each multipole l of the recorded field decays as a power of time, c_l(t) ~ t^-n_l; Fig. 1
shows l = 0..8 from an l' = 0 start, whose tails follow the proposed n = l + l' + 3. The
multipoles of the late field span tens of orders of magnitude, which is why the run needs
quad-double arithmetic.

This module runs such an evolution through the library (all arithmetic on the device, in the
run's precision, including the projection onto the spin-weighted harmonics) and derives the
local power index n_l(t) = -d ln|c_l| / d ln t from the projected series on the host.

    python -m paper_1006_0663_gb300.tails [--precision 4] [--steps N] [--out result.json]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import teuk, workloads


def reflection_free_until(p: workloads.Problem, widths: float = 15.0) -> float:
    """Time after which waves reflected at the r* boundaries can reach the observer.

    Characteristic speeds are +-1 in (t, r*) (|b| <= 1 in Sec. 3.B's system). The initial
    pulse is taken to extend `widths` widths on either side of its centre; its leading part
    reaches a boundary and comes back to the observer no earlier than this."""
    ext = widths * p.width
    outer = (p.rstar_max - (p.center + ext)) + (p.rstar_max - p.rstar_obs)
    inner = ((p.center - ext) - p.rstar_min) + (p.rstar_obs - p.rstar_min)
    return min(outer, inner)


def local_power_index(t: np.ndarray, amp: np.ndarray, stride: int = 1) -> np.ndarray:
    """n(t) = -d ln|c| / d ln t by centred differences over +-stride samples (NaN at the ends
    and where |c| = 0)."""
    t = np.asarray(t, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        la = np.log(np.asarray(amp, dtype=np.float64))
        lt = np.log(t)
        n = np.full(t.shape, np.nan)
        n[stride:-stride] = -(la[2 * stride:] - la[:-2 * stride]) / (lt[2 * stride:] - lt[:-2 * stride])
    n[~np.isfinite(n)] = np.nan
    return n


def velocity_data(p: workloads.Problem, words: int) -> np.ndarray:
    """Generic (not time-symmetric) initial data of an l' = 0 scalar field: Phi = 0 and
    Pi = Phi_t + b Phi_{r*} = A exp(-((r* - c)/w)^2), constant in theta, as word planes
    [4][words][n_r][n_theta] of exact doubles (rows 0 and n_r - 1 zero)."""
    if (p.s, p.m, p.ell) != (0, 0, 0):
        raise ValueError("velocity data are defined here for s = m = l' = 0")
    rs = p.rstar_min + np.arange(p.n_r) * p.dr
    G = np.exp(-((rs - p.center) / p.width) ** 2)
    G[[0, -1]] = 0.0
    ar, ai = p.amps
    planes = np.zeros((4, words, p.n_r, p.n_theta))
    planes[2, 0] = (ar * G)[:, None]
    planes[3, 0] = (ai * G)[:, None]
    return planes


def run(p: workloads.Problem = workloads.TAILS, precision: int | None = None, ell_max: int = 8,
        steps: int | None = None, chunk: int = 500, tune: bool = True, log=None,
        data: str = "pulse", engine: int = 0) -> dict:
    """Evolves p for `steps` outer steps (default p.steps) recording Phi at p.rstar_obs every
    step, then projects the record onto sY_lm, l = max(|m|, |s|) .. ell_max, on the device.
    data: "pulse" (the workloads' time-symmetric Gaussian) or "velocity" (velocity_data)."""
    W = precision or p.words
    steps = p.steps if steps is None else steps
    lo = max(abs(p.m), abs(p.s))
    g = teuk.Teuk.from_problem(p, precision=W)
    try:
        if engine:
            g.set_engine(engine)
        ar, ai = p.amps
        if data == "velocity":
            g.set_initial(velocity_data(p, W))
        else:
            g.set_initial_pulse(p.center, p.width, ar, ai, p.ell)
        g.set_observer(p.rstar_obs, capacity=steps)
        shape = None
        if tune:
            g.tune()
            shape = g.launch_shape()
        t0 = time.perf_counter()
        done = 0
        while done < steps:
            n = min(chunk, steps - done)
            g.step(n)
            g.sync()
            done += n
            if log:
                log(f"  {done}/{steps} outer steps, {time.perf_counter() - t0:.1f} s")
        wall = time.perf_counter() - t0
        c = g.read_multipoles(lo, ell_max)  # [n][n_ell][2][W]
        _, used = g.observe(p.rstar_obs)
    finally:
        g.close()
    t = (np.arange(c.shape[0]) + 1) * p.dt
    amp = np.hypot(c[:, :, 0, 0], c[:, :, 1, 0])  # |c_l(t)| from the leading words
    updates = float(p.n_r) * p.n_theta * p.substeps * steps
    return dict(problem=p, words=W, data=data, ell=list(range(lo, ell_max + 1)), t=t, amp=amp, coeffs=c,
                rstar_obs_used=used, wall_s=wall, updates_per_s=updates / wall, launch_shape=shape,
                reflection_free_until=reflection_free_until(p))


def power_law_fit(t: np.ndarray, amp: np.ndarray, t0: float, t1: float):
    """Least-squares n of |c| ~ t^-n over t0 <= t <= t1 (None without enough positive samples)."""
    sel = (t >= t0) & (t <= t1) & (amp > 0)
    if sel.sum() < 8:
        return None
    slope = np.polyfit(np.log(t[sel]), np.log(amp[sel]), 1)[0]
    return float(-slope)


def summarize(res: dict, times=(300.0, 500.0, 750.0, 1000.0, 1250.0, 1450.0), window: float = 0.05,
              fit=(1000.0, 1450.0)) -> dict:
    """Per multipole: |c_l| and the local power index averaged over ln t in [ln T - window,
    ln T + window] around each requested T (within the recorded, reflection-free span), and
    the power-law index fitted over the late window `fit`."""
    t, amp = res["t"], res["amp"]
    t_ok = min(t[-1], res["reflection_free_until"])
    out = {}
    for k, ell in enumerate(res["ell"]):
        n = local_power_index(t, amp[:, k], stride=8)
        row = {}
        for T in times:
            if T > t_ok:
                continue
            sel = np.abs(np.log(t) - math.log(T)) <= window
            vals = n[sel]
            vals = vals[np.isfinite(vals)]
            i = int(np.argmin(np.abs(t - T)))
            row[f"{T:g}"] = {"abs_c": float(amp[i, k]),
                             "n": float(np.mean(vals)) if vals.size else None}
        row["fit"] = {"t0": fit[0], "t1": min(fit[1], t_ok),
                      "n": power_law_fit(t, amp[:, k], fit[0], min(fit[1], t_ok))}
        out[ell] = row
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2, 4])
    ap.add_argument("--steps", type=int, default=0, help="outer steps (default: the workload's)")
    ap.add_argument("--ell-max", type=int, default=8)
    ap.add_argument("--data", default="pulse", choices=["pulse", "velocity"],
                    help="time-symmetric Gaussian pulse, or Phi = 0 with a Gaussian Pi")
    ap.add_argument("--refine", type=int, default=1,
                    help="divide dr* (and dt = 0.25 dr*) by this factor, same domain and end time")
    ap.add_argument("--substeps", type=int, default=0,
                    help="Lax-Wendroff iterations per outer step (default: the workload's)")
    ap.add_argument("--engine", type=int, default=0, choices=[0, 1],
                    help="multi-word arithmetic: 0 FP64 error-free transforms, 1 integer engine")
    ap.add_argument("--out", default="")
    args = ap.parse_args(argv)
    p = workloads.TAILS
    if args.refine > 1:
        p = p.with_(n_r=(p.n_r - 1) * args.refine + 1, steps=p.steps * args.refine)
    if args.substeps:
        p = p.with_(substeps=args.substeps)
    res = run(p, precision=args.precision or None, ell_max=args.ell_max, steps=args.steps or None,
              log=lambda s: print(s, flush=True), data=args.data, engine=args.engine)
    summ = summarize(res)
    l0 = p.ell
    print(f"tails: {p.name} ({args.data} data, dr*={p.dr:g}, k={p.substeps}), words={res['words']}, "
          f"{res['updates_per_s']:.3e} updates/s, "
          f"{res['wall_s']:.1f} s, reflection-free until t = {res['reflection_free_until']:.0f} M")
    for ell, row in summ.items():
        cells = "  ".join(f"t={T}: |c|={v['abs_c']:.3e} n={v['n'] if v['n'] is None else round(v['n'], 3)}"
                          for T, v in row.items() if T != "fit")
        fn = row["fit"]["n"]
        print(f"  l={ell} (l+l'+3 = {ell + l0 + 3}): fit n={fn if fn is None else round(fn, 3)}  {cells}")
    if args.out:
        stride = max(1, len(res["t"]) // 3000)
        doc = {"workload": p.name, "data": args.data, "engine": args.engine, "dr": p.dr, "substeps": p.substeps,
               "n_r": p.n_r,
               "words": res["words"], "updates_per_s": res["updates_per_s"],
               "wall_s": res["wall_s"], "launch_shape": res["launch_shape"],
               "rstar_obs_used": res["rstar_obs_used"],
               "reflection_free_until": res["reflection_free_until"], "ell": res["ell"],
               "t": res["t"][::stride].tolist(), "abs_c": res["amp"][::stride].T.tolist(),
               "summary": {str(k): v for k, v in summ.items()}}
        with open(args.out, "w") as f:
            json.dump(doc, f)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
