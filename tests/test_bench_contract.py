"""The benchmark's reference arm (the CPU oracle) prints one JSON line with the contract keys;
runs on the host cores only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"]


def _bench_module():
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_tables", os.path.join(root, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod, root


def test_roofline_tables_match_their_profiles():
    """Every traffic entry of bench.py names a committed profile summary that covers its kernel
    function and prints its numbers; the integer-engine kernels the autotuner picks for the
    dd and qd workloads (both dd shapes at c2, qd at c3) have one."""
    mod, root = _bench_module()
    def mentions(text, kname):  # names are printed with or without the space after the comma
        return kname.replace(" ", "") in text.replace(" ", "")

    for (workload, kname), (traffic, shape, src) in mod.TRAFFIC.items():
        text = open(os.path.join(root, src)).read()
        assert mentions(text, kname), (kname, src)
        assert workload in text, (workload, src)
    for kname, workload in [("half_ix_kernel<2, 1>", "c2"), ("full_ix_kernel<2, 1>", "c2"),
                            ("half_ix_kernel<2, 2>", "c2"), ("full_ix_kernel<2, 2>", "c2"),
                            ("half_ix_kernel<4, 1>", "c3"), ("full_ix_kernel<4, 1>", "c3")]:
        assert (workload, kname) in mod.TRAFFIC, kname
    # the engine's traffic figures are the ones printed in the summaries (MB, read + write)
    for (workload, kname), (traffic, shape, src) in mod.TRAFFIC.items():
        if "_ix_kernel" not in kname or workload == "c5":  # c5: scaled from a smaller case
            continue
        text = open(os.path.join(root, src)).read()
        found = False
        for line in text.splitlines():
            if "DRAM read + write" in line:
                nums = [float(x) for x in line.replace("MB", " ").replace("+", " ").split() if _isnum(x)]
                pairs = [nums[k] + nums[k + 1] for k in range(0, len(nums) - 1, 2)]
                found |= any(abs(p * 1e6 - traffic) < 0.02e6 for p in pairs)
        assert found, (kname, traffic, src)


def test_c5_traffic_scaled_from_its_capture():
    """The c5 engine kernel's traffic is the smaller case's bytes per point (375.1 MB over
    2046 x 512 points) times a full launch's points."""
    mod, root = _bench_module()
    text = open(os.path.join(root, "profiles", "step_kernels_ix_dd_c5.txt")).read()
    assert "375.1 MB" in text and "3.00 GB" in text
    per_point = 375.1e6 / (2046 * 512)
    assert abs(mod.TRAFFIC[("c5", "full_ix_kernel<2, 1>")][0] - per_point * 16382 * 512) < 0.01e9


def _isnum(x):
    try:
        float(x)
        return True
    except ValueError:
        return False


def test_engine_work_count_from_the_formula():
    """The integer engine's algorithmic work per point and launch: two components x (11
    products x the product window's partial products + 11 stencil multiply-adds x the row's
    limbs): double-double 4 x 4-limb windows keep columns 3..6 (10 partial products) on 6-limb
    rows, quad-double 8 x 8-limb windows keep columns 7..14 (36) on 10-limb rows."""
    mod, _ = _bench_module()
    def window(limbs, first_col):
        return sum(1 for i in range(limbs) for j in range(limbs) if i + j >= first_col)
    assert window(4, 3) == 10 and window(8, 7) == 36
    assert mod.IX_PAIRS[2] == 2 * (11 * window(4, 3) + 11 * 6) == 352
    assert mod.IX_PAIRS[4] == 2 * (11 * window(8, 7) + 11 * 10) == 1012


def test_roofline_arithmetic_on_a_sampled_timing():
    """roofline_for on a synthetic c2 run whose kernel times are a sample (one timed launch of
    each kernel, as graph replay gives): the dominant kernel is the one with the longer average
    launch; on the integer engine achieved = limb multiply-add pairs per point x points /
    duration against the measured product-window throughput; the step fraction scales the
    average launch by the launches of the timed steps; the HBM fraction uses the kernel's
    algorithmic bytes and the measured copy bandwidth."""
    mod, root = _bench_module()
    from paper_1006_0663_gb300 import workloads
    prob = workloads.CONFIGS["c2"]
    steps, k = 10, prob.substeps
    res = {"kernel_times": (0.068, 0.080, 1, 1), "ms_total": 10 * 12.25, "launches": steps * 2 * k,
           "rows_per_block": {"threads_theta": 128, "rows_per_block": 2, "variant": 1}}
    r = mod.roofline_for(res, prob, 2, 1, {"sm_mhz": 2070.0}, 152, 0.5e12, 9.0e12, "c2")
    assert r["kernel"] == "full_ix_kernel<2, 1>"
    pts = (prob.n_r - 2) * prob.n_theta
    assert abs(r["achieved"] * 1e12 - 352 * pts / 0.080e-3) < 1e3
    assert abs(r["peak"] * 1e12 - 9.0e12) < 1e3
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert abs(r["fraction_of_step_in_dominant_kernel"] - 0.080 * steps * k / (10 * 12.25)) < 1e-12
    assert r["traffic"] == mod.TRAFFIC[("c2", "full_ix_kernel<2, 1>")][0]
    # algorithmic bytes of an engine full-step point: 12 dd values moved + 9 table entries of 20 B
    assert mod.BYTES_FULL_IX[2] == 12 * 16 + 9 * 20
    assert abs(r["hbm"]["achieved_gbs"] - 372 * pts / 0.080e-3 / 1e9) < 1e-6
    assert abs(r["hbm"]["frac"] - r["hbm"]["achieved_gbs"] / r["hbm"]["peak_gbs"]) < 1e-12
    assert abs(r["fp64_equivalent"]["x_fp64_pipe_peak"]
               - mod.OPS_FULL[2] * pts / 0.080e-3 / (2 * 152 * 2070e6)) < 1e-9
    # the FP64 path counts the scheme's FP64 operations against 2 per SM per cycle
    r1 = mod.roofline_for(dict(res, kernel_times=(0.10, 0.09, 1, 1)), prob, 2, 0, {"sm_mhz": 2000.0}, 152,
                          0.5e12, 9.0e12, "c2")
    assert r1["kernel"].startswith("half_kernel<2")
    assert abs(r1["achieved"] * 1e12 - mod.OPS_HALF[2] * (prob.n_r - 1) * prob.n_theta / 0.10e-3) < 1e3
    assert abs(r1["peak"] * 1e12 - 2 * 152 * 2000e6) < 1e3
