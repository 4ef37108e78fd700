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
    """Every traffic and instruction-count entry of bench.py names a committed profile summary
    that covers its kernel function and prints its numbers; the integer-engine kernels the
    autotuner picks for the benchmark's workloads (both dd shapes at c2, qd at c3) have both."""
    mod, root = _bench_module()
    def mentions(text, kname):  # names are printed with or without the space after the comma
        return kname.replace(" ", "") in text.replace(" ", "")

    for (workload, kname), (traffic, shape, src) in mod.TRAFFIC.items():
        text = open(os.path.join(root, src)).read()
        assert mentions(text, kname), (kname, src)
        assert workload in text, (workload, src)
    for kname, (inst, src) in mod.IX_INST.items():
        text = open(os.path.join(root, src)).read()
        assert mentions(text, kname), (kname, src)
        assert f" {inst} " in text or f" {inst}\n" in text, (kname, inst, src)
    for kname, workload in [("half_ix_kernel<2, 1>", "c2"), ("full_ix_kernel<2, 1>", "c2"),
                            ("half_ix_kernel<2, 2>", "c2"), ("full_ix_kernel<2, 2>", "c2"),
                            ("half_ix_kernel<4, 1>", "c3"), ("full_ix_kernel<4, 1>", "c3")]:
        assert (workload, kname) in mod.TRAFFIC, kname
        assert kname in mod.IX_INST, kname
    # the engine's traffic figures are the ones printed in the summaries (MB, read + write)
    for (workload, kname), (traffic, shape, src) in mod.TRAFFIC.items():
        if "_ix_kernel" not in kname:
            continue
        text = open(os.path.join(root, src)).read()
        found = False
        for line in text.splitlines():
            if "DRAM read + write" in line:
                nums = [float(x) for x in line.replace("MB", " ").replace("+", " ").split() if _isnum(x)]
                pairs = [nums[k] + nums[k + 1] for k in range(0, len(nums) - 1, 2)]
                found |= any(abs(p * 1e6 - traffic) < 0.02e6 for p in pairs)
        assert found, (kname, traffic, src)


def _isnum(x):
    try:
        float(x)
        return True
    except ValueError:
        return False
