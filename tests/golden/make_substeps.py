"""Writes tests/golden/substeps.json: the Lax-Wendroff iterations per outer step k of every
workload, from the oracle's stability analysis (oracle/stability.py) and nothing else.

The paper gives no time-step rule (Sec. 3.B states only that the scheme is stable). The
reading adopted: k is the smallest integer for which the excess amplification of the worst
local mode of the discrete operator, over the whole run, stays below 10x.

    python tests/golden/make_substeps.py [name ...]
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.stability import analyse  # noqa: E402
from paper_1006_0663_gb300 import workloads  # noqa: E402


def main(names=()):
    """All workloads, or only the named ones (the others are kept from the existing file)."""
    path = os.path.join(HERE, "substeps.json")
    out = {"reading": "smallest k with (worst excess amplification)^(steps k) <= 10; "
                      "oracle/stability.py", "configs": {}, "batch": []}
    if names and os.path.exists(path):
        with open(path) as f:
            out = json.load(f)
    for name, p in workloads.CONFIGS.items():
        if names and name not in names:
            continue
        k, lam = analyse(p)
        out["configs"][name] = {"substeps": k, "max_abs_lambda": lam}
        print(name, k, lam, flush=True)
    if not names or "c4" in names:
        out["batch"] = []
        for i in range(workloads.BATCH_SIZE):
            k, lam = analyse(workloads.batch_member(i, substeps=1))
            out["batch"].append(k)
            print(f"c4[{i}]", k, flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(tuple(sys.argv[1:]))
