"""The workload table's substep counts are the oracle's stability analysis, as stored in
tests/golden/substeps.json by tests/golden/make_substeps.py (which calls only oracle/)."""
import json
import os

from paper_1006_0663_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "substeps.json")


def test_substeps_match_the_stability_analysis():
    with open(GOLDEN) as f:
        g = json.load(f)
    for name, p in workloads.CONFIGS.items():
        assert p.substeps == g["configs"][name]["substeps"], name
    assert list(workloads.BATCH_SUBSTEPS) == g["batch"]
    assert len(g["batch"]) == workloads.BATCH_SIZE
