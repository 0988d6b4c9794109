"""The committed profile summaries stay tied to the sources and commands that made them."""
import glob
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def test_recorded_dram_traffic_matches_the_kernel_sources():
    """bench.py reports ncu DRAM traffic only while the Dslash sources hash to the value
    recorded with it; every recorded capture names its summary, and the summary exists."""
    with open(os.path.join(PROFILES, "dram_traffic.json")) as f:
        d = json.load(f)
    entries = {k: v for k, v in d.items() if not k.startswith("_")}
    assert entries
    for key, e in entries.items():
        assert e["bytes_per_launch"] > 0
        assert os.path.exists(os.path.join(ROOT, e["capture"])), e["capture"]
    stale = [k for k, e in entries.items() if e["csrc_hash"] != bench.csrc_hash()]
    for key in stale:
        assert bench.recorded_traffic(key) is None
    if stale:
        pytest.skip(f"Dslash sources changed since the ncu captures of {stale}: bench.py reports "
                    "traffic null until they are retaken")


def test_every_summary_gives_its_command():
    for p in glob.glob(os.path.join(PROFILES, "*.md")):
        text = open(p).read()
        assert "ommand" in text and "bench.py" in text, p
    for p in glob.glob(os.path.join(PROFILES, "solvers_*.json")):
        with open(p) as f:
            d = json.load(f)
        assert d["command"].startswith("python bench.py --workload"), p
        assert "compare" in d, p
