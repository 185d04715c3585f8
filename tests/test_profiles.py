"""The committed profile summaries state how they were made: each gives the
command (committed files only, ncu with the GPU clocks left alone), and the
DRAM figures the bench reads name a source file that exists."""

import glob
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def test_every_summary_gives_its_command():
    mds = sorted(glob.glob(os.path.join(PROFILES, "*.md")))
    assert mds
    for path in mds:
        text = open(path).read()
        assert "python bench.py" in text, path
        assert "_work" not in text and "gpurun" not in text, path
        # the indented command block, continuation lines joined
        cmds, cur = [], ""
        for line in text.splitlines():
            if line.startswith("    "):
                cur += " " + line.strip().rstrip("\\")
                if not line.rstrip().endswith("\\"):
                    cmds.append(cur)
                    cur = ""
        parts = [q.strip() for c in cmds for q in c.split("&&")]
        profiled = [q for q in parts if q.startswith("ncu ")]
        assert profiled, path
        for c in profiled:
            assert "--clock-control none" in c, (path, c)


def test_traffic_records_name_existing_sources():
    with open(os.path.join(PROFILES, "traffic.json")) as f:
        d = json.load(f)
    assert d
    for kernel, rec in d.items():
        assert os.path.exists(os.path.join(ROOT, rec["source"])), kernel
        assert len(rec["source_sha16"]) == 16, kernel
        assert rec["dram_bytes_per_work"] > 0 and rec["work"] > 0, kernel
        assert abs(rec["dram_bytes"] / rec["work"] - rec["dram_bytes_per_work"]) <= 1e-9 * rec["dram_bytes_per_work"]
