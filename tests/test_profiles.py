"""The committed ncu summaries: every capture command keeps the GPU's clocks
(--clock-control none), names one kernel and a bounded launch count when it
collects more than the launch list, and runs committed files only; the traffic
records name existing summaries and kernel sources."""

import glob
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _commands(path):
    return [l.strip() for l in open(path) if l.strip().startswith(("ncu ", "python "))]


def test_every_summary_gives_its_commands_and_they_are_safe():
    files = sorted(glob.glob(os.path.join(PROFILES, "*.md")))
    assert len(files) >= 10
    for path in files:
        if os.path.basename(path) == "README.md":
            continue
        cmds = _commands(path)
        assert cmds, f"{os.path.basename(path)} gives no command"
        for c in cmds:
            for script in re.findall(r"python3? (\S+\.py)", c):
                assert os.path.exists(os.path.join(ROOT, script)), (path, script)
            if c.startswith("ncu "):
                assert "--clock-control none" in c, (path, c)
                if "--metrics gpu__time_duration.sum " not in c:      # more than the launch list
                    assert re.search(r"-k regex:\S+", c) and re.search(r" -c [123] ", c), (path, c)


def test_traffic_records_point_at_existing_summaries_and_sources():
    rec = json.load(open(os.path.join(PROFILES, "traffic.json")))
    for key, e in rec.items():
        kernel, workload = key.split(":", 1)
        summary = re.search(r"profiles/(\S+\.md)", e["note"]).group(1)
        assert os.path.exists(os.path.join(PROFILES, summary)), key
        assert summary.startswith(kernel) and workload in summary, key
        for f in e["sources"]:
            assert os.path.exists(os.path.join(ROOT, "paper_2012_07145_gb300", "csrc", f)), (key, f)
        assert e["dram_bytes_per_launch"] > 0
