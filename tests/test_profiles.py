"""Every command that a summary under profiles/ names runs committed files:
bench.py's workloads and calls that appear there exist, and no summary
points into a scratch folder."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_profile_commands_name_existing_workloads_and_calls():
    import bench
    src = open(os.path.join(ROOT, "bench.py")).read()
    workloads = set(re.findall(r'"([a-z_]+)"', src[src.index("--workload"):src.index("--workload") + 400]))
    calls = set(bench.CALLS_ONE)
    files = glob.glob(os.path.join(ROOT, "profiles", "*.md"))
    assert files
    for f in files:
        text = open(f).read()
        assert "_work/" not in text, f
        for w in re.findall(r"--workload (\w+)", text):
            assert w in workloads or w in bench.ROWS, (f, w)
        for c in re.findall(r"--call ([\w-]+)", text):
            assert c in calls, (f, c)
