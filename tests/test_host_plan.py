"""The host tier's per-step plan (ring halves, chunk slots, the source of each
visible chunk's rows, the optimizer's rounds and the copy runs) checked on
the CPU: tests/host_plan_check.cpp runs random sequences of chunk-touch maps
through the planner the runtime uses and checks every invariant the copy
ordering relies on (slots inside the step's ring half, no two chunks of a
round or of consecutive rounds in one slot, each visible chunk sourced once,
device copies only from the previous step's slots in the other half, history
carried to the next step)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2509_15645_b300", "csrc")


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_host_plan_invariants(tmp_path):
    exe = tmp_path / "host_plan_check"
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Wextra", "-Werror", f"-I{CSRC}",
                    os.path.join(HERE, "host_plan_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout
