"""CPU checks of the serving loop's host scheduling core (admission by a
device-memory budget in FIFO order, packing of a tick into a cartridge-grouped
work list, busy rules, idle reclaim, slot accounting): tests/sched_check.cpp
compiled against the library's serve_sched.cpp and run."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1907_08467_gb300", "csrc")


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_scheduler_invariants(tmp_path):
    exe = str(tmp_path / "sched_check")
    cmd = ["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC,
           os.path.join(ROOT, "tests", "sched_check.cpp"), os.path.join(CSRC, "serve_sched.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
