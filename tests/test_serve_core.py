"""Scheduling of the serving loop (serve_core.h) on the host, with a fake
backend: admission under the memory budget in arrival order, per-stream FIFO
completion, one batch in flight per stream, batches that follow the backlog,
oldest-arrival-first dispatch, cancellation and error reporting.  The harness
is C++ (tests/serve_core_harness.cpp) built with the host compiler."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("serve") / "harness")
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-Wall",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2112_10591_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "serve_core_harness.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    return r


@pytest.mark.parametrize("scenario", ["admission", "fifo_and_batches", "continuous_batching",
                                      "oldest_first", "errors_and_cancel"])
def test_scenario(harness, scenario):
    lines = [ln for ln in harness.stdout.splitlines() if ln.split(" ")[1:2] == [scenario]
             or ln.startswith(("PASS " + scenario, "FAIL " + scenario))]
    assert lines, harness.stdout + harness.stderr
    assert lines[0].startswith("PASS"), lines[0]


def test_exit_status(harness):
    assert harness.returncode == 0, harness.stdout + harness.stderr
