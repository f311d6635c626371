"""Host-side tests of the rendering service's scheduling core (admission, tickets, bounded waits,
request time-outs, stop, statistics, a fake executor with injected failures): the C++ harness
tests/native/test_serve_core.cpp is compiled with the host compiler and run. No GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_serve_core_native(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "serve_core_test"
    src = os.path.join(ROOT, "tests", "native", "test_serve_core.cpp")
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-Wall", "-o", str(exe), src], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "all checks passed" in r.stdout
