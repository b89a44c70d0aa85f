"""Host-side logic of the library, without a GPU: segment geometry, keyed
piece planning, the range allocator, and the bucket-partitioned large-key
reduce's offsets and bulk-copy protocol (tests/cpp/host_logic.cpp, built with
the host C++ compiler from the library's own headers)."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_host_logic(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "host_logic")
    src = os.path.join(ROOT, "tests", "cpp", "host_logic.cpp")
    inc = ["-I" + os.path.join(ROOT, "include"),
           "-I" + os.path.join(ROOT, "paper_1505_01120_gb300", "csrc")]
    subprocess.run([cxx, "-std=c++17", "-O2", *inc, src, "-o", exe], check=True,
                   capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr
