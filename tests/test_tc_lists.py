"""Host logic of the tensor-core far field: the group work lists (csrc/tc_lists.h), compiled with
the host compiler and checked on randomised block lists against brute force."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_group_lists(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "tc_lists_check"
    src = os.path.join(ROOT, "tests", "tc_lists_check.cpp")
    inc = os.path.join(ROOT, "paper_1812_10722_gb300", "csrc")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", inc, src, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
