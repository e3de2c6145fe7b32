"""The C ABI from plain C: tests/c_client/hrkan_client.c includes only
include/hrkan.h, compiles as strict C99 with gcc, links libhrkan.so and runs
the host-side entry points (shape queries, argument validation, the
checkpoint file).  No GPU is needed."""
import os
import shutil
import subprocess

import pytest

from paper_2409_14248_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_client_builds_and_runs(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc is not installed")
    lib = build.build()
    exe = str(tmp_path / "hrkan_client")
    libdir = os.path.dirname(lib)
    cmd = [gcc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_client", "hrkan_client.c"), "-o", exe, "-L", libdir, "-lhrkan",
           f"-Wl,-rpath,{libdir}", "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe, str(tmp_path / "client.ck")], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    assert "all checks passed" in r.stdout
