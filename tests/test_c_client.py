"""The header is valid C and a plain-C program links against the library and
calls its host-only entry points (no device needed)."""
import os
import shutil
import subprocess

import pytest

from paper_1808_00270_gb300 import build as B

SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c", "host_calls.c")


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_c_client_calls_host_entry_points(tmp_path):
    lib = B.build()
    exe = tmp_path / "host_calls"
    cmd = ["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(B.ROOT, "include"), SRC, "-o", str(exe),
           "-L", os.path.dirname(lib), "-l:" + os.path.basename(lib), "-Wl,-rpath," + os.path.dirname(lib), "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stdout, out.stderr)
