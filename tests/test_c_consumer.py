"""The C ABI from plain C (no GPU): tests/native/c_consumer.c is compiled as
C99 with -pedantic -Werror against include/apsp.h, linked to the built
libapsp.so and run (host-side entry points only)."""
import os
import shutil
import subprocess

import pytest

from paper_1001_4108_gb300 import binding

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_plain_c_consumer(tmp_path):
    if not os.path.exists(binding.LIB_PATH):
        pytest.skip("libapsp.so not built")
    libdir = os.path.dirname(binding.LIB_PATH)
    exe = tmp_path / "c_consumer"
    subprocess.run(["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-O1",
                    "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "native", "c_consumer.c"),
                    "-L", libdir, "-lapsp", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("ok")
