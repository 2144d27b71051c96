"""Host check of the phase-3 tile sets of the lookahead schedule (no GPU):
compiles tests/native/tileset_check.cpp against the library's tileset.h and
runs it (every tile of every stage exactly once; cross + rest = all)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_tilesets_cover_each_tile_once(tmp_path):
    exe = tmp_path / "tileset_check"
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-o", str(exe),
                    os.path.join(HERE, "native", "tileset_check.cpp")], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() == "ok"
