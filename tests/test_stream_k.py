"""Host check of the stream-K GEMM's work split (csrc/stream_k.cuh, the
header its kernels use): compiled with g++ and run over many (tiles, K
slices, grid) combinations, including the grid the library picks.  No GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_stream_k_split_covers_every_iteration_once(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "stream_k_check"
    subprocess.run([gxx, "-O2", "-std=c++17", "-Wall", "-Werror", os.path.join(HERE, "stream_k_check.cpp"),
                    "-o", str(exe)], check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok "), r.stdout
    assert int(r.stdout.split()[1]) > 1000
