"""Host checks of index arithmetic that the kernels share with plain C++
headers: the stream-K GEMM's work split (csrc/stream_k.cuh) and the
deterministic dense assembly's colouring and pair schedule
(csrc/dense_sched.cuh).  Each check is compiled with g++ and run; no GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(tmp_path, name):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / name
    subprocess.run([gxx, "-O2", "-std=c++17", "-Wall", "-Werror", os.path.join(HERE, name + ".cpp"),
                    "-o", str(exe)], check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok "), r.stdout
    return int(r.stdout.split()[1])


def test_stream_k_split_covers_every_iteration_once(tmp_path):
    """1504 (tiles, K slices, grid) cases, including the grid the library picks."""
    assert _run(tmp_path, "stream_k_check") > 1000


def test_dense_schedule_single_writer(tmp_path):
    """Folded pair enumeration for n up to 1333; proper greedy colouring, every
    unordered triangle pair once and one writer per entry and launch on tori,
    random triangle soups and fans."""
    assert _run(tmp_path, "dense_sched_check") > 900
