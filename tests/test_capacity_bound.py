"""The sampled run capacities of the row-tile update (host arithmetic, no GPU).

The overflow list of a sampled pass starts after rec_words x
sample_capacity_bound() words of the workspace, so the capacities of all
tiles must never sum above that bound, whatever the sample's counts; and
sample_capacity must use the exact ceiling of sqrt(c + 1).  The header is
compiled on the host with g++ and checked over even, single-tile, geometric
and random count vectors of the largest possible sample.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_capacity_sum_within_bound(tmp_path):
    exe = str(tmp_path / "capacity_bound_check")
    cmd = ["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_1901_06207_b300", "csrc"), "-I", "/usr/local/cuda/include",
           os.path.join(ROOT, "tests", "capacity_bound_check.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("build failed:\n" + r.stderr[-2000:])
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout[-500:]
    rows = [list(map(int, line.split())) for line in out.stdout.split("\n") if line.strip()]
    assert len(rows) == 5 * 4 * 4
    for m, nb, kind, total, bound in rows:
        assert total <= bound, (m, nb, kind, total, bound)
        # and the bound is not far above what it bounds: 1/8 slack, 4 sigma, 256 per tile, rounding
        assert bound <= 1.25 * m + 260 * nb + 4 * 16 * ((nb * (m / 16 + 2048 + nb)) ** 0.5 + nb) + 64 * 1024
