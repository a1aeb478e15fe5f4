"""The one-launch step's planner (host code) checked without a GPU.

tests/plan_check.cpp is compiled with g++ against the library's own planner header and
checks, for each geometry, that every U/theta tile waits for exactly the phase-field tiles
whose phi^{n+1} its ring reads (recomputed by brute force from the kernels' index ranges)
and that all of those come earlier in the ticket order, the property that makes every wait
of the launch end.  The geometries cover ragged tiles, z-chunks of one and two planes (the
ring then reaches two chunks away), 2D one-row blocks, batches of uneven simulations in the
batch's item order, and lags of zero to more than the whole launch.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "plan_check.cpp")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-Wall", "-o", exe, SRC], check=True)
    return exe


def run(checker, by, lag, sims, batch_order=0):
    args = [checker, str(by), str(lag), str(batch_order)]
    for s in sims:
        args += [str(v) for v in s]
    r = subprocess.run(args, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok")
    return r.stdout


@pytest.mark.parametrize("by", [4, 6, 8])
@pytest.mark.parametrize("zchunk", [1, 2, 3, 8, 13])
def test_single_simulation_ragged(checker, by, zchunk):
    # 67 columns (3 tiles, last ragged), rows not a multiple of by - 2, 29 planes
    run(checker, by, 5, [(67, 23, 29, zchunk)])


@pytest.mark.parametrize("lag", [0, 1, 40, 100000])
def test_lags(checker, lag):
    run(checker, 8, lag, [(95, 31, 40, 16)])


def test_one_chunk_and_tiny_grids(checker):
    run(checker, 8, 3, [(30, 6, 20, 20)])    # one tile, one chunk
    run(checker, 4, 3, [(1, 1, 1, 1)])       # a single node
    run(checker, 8, 3, [(2, 3, 5, 32)])      # chunk longer than the grid
    run(checker, 6, 0, [(61, 4, 3, 1)])      # one-plane chunks


def test_2d_one_row_blocks(checker):
    run(checker, 1, 10, [(130, 1, 57, 8)])
    run(checker, 1, 0, [(30, 1, 9, 1)])


def test_batch_of_uneven_simulations(checker):
    sims = [(48, 48, 48, 48), (64, 64, 64, 32), (80, 80, 80, 40), (96, 96, 96, 48), (33, 29, 23, 23)]
    out = run(checker, 8, 50, sims, batch_order=1)
    assert int(out.split()[1]) > 0


def test_checker_catches_a_planted_fault(checker, tmp_path):
    """The same checker against a planner that forgets the plane below the chunk: the
    check must fail, so a passing run means the dependency rule was really verified."""
    src = open(SRC).read()
    hdr = open(os.path.join(ROOT, "paper_1602_07483_gb300", "csrc", "lbpf_plan.h")).read()
    bad = hdr.replace("std::max(w.z0 - 2, 0) / g.zchunk", "std::max(w.z0 - 1, 0) / g.zchunk")
    assert bad != hdr
    (tmp_path / "lbpf_plan.h").write_text(bad)
    (tmp_path / "plan_check.cpp").write_text(
        src.replace('#include "../paper_1602_07483_gb300/csrc/lbpf_plan.h"', '#include "lbpf_plan.h"'))
    exe = str(tmp_path / "bad_check")
    subprocess.run([shutil.which("g++"), "-std=c++17", "-O2", "-o", exe, str(tmp_path / "plan_check.cpp")],
                   check=True)
    r = subprocess.run([exe, "8", "5", "0", "64", "20", "40", "1"], capture_output=True, text=True)
    assert r.returncode == 1 and "violation" in r.stdout
