"""Host check of the fused-pass schedule, both pass formations (no GPU): for
generated grid circuits, each qubit's events in its half's schedule must be the
circuit's events on that qubit.  The non-diagonal gates must come in the same
order, with the same multiset of diagonal terms between them (Section 2.4: the
diagonal gates of a layer commute).  The checker, tests/pass_schedule_check.cpp,
is compiled from the library's planner source."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = os.environ.get("CUDA_HOME", "/usr/local/cuda") + "/include"


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("psc") / "pass_schedule_check")
    src = os.path.join(ROOT, "tests", "pass_schedule_check.cpp")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I" + CUDA_INC, src, "-o", exe], check=True)
    return exe


def run(exe, R, C, d, seed, b, fuse, order):
    r = subprocess.run([exe] + [str(v) for v in (R, C, d, seed, b, fuse, order)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    return [int(v) for v in r.stdout.split()[1:]]


@pytest.mark.parametrize("R,C,d,seed,b", [(6, 10, 16, 0, 3), (8, 8, 22, 0, 4), (6, 7, 22, 0, 3), (6, 5, 16, 3, 3),
                                          (4, 4, 10, 0, 2), (3, 2, 16, 5, 2), (8, 7, 40, 2, 4)])
def test_schedule_preserves_every_qubits_events(checker, R, C, d, seed, b):
    passes = {}
    for order in (0, 1):
        for fuse in (4, 8, 10, 13):
            passes[(order, fuse)] = run(checker, R, C, d, seed, b, fuse, order)
    # the dependency-aware formation never needs more passes than the in-order one
    for fuse in (4, 8, 10, 13):
        assert sum(passes[(0, fuse)]) <= sum(passes[(1, fuse)])


def test_schedule_on_random_circuits(checker):
    rng = np.random.default_rng(7)
    for _ in range(24):
        R = int(rng.integers(2, 9))
        C = int(rng.integers(1, 9))
        if R * C > 64:
            continue
        b = int(rng.integers(1, R))
        if b * C > 32 or (R - b) * C > 32:
            continue
        d = int(rng.integers(2, 30))
        fuse = int(rng.integers(4, 14))
        for order in (0, 1):
            run(checker, R, C, d, int(rng.integers(0, 1000)), b, fuse, order)


@pytest.mark.parametrize("R,C,d,seed,rows", [(6, 3, 12, 1, [2, 4]), (8, 2, 12, 0, [2, 4, 6]), (8, 7, 10, 0, [2, 5]),
                                             (9, 3, 14, 3, [3, 6]), (8, 8, 12, 1, [3, 5]), (4, 4, 10, 3, [1, 2, 3])])
def test_multi_part_schedules(checker, R, C, d, seed, rows):
    """Every part of a multi-part cut: its gates, its internal CZs, P_l slots for the
    boundary below it and Z^l slots for the one above, with its own copy bits."""
    for order in (0, 1):
        for fuse in (4, 10, 13):
            r = subprocess.run([checker, str(R), str(C), str(d), str(seed), "multi", str(fuse), str(order)] +
                               [str(x) for x in rows], capture_output=True, text=True)
            assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr


@pytest.mark.parametrize("R,C,d,seed,b", [(6, 5, 16, 1, 3), (4, 4, 8, 1, 2), (6, 10, 16, 0, 3), (8, 8, 9, 2, 4),
                                          (5, 4, 15, 2, 2)])
def test_output_phase_schedules(checker, R, C, d, seed, b):
    """Output-sign cuts: the cut CZs that commute to the end leave the halves; every
    other event stays (the checker recomputes which cuts qualify)."""
    for order in (0, 1):
        for fuse in (4, 13):
            r = subprocess.run([checker, str(R), str(C), str(d), str(seed), str(b), str(fuse), str(order), "phase"],
                               capture_output=True, text=True)
            assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
