"""Host execution of the planner's schedules against the oracle (no GPU).

tests/schedule_exec_check.cpp is compiled from the library's planner source.  It
evolves both halves of listed copies through the fused-pass schedule (copy-tree
levels with their hoisted ops, passes, diagonal ops with cut slots) in FP64 with
full gate matrices; every leaf must equal the oracle's gate-by-gate half-state of
that copy (Supplementary A, Eqs. 1, 4-5).  It also evaluates selected leaf entries
from an ancestor d levels up (the sparse leaves' formula), which must equal the
leaf's own entries.  Multi-part plans (Section 3, Fig. 3) are executed part by part
against the oracle's part states.  This pins the schedule transformations
(dependency-aware pass formation, ops moved up the copy tree, controlled-gate
slots, the P_l / Z^l slots of middle parts) independently of the GPU kernels."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import circuit as oc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = os.environ.get("CUDA_HOME", "/usr/local/cuda") + "/include"


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("sec") / "schedule_exec_check")
    src = os.path.join(ROOT, "tests", "schedule_exec_check.cpp")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I" + CUDA_INC, src, "-o", exe], check=True)
    return exe


def check(exe, tmp_path, R, C, depth, gates, b, fuse, order, copies):
    n, n_u = R * C, b * C
    txt = tmp_path / "circuit.txt"
    txt.write_text(oc.to_text(R, C, depth, 0, gates))
    out = tmp_path / "leaves.bin"
    r = subprocess.run([exe, str(txt), str(b), str(fuse), str(order), str(out)] + [str(int(k)) for k in copies],
                       capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    _, tried, worst = r.stdout.split()
    data = np.fromfile(str(out), dtype=np.complex128)
    plan = oc.CutPlan(n, n_u, gates)
    pos = 0
    for k in copies:
        for half, nh in ((0, n_u), (1, n - n_u)):
            got = data[pos:pos + (1 << nh)]
            pos += 1 << nh
            ref = oracle.half_state(plan, half, int(k))
            scale = max(float(np.max(np.abs(ref))), 1e-300)
            assert float(np.max(np.abs(got - ref))) <= 1e-12 * scale, (k, half)
    assert pos == data.size
    assert float(worst) <= 1e-12
    return int(tried)


@pytest.mark.parametrize("R,C,d,seed,b", [(4, 4, 10, 0, 2), (4, 5, 16, 0, 2), (6, 4, 17, 2, 3),
                                          (4, 6, 22, 1, 2), (3, 4, 20, 5, 1), (5, 4, 14, 3, 2)])
def test_schedules_of_generated_circuits(checker, tmp_path, R, C, d, seed, b):
    gates, plan = oc.grid_cut(R, C, d, seed, b)
    copies = sorted({0, plan.copies // 3, plan.copies - 1})
    tried = 0
    for fuse, order in ((13, 0), (13, 1), (5, 0), (8, 1)):
        tried += check(checker, tmp_path, R, C, d, gates, b, fuse, order, copies)
    if plan.c > 0:
        assert tried > 0


@pytest.mark.parametrize("name", ["CX", "CT", "CY2"])
def test_schedules_with_controlled_gate_cuts(checker, tmp_path, name):
    from circuits import cx_cut_circuit
    for seed in (0, 1):
        R, C, b, depth, gates = cx_cut_circuit(seed, name)
        plan = oc.CutPlan(R * C, b * C, gates)
        copies = sorted({0, plan.copies // 2 + 1, plan.copies - 1})
        for fuse, order in ((13, 0), (6, 1)):
            check(checker, tmp_path, R, C, depth, gates, b, fuse, order, copies)


def test_schedules_of_random_circuits(checker, tmp_path):
    from circuits import with_cross_controlled
    rng = np.random.default_rng(21)
    for _ in range(12):
        R = int(rng.integers(2, 6))
        C = int(rng.integers(2, 5))
        b = int(rng.integers(1, R))
        if b * C > 12 or (R - b) * C > 12:
            continue
        d = int(rng.integers(3, 24))
        seed = int(rng.integers(0, 1000))
        gates = with_cross_controlled(R, C, d, seed, b, rng, p=0.4, max_cuts=8)
        plan = oc.CutPlan(R * C, b * C, gates)
        copies = sorted({0, int(rng.integers(0, plan.copies)), plan.copies - 1})
        check(checker, tmp_path, R, C, d, gates, b, int(rng.integers(4, 14)), int(rng.integers(0, 2)), copies)


@pytest.mark.parametrize("R,C,d,seed,rows", [(6, 3, 16, 0, (2, 4)), (8, 2, 20, 3, (2, 5, 6)), (6, 4, 12, 1, (3,))])
def test_schedules_of_multi_part_cuts(checker, tmp_path, R, C, d, seed, rows):
    gates = oc.generate(R, C, d, seed, rows[0])
    plan = oc.MultiCutPlan(R, C, rows, gates)
    txt = tmp_path / "circuit.txt"
    txt.write_text(oc.to_text(R, C, d, 0, gates))
    cbits = [len(plan.local[p]) for p in range(plan.t)]
    copies = sorted({0, 1, 5, (1 << max(cbits)) - 1})
    for fuse, order in ((13, 0), (5, 1)):
        out = tmp_path / "parts.bin"
        r = subprocess.run([checker, str(txt), "multi:" + ",".join(str(x) for x in rows), str(fuse), str(order),
                            str(out)] + [str(k) for k in copies], capture_output=True, text=True)
        assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
        data = np.fromfile(str(out), dtype=np.complex128)
        pos = 0
        for k in copies:
            for p in range(plan.t):
                if k >> cbits[p]:
                    continue
                got = data[pos:pos + (1 << plan.nq[p])]
                pos += 1 << plan.nq[p]
                ref = oracle.part_state(plan, p, int(k))
                scale = max(float(np.max(np.abs(ref))), 1e-300)
                assert float(np.max(np.abs(got - ref))) <= 1e-12 * scale, (k, p)
        assert pos == data.size
