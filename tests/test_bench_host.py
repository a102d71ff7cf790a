"""Host-side logic of bench.py (no GPU): the algorithmic per-DOF figures behind the
roofline, the whole-job PID, the derived FP64 peak, and that the committed ncu
evidence (NCU_TRAFFIC and the profiles' hash lines) belongs to the kernel sources
as they stand."""
import glob
import os
import re

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_bytes_and_flops_per_dof():
    # minimum-traffic three-kernel schedule: 46 + 117 f words per DOF and stage, f = 3/n
    b64, blv64, flv = bench.algorithmic_per_dof(8, 8)
    assert b64 == pytest.approx(719.0) and blv64 == pytest.approx((20 + 48 * 3 / 8) * 8)
    b32, _, _ = bench.algorithmic_per_dof(8, 4)
    assert b32 == pytest.approx(359.5)
    b6, _, _ = bench.algorithmic_per_dof(6, 4)  # N = 5: 104.5 words
    assert b6 == pytest.approx(418.0)
    # lifting + volume flops at n = 8 (FMA = 2): 90 n + 180 + 70 + 180 + 90 + 90 + 30 n
    assert flv == 90 * 8 + 180 + 70 + 180 + 90 + 90 + 30 * 8 == 1570


def test_whole_job_pid_and_peak():
    # 2,097,152 DOF x 5 stages x 50 steps in 1.0245 s -> 1.954 ns per DOF-stage; two replicas: half
    assert bench.whole_job_pid(1.0245, 50, 2097152, 1) == pytest.approx(1.0245e9 / (50 * 5 * 2097152))
    assert bench.whole_job_pid(1.0, 10, 1000, 2) == pytest.approx(0.5 * bench.whole_job_pid(1.0, 10, 1000, 1))
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.25856)
    assert bench.max_over_ranks(3.5) == 3.5


def test_kernel_hash_ignores_comments_only():
    texts = []
    for f in bench.KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            texts.append(fh.read())
    h = bench.kernel_source_hash(texts)
    assert h == bench.kernel_source_hash()
    commented = [t.replace("namespace flexi {", "namespace flexi {  // a comment\n/* block */\n", 1) for t in texts]
    assert bench.kernel_source_hash(commented) == h
    changed = list(texts)
    changed[0] = changed[0].replace("real(0.5)", "real(0.25)", 1)
    assert bench.kernel_source_hash(changed) != h


def test_committed_ncu_evidence_matches_the_kernel_sources():
    """NCU_TRAFFIC and the profiles' hash lines name the current kernel sources; a
    kernel change without a new capture shows up here (and bench.py reports a null
    roofline.traffic)."""
    h = bench.kernel_source_hash()
    assert {k[1] for k in bench.NCU_TRAFFIC} == {h}
    assert {k[0] for k in bench.NCU_TRAFFIC} == {"fp64", "fp32"}
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        text = open(path, encoding="utf-8").read()
        for m in re.finditer(r"Kernel sources hash[^:]*: ([0-9a-f]{16})", text):
            assert m.group(1) == h, (os.path.basename(path), m.group(1), h)
