"""The benchmark's roofline model of the near/far kernel (bench.kernel_work
and bench.roofline): per-pair instruction and MUFU counts, worked by hand
for small pair counts, and the launch groups of up to 8 fields that the
library forms (the Hartree field joins the last group when it fits)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as b

    return b


INFO = {"near_pairs": 100, "far_pairs": 200, "near_pairs_nogauss": 10, "far_pairs_nogauss": 50, "degree": 8}


def test_kernel_work_counts(bench):
    # 2 Yukawa fields + Hartree: near 10 + 12 + 5 (2 without the Gaussian),
    # far on the tensor grid 4 + 10 + 5 (1 without)
    instr, xu = bench.kernel_work(INFO, 2, True)
    assert instr == 90 * 27 + 10 * 24 + 150 * 19 + 50 * 15
    # MUFU in ex2 units: rsqrt 2 + 2 Yukawa + 1 Gaussian where present
    assert xu == 300 * 4 + 240 * 1
    # other degrees take the record far path (8 geometry instructions)
    instr6, _ = bench.kernel_work(dict(INFO, degree=5), 2, True)
    assert instr6 == instr + 200 * 4


def test_roofline_groups(bench):
    def work(ny, hh):
        return bench.roofline(INFO, ny, hh, 1.0, 2000.0, 152)[2]["instr_per_interaction"]

    # one launch: 2 + H, 7 + H, 8 Yukawa alone
    i, _ = bench.kernel_work(INFO, 2, True)
    assert work(2, True) == pytest.approx(i / (300 * 3))
    # 8 Yukawa + H: two launches, the Hartree field alone in the second
    i8, _ = bench.kernel_work(INFO, 8, False)
    i0, _ = bench.kernel_work(INFO, 0, True)
    assert work(8, True) == pytest.approx((i8 + i0) / (300 * 9))
    # 21 Yukawa + H: 8, 8 and 5 + H
    i5, _ = bench.kernel_work(INFO, 5, True)
    assert work(21, True) == pytest.approx((2 * i8 + i5) / (300 * 22))


def test_oracle_sample_covers_nucleus_and_every_thread(bench):
    """The CPU legs time the oracle on at least 2 batches per thread and
    always on the batches that meet at the nucleus; the sample reports the
    oracle's fields there, which the error leg compares with the GPU."""
    import numpy as np

    import oracle
    from paper_2003_01833_gb300 import workloads as W

    wl = W.hydrogen_adaptive()
    wl.degree, wl.leaf_size = 4, 500
    before = oracle.threads()
    try:
        smp = bench.OracleSample(wl, nthreads=2)
        assert smp.threads == 2 and len(smp.nuc) >= 1
        rate, desc, outs, pts, nuc_pts = smp.run(2 * smp.threads, seed=0)
    finally:
        oracle.threads(before)  # the later oracle tests use every core
    assert rate > 0 and len(outs) == 2
    assert set(nuc_pts) <= set(pts)
    nb = sum(1 for c in smp.leaves if set(smp.ot.points(c)) <= set(pts))
    assert nb >= max(2 * smp.threads, len(smp.nuc) + 1)
    # the oracle's own fields against themselves: zero error; a 1e-6 relative
    # perturbation of the nucleus targets shows up there and not elsewhere
    e0 = bench.rel_err_vs_oracle(outs, outs, wl.mesh.w, pts, nuc_pts)
    assert all(v[s][k] == 0.0 for v in e0.values() for s in ("nucleus", "other") for k in ("plain", "weighted"))
    g = [o.copy() for o in outs]
    for o in g:
        o[nuc_pts] *= 1 + 1e-6
    e1 = bench.rel_err_vs_oracle(g, outs, wl.mesh.w, pts, nuc_pts)
    for v in e1.values():
        assert abs(v["nucleus"]["plain"] - 1e-6) < 1e-9 and v["other"]["plain"] == 0.0
    np.testing.assert_allclose(e1["hartree"]["nucleus"]["weighted"], 1e-6, rtol=1e-3)


def test_workload_names_match_between_arms(bench):
    from paper_2003_01833_gb300 import workloads as W

    wl = W.hydrogen_1s()
    assert bench.workload_name(wl) == bench.workload_name(wl)
    assert f"{wl.n} points" in bench.workload_name(wl)


def test_reference_arm_prints_its_line(bench, capsys):
    """bench.py --impl reference (the oracle on the host cores) on the small
    Li mesh: one JSON line with the keys the comparison of the two arms reads,
    the same workload string as the GPU arm, and the oracle thread count put
    back afterwards."""
    import argparse
    import json

    import oracle

    before = oracle.threads()
    saved = bench.WORKLOAD
    try:
        bench.WORKLOAD = "li-small"
        bench.run_reference(argparse.Namespace(gpus=1, steps=1, warmup=0))
    finally:
        bench.WORKLOAD = saved
        oracle.threads(before)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == bench.UNIT
    assert line["metric"] == bench.METRIC and line["higher_is_better"] is True
    assert line["config"]["workload"].startswith("Li atom") and "99000 points" in line["config"]["workload"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
