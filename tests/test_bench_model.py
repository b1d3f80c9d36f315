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
