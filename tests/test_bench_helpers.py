"""bench.py's host-side pieces (CPU only): the two-pipe ALU ceiling used as
the roofline peak, and the pixel-sampled oracle timing behind the
cpu_baseline of the c3 / c4 / c5 lines."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from workloads import random_problem  # noqa: E402


def test_two_pipe_ceiling_balances_the_pipes():
    r = bench.alu_terms_per_clk_per_sm()
    # at the optimum share a, the MUFU and FP32 pipes take the same time
    m = bench.MUFU_PER_TERM / bench.MUFU_PER_CLK_PER_SM
    F = 1.0 / bench.FP32_PER_CLK_PER_SM
    fm, fp = bench.FP32_PER_TERM_MUFU_PATH, bench.FP32_PER_TERM_POLY_PATH
    a = 1.0 - 1.0 / (r * m)
    assert 0.0 < a < 1.0
    assert abs(m * (1 - a) - F * (fm * (1 - a) + fp * a)) < 1e-12
    # more than either pipe alone allows
    assert r > 1.0 / m and r > 1.0 / (F * fp)
    assert abs(r - 12.40) < 0.01      # the figure quoted with the roofline


@pytest.mark.parametrize("kind", ["wgs", "grad"])
def test_sampled_oracle_stride_and_terms(kind, monkeypatch):
    ps = [random_problem(3, 40, 30, 12, [2, 3, 4]), random_problem(4, 24, 24, 5, [2, 3])]
    per = 2 if kind == "wgs" else 3
    total = sum(per * p.N * p.M for p in ps)
    monkeypatch.setitem(bench.ORACLE_SAMPLE_TERMS, kind, total / 3.5)
    terms, secs, stride = bench.oracle_sampled(kind, ps, 1)
    assert stride == 4                                   # ceil(3.5)
    assert terms == sum(per * p.N * len(np.arange(0, p.M, 4)) for p in ps)
    assert secs > 0.0
    line = bench._sampled_baseline(kind, ps, "sample")
    assert line["kind"] == "oracle" and line["unit"] == bench.UNIT and line["value"] > 0
    assert "every 4-th pixel" in line["sample"]
