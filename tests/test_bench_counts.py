"""The per-unit work figures behind bench.py's roofline, checked against the
numbers written out by hand from the hot-path formulas (n = 50, m = 100,
p = 10, the workload the metric is quoted on)."""
import numpy as np

import bench


def test_fma_counts_degenerate_workload():
    factor, rhs, it = bench.fma_counts(50, 100, 10)
    # m n(n+1)/2 = 127,500 (G'WG), n^3/6 = 20,833.3, p n^2/2 = 12,500,
    # p^2 n/2 = 2,500, p^3/6 = 166.7
    assert abs(factor - 163_500.0) < 1e-6
    # n^2 + 2mn + 2pn + p^2 = 2,500 + 10,000 + 1,000 + 100
    assert rhs == 13_600
    # factor + 2 rhs + residuals (n^2 + 2mn + 2pn = 13,500)
    assert abs(it - 204_200.0) < 1e-6


def test_forward_flops_per_instance():
    # start (factor + one rhs), 13.16 Newton iterations, final factor; x 2
    iters = np.full(100, 13.16)
    per = bench.forward_flops(50, 100, 10, iters) / 100
    expect = 2 * ((163_500 + 13_600) + 13.16 * 204_200 + 163_500)
    assert abs(per - expect) < 1e-3
    assert abs(per / 1e6 - 6.055) < 0.01


def test_backward_bytes_per_instance():
    # read, with the plain-Schur factor sizes of the hot-path table: L
    # (n(n+1)/2 = 1,275), Y (pn = 500), L_S (p(p+1)/2 = 55), z and W (2m =
    # 200), x and y (n + p = 60), G (mn = 5,000), g (n = 50) = 7,140 floats;
    # write dQ, dq, dA, db, dG, dh = 2,500 + 50 + 500 + 10 + 5,000 + 100 =
    # 8,160 floats
    assert bench.backward_bytes(50, 100, 10, 1) == 4 * (7_140 + 8_160)
    assert bench.backward_bytes(50, 100, 10, 4096) == 4096 * 61_200


def test_fp32_peak():
    assert abs(bench.fp32_alu_peak_tflops() - 152 * 128 * 2 * 2.07e-3) < 1e-9


def test_profile_commands_are_valid_bench_invocations():
    """Every `python bench.py ...` command quoted in profiles/ parses with the
    bench's own argument parser (the summaries must name commands that run)."""
    import glob
    import os
    import re
    import shlex

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    files = sorted(glob.glob(os.path.join(root, "profiles", "*.md")))
    assert files
    found = 0
    for path in files:
        text = open(path).read().replace("\\\n", " ")
        for cmd in re.findall(r"python bench\.py([^\n`]*)", text):
            bench.parse(shlex.split(cmd))
            found += 1
    assert found >= len(files)
