"""Pins of the compact volume rules the volume kernels integrate with (3D, k = 3, 4, 5):
read from the committed table header and checked, independently of the library's
self-test, against the closed form int_T x^a y^b z^c = a! b! c! / (a + b + c + 3)! on the
unit tetrahedron for every a + b + c <= 3k - 1, with positive weights and interior points
(the rules replace the collapsed Gauss-Jacobi rule only where the integrand is a
polynomial of that degree, so exactness is the whole requirement)."""
import math
import os
import re

import numpy as np
import pytest

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2408_06698_gb300", "csrc", "volume_rules.h")


def _rule(k):
    text = open(HEADER).read()
    n = int(re.search(rf"kTetRule{k}N = (\d+);", text).group(1))
    body = re.search(rf"kTetRule{k}\[{n} \* 4\] = \{{(.*?)\}};", text, re.S).group(1)
    vals = np.array([float(v) for v in body.replace("\n", " ").split(",") if v.strip()])
    assert vals.size == 4 * n
    r = vals.reshape(n, 4)
    return r[:, :3], r[:, 3]


@pytest.mark.parametrize("k,npts", [(3, 46), (4, 100), (5, 190)])
def test_compact_rule_is_exact_to_degree_3k_minus_1(k, npts):
    X, w = _rule(k)
    assert X.shape == (npts, 3)
    deg = 3 * k - 1
    worst = 0.0
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
                got = float(np.sum(w * X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c))
                worst = max(worst, abs(got - exact) / exact)
    assert worst < 1e-13, worst
    # one degree more is not integrated exactly (the rule is not accidentally richer)
    d1 = deg + 1
    miss = max(abs(float(np.sum(w * X[:, 0] ** a * X[:, 1] ** (d1 - a))) -
                   math.factorial(a) * math.factorial(d1 - a) / math.factorial(d1 + 3))
               / (math.factorial(a) * math.factorial(d1 - a) / math.factorial(d1 + 3)) for a in range(d1 + 1))
    assert miss > 1e-10


@pytest.mark.parametrize("k", [3, 4, 5])
def test_compact_rule_weights_positive_points_interior(k):
    X, w = _rule(k)
    assert np.all(w > 0)
    bary = np.column_stack([1.0 - X.sum(1), X])
    assert bary.min() > 1e-4
    assert abs(w.sum() - 1.0 / 6.0) < 1e-15


def test_bench_flop_model_uses_the_kernels_rule_sizes():
    """bench.py's algorithmic flop count of the volume kernel uses the point counts of the
    committed rules (and of the header's compact_volume_points)."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    internal = open(os.path.join(os.path.dirname(HEADER), "hopu_internal.h")).read()
    for k in (3, 4, 5):
        X, _ = _rule(k)
        assert bench.COMPACT_VOLUME_POINTS[(3, k)] == X.shape[0]
        assert f"k == {k} ? {X.shape[0]}" in internal
        assert bench.shape(3, k)["nq_kernel"] == X.shape[0]
