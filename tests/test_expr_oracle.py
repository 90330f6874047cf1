"""Pins of the oracle's expression relations (the paper's non-polynomial
relations, Sec. 2.1 and Sec. 2.4): the postfix interpreter against the same
formulas written directly in Python, special values, the Appendix A plot
decided in exact rational arithmetic, the no-false-negative guarantee of
Sec. 3.4 with a valid tolerance, and undefined points (Sec. 2.4)."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1609_00061_gb300 import workloads as W
from paper_1609_00061_gb300.workloads import (Ex, abs_, atan_, cos_, cosh_, exp_, log_, sin_,
                                              sinh_, sqrt_, tan_, tanh_)

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

x, y, z = Ex.port(0), Ex.port(1), Ex.port(2)

# (program built with the operators, the same formula in Python)
FORMULAS = [
    (x - y, lambda a, b, c: a - b),
    (y - x, lambda a, b, c: b - a),
    (x / y, lambda a, b, c: a / b),
    (2.5 / x - y * 3.0, lambda a, b, c: 2.5 / a - b * 3.0),
    (x ** 3 - 2 * x * y + z, lambda a, b, c: a * a * a - 2 * a * b + c),
    (x ** -2 + 1, lambda a, b, c: 1.0 / (a * a) + 1),
    (x ** 0 + y, lambda a, b, c: 1.0 + b),
    (-x + abs_(y - 1.5), lambda a, b, c: -a + abs(b - 1.5)),
    (sqrt_(abs_(x)) * exp_(y / 4), lambda a, b, c: math.sqrt(abs(a)) * math.exp(b / 4)),
    (log_(x * x + 0.1) - sin_(z), lambda a, b, c: math.log(a * a + 0.1) - math.sin(c)),
    (cos_(x + z * y) - y ** 2, lambda a, b, c: math.cos(a + c * b) - b * b),
    (tan_(x) / (y - 3.0), lambda a, b, c: math.tan(a) / (b - 3.0)),
    (sinh_(x) + cosh_(y) - tanh_(z), lambda a, b, c: math.sinh(a) + math.cosh(b) - math.tanh(c)),
    (atan_(x / (z + 4.0)) * 2, lambda a, b, c: math.atan(a / (c + 4.0)) * 2),
    (abs_(x) ** y, lambda a, b, c: abs(a) ** b),
    (1.0 - (2.0 - (3.0 - x)), lambda a, b, c: 1.0 - (2.0 - (3.0 - a))),
]


@pytest.mark.parametrize("k", range(len(FORMULAS)))
def test_interpreter_matches_direct_formula(orc, k):
    """Operand order, arity and every instruction: the postfix interpreter
    gives the value of the formula written out (a dropped term, a swapped
    operand or a wrong op fails here)."""
    e, f = FORMULAS[k]
    ops, consts = e.program()
    rng = np.random.default_rng(40 + k)
    for _ in range(200):
        p = rng.uniform(-2.0, 2.0, 3)
        got = orc.eval_expr(ops, consts, p)
        try:
            want = f(*p)
        except (ValueError, ZeroDivisionError, OverflowError):
            want = math.nan
        if math.isnan(want):
            assert math.isnan(got) or not math.isfinite(got)
            continue
        assert got == pytest.approx(want, rel=1e-13, abs=1e-13), (k, p)


def test_special_values(orc):
    cases = [(exp_(x), 0.0, 1.0), (log_(x), 1.0, 0.0), (tan_(x), 0.0, 0.0), (cosh_(x), 0.0, 1.0),
             (sqrt_(x), 4.0, 2.0), (sqrt_(x), 2.25, 1.5), (x ** 5, 2.0, 32.0),
             (x ** -3, 2.0, 0.125), (abs_(x), -7.0, 7.0), (sinh_(x), 0.0, 0.0),
             (atan_(x), 0.0, 0.0), (cos_(x), 0.0, 1.0)]
    for e, at, want in cases:
        ops, consts = e.program()
        assert orc.eval_expr(ops, consts, [at, 0.0, 0.0]) == want
    # magnitudes: the largest value pushed
    ops, consts = (x * 100.0 - 1e6).program()
    f, mag = orc.eval_expr(ops, consts, [2.0, 0, 0], with_mag=True)
    assert f == 200.0 - 1e6 and mag == 1e6


def test_undefined_points_are_off(orc):
    """ln of a negative number and division by zero give NaN or Inf: off."""
    ops, consts = log_(x).program()
    p = orc.plot_expr(ops, consts, W.KIND_LE, 10.0, [-2.0], [2.0], [8])
    assert list(p) == [0, 0, 0, 0, 1, 1, 1, 1]
    ops, consts = (1.0 / (x * x) - 1.0e300 * 1e10).program()   # -inf everywhere: off
    p = orc.plot_expr(ops, consts, W.KIND_LE, 1.0, [-1.0], [1.0], [4])
    assert p.sum() == 0


def test_appendix_a_plot_as_expression(orc):
    """Appendix A's M1 = [|y - x^2| < 0.05] written as an expression: the pixel
    decisions of the exact rational arithmetic (borderline pixels excepted)."""
    g = json.load(open(os.path.join(GOLDEN, "appendix_a.json")))
    lo, hi, r, tol = g["lower"], g["upper"], g["resolution"], g["tol"]
    ops, consts = (y - x ** 2).program()
    m1 = orc.plot_expr(ops, consts, 0, tol, [lo, lo], [hi, hi], [r, r], strict=True)
    step = (Fraction(hi) - Fraction(lo)) / r
    for i in range(1, r + 1):
        for j in range(1, r + 1):
            xx = Fraction(lo) + (i - Fraction(1, 2)) * step
            yy = Fraction(lo) + (j - Fraction(1, 2)) * step
            v = abs(yy - xx * xx)
            if abs(v - Fraction(tol)) < Fraction(1, 10 ** 12):
                continue
            assert m1[i - 1, j - 1] == int(v < Fraction(tol)), (i, j)


@pytest.mark.parametrize("res", [37, 64, 200])
def test_no_false_negative_with_valid_tolerance(orc, res):
    """Sec. 3.4: with a valid tolerance every pixel that holds a point of the
    solution set is on.  cos(x) - y = 0 on [-3, 3)^2: |df/dx| <= 1 and
    |df/dy| = 1, so eps = (dx + dy) / 2 is valid (mean value theorem in the
    max norm); the points (t, cos t) must all land in on pixels."""
    ops, consts = (cos_(x) - y).program()
    d = 6.0 / res
    eps = d * (1 + 2 ** -20)
    p = orc.plot_expr(ops, consts, W.KIND_EQ, eps, [-3.0, -3.0], [3.0, 3.0], [res, res])
    for t in np.linspace(-2.999, 2.999, 4001):
        i = int((t + 3.0) / d)
        j = int((math.cos(t) + 3.0) / d)
        assert p[i, j] == 1, (t, i, j)


def test_solve_with_expressions_matches_brute_force(orc):
    """The oracle's solve on a small expression system equals Algorithm 1 run
    on the same plots (any tree gives the same result, Sec. 3.3)."""
    sy = W.input_exemplar(eps=0.1)
    small = W.System("exemplar_small", [(a, b, 8) for a, b, _ in sy.axes], sy.rels, sy.exposed)
    plots = [orc.plot_relation(r, small.axes) for r in small.rels]
    link_res = [a[2] for a in small.axes]
    want = orc.gam(link_res, [p.data for p in plots], [p.vars for p in plots], small.exposed)
    got = orc.solve(small.axes, small.rels, small.exposed).data
    assert np.array_equal(got, want)


# ------------------------------------------------------- counting semiring
@pytest.mark.parametrize("case", [((0, 1), (1, 2), (0, 2), {0: 5, 1: 7, 2: 3}),
                                  ((0, 1, 2), (2, 1, 3), (0, 3), {0: 4, 1: 3, 2: 5, 3: 6}),
                                  ((0, 1, 2), (0, 2, 3), (3, 0, 1), {0: 2, 1: 4, 2: 6, 3: 3}),
                                  ((0, 1), (1, 2), (2,), {0: 4, 1: 5, 2: 3}),
                                  ((1, 0), (1, 0), (), {0: 6, 1: 7})])
def test_oracle_count_against_einsum(orc, case):
    """The counting cluster (Sec. 2.2 footnote) against numpy's integer einsum,
    and its support against the Boolean cluster."""
    xv, yv, keep, rmap = case
    rng = np.random.default_rng(len(xv) * 10 + len(keep))
    vres = [rmap[v] for v in range(max(rmap) + 1)]
    X = (rng.random([rmap[v] for v in xv]) < 0.5).astype(np.uint8)
    Y = (rng.random([rmap[v] for v in yv]) < 0.5).astype(np.uint8)
    letters = "abcdefgh"
    spec = (''.join(letters[v] for v in xv) + "," + ''.join(letters[v] for v in yv) + "->"
            + ''.join(letters[v] for v in keep))
    want = np.einsum(spec, X.astype(np.int64), Y.astype(np.int64))
    got = orc.contract_count(orc.Arr(X, xv), orc.Arr(Y, yv), keep, vres)
    assert np.array_equal(got.astype(np.int64), want)
    boolean = orc.contract(orc.Arr(X, xv), orc.Arr(Y, yv), keep, vres).data
    assert np.array_equal(boolean, (want > 0).astype(np.uint8))


def test_oracle_count_circle_parabola(orc):
    """x^2 + y^2 = 1 and y = z^2 - 1/2: for (x, z) pixels near a solution the
    number of y pixels shared by both plots is small and positive; everywhere
    the count is zero exactly where the Boolean product is off."""
    sy = W.circle_parabola(res=64)
    a, b = (orc.plot_relation(r, sy.axes) for r in sy.rels)
    cnt = orc.contract_count(a, b, (0, 2), [64, 64, 64])
    boolean = orc.solve(sy.axes, sy.rels, sy.exposed).data
    assert np.array_equal(cnt > 0, boolean > 0)
    assert 0 < cnt.max() <= 64
