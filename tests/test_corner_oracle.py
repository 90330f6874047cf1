"""Pins of the oracle's corner-lattice plot (an optional sample rule beside
the paper's centre rule of Sec. 3.2): closed forms on linear relations
(which corners a pixel has, the sign-change clause, the comparison kinds and
the strict flag), brute force in exact rational arithmetic at the lattice
points, the diagonal of a repeated variable, expression relations, non-finite
corner values, and the no-false-negative guarantee of a valid tolerance
(full pixel width instead of half)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1609_00061_gb300 import workloads as W
from paper_1609_00061_gb300.workloads import Ex


def glex(n, degree):
    """Monomial exponent tuple -> coefficient index in graded lex order (total
    degree ascending, tuples of one degree in descending lex order)."""
    from itertools import product
    order = []
    for t in range(degree + 1):
        order += sorted((e for e in product(range(t + 1), repeat=n) if sum(e) == t), reverse=True)
    return {e: k for k, e in enumerate(order)}


def lattice(lo, hi, res):
    """The lattice coordinates as the rule defines them (one product, one sum)."""
    d = (hi - lo) / res
    return [lo + float(i) * d for i in range(res + 1)]


def closed_eq(cs, a, eps, strict=False):
    """f = x - a, kind EQ, exact: some corner within eps of a, or a strictly
    between the pixel's two corners."""
    out = []
    for i in range(len(cs) - 1):
        near = any((abs(Fraction(c) - Fraction(a)) < Fraction(eps)) if strict
                   else (abs(Fraction(c) - Fraction(a)) <= Fraction(eps))
                   for c in (cs[i], cs[i + 1]))
        out.append(int(near or cs[i] < a < cs[i + 1]))
    return np.array(out, dtype=np.uint8)


@pytest.mark.parametrize("a,eps,strict", [
    (0.3, 0.0, False), (0.25, 0.0, False), (0.25, 0.0, True), (-2.0, 0.0, False),
    (2.0, 0.0, False),
    (0.3125, 0.125, False), (0.3125, 0.0625, False), (0.3125, 0.0625, True),
    (-1.0625, 0.5, False), (5.0, 0.5, False), (1.7, 0.3, True)])
def test_linear_eq_closed_form(orc, a, eps, strict):
    """1-D f = x - a on [-2, 2) at 16 pixels (a dyadic lattice): which pixels
    are on follows from the two corners of each pixel; a at a lattice point
    turns both neighbours on, a inside one pixel turns it on by the sign
    change alone (eps = 0), and the strict flag drops corners exactly eps away
    (a corner value of exactly 0 has no sign: strict with eps = 0 leaves a
    lattice-point root off)."""
    got = orc.plot_corner([0], 1, W.KIND_EQ, eps, [-2.0], [2.0], [16], strict,
                          degree=1, coeffs=[-a, 1.0])
    want = closed_eq(lattice(-2.0, 2.0, 16), a, eps, strict)
    assert np.array_equal(got, want)
    if a == 0.3 and eps == 0.0:
        assert np.flatnonzero(got).tolist() == [9]
    if a == 0.25 and eps == 0.0:
        assert np.flatnonzero(got).tolist() == ([] if strict else [8, 9])


@pytest.mark.parametrize("kind", [W.KIND_LE, W.KIND_LT])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_linear_inequalities_closed_form(orc, kind, sign):
    """f = sign (x - a) <= eps (or < eps): on iff the pixel's lower corner
    (sign +1) or its upper corner (sign -1) satisfies it: both corners of
    every pixel are visited, and no sign-change clause applies to S = (-inf, 0]."""
    a, eps = 0.375, 0.25
    cs = lattice(-2.0, 2.0, 16)
    got = orc.plot_corner([0], 1, kind, eps, [-2.0], [2.0], [16], False,
                          degree=1, coeffs=[-sign * a, sign])
    want = []
    for i in range(16):
        vals = [sign * (c - a) for c in (cs[i], cs[i + 1])]
        want.append(int(any((v < eps) if kind == W.KIND_LT else (v <= eps) for v in vals)))
    assert np.array_equal(got, np.array(want, dtype=np.uint8))
    # by hand: sign +1 and <= gives x_i <= 0.625, pixels 0..10
    if sign > 0 and kind == W.KIND_LE:
        assert np.flatnonzero(got).tolist() == list(range(11))


def test_axis_orientation(orc):
    """Two variables, f depending on one of them: the plot is constant along
    the other axis and follows the 1-D closed form along its own (first
    variable slowest)."""
    lo, hi, res = [-2.0, -1.0], [2.0, 3.0], [16, 8]
    # f(x, y) = x - 0.3 (coefficients 1, x, y)
    gx = orc.plot_corner([0, 1], 2, W.KIND_EQ, 0.0, lo, hi, res, degree=1,
                         coeffs=[-0.3, 1.0, 0.0])
    want_x = closed_eq(lattice(-2.0, 2.0, 16), 0.3, 0.0)
    assert np.array_equal(gx, np.repeat(want_x[:, None], 8, axis=1))
    # f(x, y) = y - 1.2
    gy = orc.plot_corner([0, 1], 2, W.KIND_EQ, 0.0, lo, hi, res, degree=1,
                         coeffs=[-1.2, 0.0, 1.0])
    want_y = closed_eq(lattice(-1.0, 3.0, 8), 1.2, 0.0)
    assert np.array_equal(gy, np.repeat(want_y[None, :], 16, axis=0))


def exact_poly(n, degree, coeffs, x):
    """Exact rational value of the polynomial (graded lex order) at x."""
    val = Fraction(0)
    xs = [Fraction(v) for v in x]
    for e, k in glex(n, degree).items():
        term = Fraction(coeffs[k])
        for q in range(n):
            term *= xs[q] ** e[q]
        val += term
    return val


def brute_corner(n, degree, coeffs, kind, eps, lo, hi, res, strict, port_var, nv, tol):
    """Exact-rational corner plot at the float lattice; -1 where a corner value
    lies closer than tol to eps or to 0 (rounding may decide those either way;
    tol = 0 when the float evaluation is exact)."""
    from itertools import product
    lat = [lattice(lo[k], hi[k], res[k]) for k in range(nv)]
    vals = {}
    for idx in product(*[range(r + 1) for r in res]):
        x = [lat[port_var[p]][idx[port_var[p]]] for p in range(n)]
        vals[idx] = exact_poly(n, degree, coeffs, x)
    out = np.zeros(tuple(res), dtype=np.int8)
    feps = Fraction(eps)
    for pix in product(*[range(r) for r in res]):
        on = pos = neg = False
        unsure = False
        for m in range(1 << nv):
            c = tuple(pix[k] + ((m >> k) & 1) for k in range(nv))
            f = vals[c]
            d = abs(f) if kind == W.KIND_EQ else f
            if abs(d - feps) < tol or (kind == W.KIND_EQ and abs(f) < tol):
                unsure = True
            if (d < feps) if (strict or kind == W.KIND_LT) else (d <= feps):
                on = True
            pos |= f > 0
            neg |= f < 0
        v = int(on or (kind == W.KIND_EQ and pos and neg))
        out[pix] = -1 if unsure else v
    return out


@pytest.mark.parametrize("case", range(6))
def test_random_polynomials_exact_rationals(orc, case):
    """Random cubics of 2 and 3 variables on boxes whose lattice is not dyadic,
    ragged resolutions, every kind: every pixel not within rounding of a
    threshold agrees with the exact rational decision at its corners."""
    rng = np.random.default_rng(700 + case)
    n = 2 if case < 4 else 3
    res = [int(v) for v in rng.integers(5, 12 if n == 2 else 7, n)]
    lo = [float(v) for v in rng.uniform(-3.0, -0.5, n)]
    hi = [float(v) for v in rng.uniform(0.5, 3.0, n)]
    coeffs = rng.standard_normal(W.coeff_count(n, 3))
    kind = [W.KIND_EQ, W.KIND_LE, W.KIND_LT, W.KIND_EQ, W.KIND_EQ, W.KIND_LE][case]
    eps = float(rng.uniform(0.05, 0.6))
    strict = case == 3
    got = orc.plot_corner(list(range(n)), n, kind, eps, lo, hi, res, strict, degree=3,
                          coeffs=coeffs)
    want = brute_corner(n, 3, coeffs, kind, eps, lo, hi, res, strict, list(range(n)), n,
                        Fraction(1, 10 ** 9))
    sure = want >= 0
    assert sure.mean() > 0.9
    assert np.array_equal(got[sure], want[sure].astype(np.uint8))
    assert 0 < got.sum() < got.size


def test_repeated_variable_diagonal(orc):
    """A variable on two ports: the corners are those of the pixel over the
    distinct variables.  f(x, x, y) = x * x' - y equals g(x, y) = x^2 - y,
    exactly on a dyadic lattice, and both agree with exact rationals."""
    lo, hi, res = [-2.0, -1.0], [2.0, 3.0], [16, 16]
    # ports (x, x, y), degree 2: coefficients of 1, a, b, c, a^2, ab, ac, b^2, bc, c^2
    f = np.zeros(W.coeff_count(3, 2))
    f[glex(3, 2)[(1, 1, 0)]] = 1.0
    f[glex(3, 2)[(0, 0, 1)]] = -1.0
    g = np.zeros(W.coeff_count(2, 2))
    g[glex(2, 2)[(2, 0)]] = 1.0
    g[glex(2, 2)[(0, 1)]] = -1.0
    for eps in (0.0, 0.3):
        a = orc.plot_corner([0, 0, 1], 2, W.KIND_EQ, eps, lo, hi, res, degree=2, coeffs=f)
        b = orc.plot_corner([0, 1], 2, W.KIND_EQ, eps, lo, hi, res, degree=2, coeffs=g)
        assert np.array_equal(a, b)
        want = brute_corner(3, 2, f, W.KIND_EQ, eps, lo, hi, res, False, [0, 0, 1], 2,
                            Fraction(0))
        assert np.array_equal(a, want.astype(np.uint8))
        assert a.sum() > 0


def test_expression_matches_polynomial(orc):
    """The same relation as an expression program and as a polynomial: on a
    dyadic lattice both evaluate exactly, so the corner plots are equal."""
    x, y = Ex.port(0), Ex.port(1)
    ops, consts = (x * x + y * y - 1.0).program()
    c = np.zeros(W.coeff_count(2, 2))
    c[0] = -1.0
    c[glex(2, 2)[(2, 0)]] = 1.0
    c[glex(2, 2)[(0, 2)]] = 1.0
    lo, hi, res = [-2.0, -2.0], [2.0, 2.0], [32, 32]
    for kind, eps in ((W.KIND_EQ, 0.0), (W.KIND_EQ, 0.2), (W.KIND_LE, 0.0)):
        a = orc.plot_corner([0, 1], 2, kind, eps, lo, hi, res, expr=(ops, consts))
        b = orc.plot_corner([0, 1], 2, kind, eps, lo, hi, res, degree=2, coeffs=c)
        assert np.array_equal(a, b) and a.sum() > 0


def test_non_finite_corners_take_no_part(orc):
    """f = 1/x with a corner exactly at x = 0: that corner's value is +Inf and
    counts neither as a value within eps nor as a sign, so no pixel turns on
    (a non-finite corner taken as positive would light the pixel left of 0)."""
    x = Ex.port(0)
    ops, consts = (1.0 / x).program()
    got = orc.plot_corner([0], 1, W.KIND_EQ, 0.0, [-2.0], [2.0], [16], expr=(ops, consts))
    assert got.sum() == 0
    # f = x - 0.3 written with a 0/0 term that is NaN only at x = 0: the
    # pixel [0.25, 0.5) still turns on by its sign change, and the pixel
    # [0, 0.25) (corner 0 is NaN, corner 0.25 is negative) stays off
    ops, consts = (x - 0.3 + (x - x) / x).program()
    got = orc.plot_corner([0], 1, W.KIND_EQ, 0.0, [-2.0], [2.0], [16], expr=(ops, consts))
    assert np.flatnonzero(got).tolist() == [9]


def test_tolerance_uses_full_width(orc):
    """The corner tolerance is twice the centre one (scaling by 2 is exact),
    and for a linear f = a x + b y + c it is (|a| dx + |b| dy)(1 + 2^-30)."""
    rng = np.random.default_rng(9)
    for n, deg in ((2, 3), (3, 3), (1, 5)):
        c = rng.standard_normal(W.coeff_count(n, deg))
        lo = list(rng.uniform(-3, -1, n))
        hi = list(rng.uniform(1, 3, n))
        res = [int(v) for v in rng.integers(20, 300, n)]
        e0 = orc.valid_tolerance(deg, c, lo, hi, res)
        e1 = orc.valid_tolerance(deg, c, lo, hi, res, corner=True)
        assert e1 == 2.0 * e0
    a, b = 1.75, -0.5
    e = orc.valid_tolerance(1, [0.25, a, b], [-1.0, -2.0], [1.0, 2.0], [8, 16], corner=True)
    assert e == pytest.approx((abs(a) * 0.25 + abs(b) * 0.25) * (1 + 2.0 ** -30), rel=1e-15)


def test_no_false_negatives_with_valid_tolerance(orc):
    """With the corner tolerance, every pixel that holds a solution is on
    (circle points, and roots of a random cubic found numerically along y)."""
    c = np.zeros(W.coeff_count(2, 2))
    c[0] = -1.0
    c[glex(2, 2)[(2, 0)]] = 1.0
    c[glex(2, 2)[(0, 2)]] = 1.0
    lo, hi, res = [-2.0, -2.0], [2.0, 2.0], [64, 64]
    eps = orc.valid_tolerance(2, c, lo, hi, res, corner=True)
    p = orc.plot_corner([0, 1], 2, W.KIND_EQ, eps, lo, hi, res, degree=2, coeffs=c)
    for t in np.linspace(0.0, 2 * math.pi, 997):
        px, py = math.cos(t), math.sin(t)
        i, j = int((px + 2.0) / 4.0 * 64), int((py + 2.0) / 4.0 * 64)
        assert p[i, j] == 1
    rng = np.random.default_rng(31)
    cc = rng.standard_normal(W.coeff_count(2, 3))
    lo, hi, res = [-3.0, -3.0], [3.0, 3.0], [96, 80]
    eps = orc.valid_tolerance(3, cc, lo, hi, res, corner=True)
    p = orc.plot_corner([0, 1], 2, W.KIND_EQ, eps, lo, hi, res, degree=3, coeffs=cc)
    hits = 0
    for x0 in rng.uniform(-2.9, 2.9, 300):
        # f(x0, y) as a cubic in y: coefficient of y^j gathers c_e x0^(e_x), e_y = j
        py = np.zeros(4)
        for ex in range(4):
            for ey in range(4 - ex):
                py[ey] += cc[glex(2, 3)[(ex, ey)]] * x0 ** ex
        for r in np.roots(py[::-1]):
            if abs(r.imag) < 1e-12 and -3.0 < r.real < 3.0:
                i = int((x0 + 3.0) / 6.0 * 96)
                j = int((r.real + 3.0) / 6.0 * 80)
                assert p[i, j] == 1
                hits += 1
    assert hits > 50
