"""Pins for the CPU oracle against facts it does not compute itself.

Every check here compares the oracle with something independent of its code:
exact rational arithmetic, a brute-force loop written out in Python, numpy's
integer matmul / einsum / kron, closed-form solution sets, or the accuracy
guarantees of Sec. 3.2 and Thm. (extended accuracy), Sec. 3.4.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1609_00061_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ------------------------------------------------------------ polynomial format
def graded_lex(n, degree):
    """Graded lex order written out independently: by total degree, then
    descending lexicographic exponent tuples."""
    out = []
    for t in range(degree + 1):
        tup = [e for e in itertools.product(range(t + 1), repeat=n) if sum(e) == t]
        out.extend(sorted(tup, reverse=True))
    return out


@pytest.mark.parametrize("n,degree", [(1, 3), (2, 3), (3, 2), (3, 3), (4, 2)])
def test_coefficient_order(orc, n, degree):
    order = graded_lex(n, degree)
    assert orc.coeff_count(n, degree) == len(order) == math.comb(n + degree, degree)
    for i, e in enumerate(order):
        assert orc.coeff_index(e, degree) == i
    if n == 2 and degree == 3:
        assert order == [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (3, 0), (2, 1), (1, 2), (0, 3)]


def exact_poly(coeffs, degree, x):
    n = len(x)
    s = Fraction(0)
    for c, e in zip(coeffs, graded_lex(n, degree)):
        term = Fraction(c)
        for xi, ei in zip(x, e):
            term *= Fraction(xi) ** ei
        s += term
    return s


def test_eval_exact_on_dyadic_points(orc):
    """Small integer coefficients at dyadic points: every FP64 operation is exact,
    so the nested evaluation must equal the exact rational value."""
    rng = np.random.default_rng(1)
    for n, degree in [(1, 4), (2, 3), (3, 3), (4, 2)]:
        m = math.comb(n + degree, degree)
        for _ in range(20):
            c = rng.integers(-7, 8, m).astype(np.float64)
            x = rng.integers(-12, 13, n) / 8.0
            assert orc.eval_poly(degree, c, x) == float(exact_poly(c, degree, x))


def test_eval_close_on_random_points(orc):
    rng = np.random.default_rng(2)
    for n, degree in [(2, 3), (3, 3)]:
        m = math.comb(n + degree, degree)
        for _ in range(50):
            c = rng.normal(size=m)
            x = rng.uniform(-3, 3, n)
            ex = exact_poly(c, degree, x)
            scale = float(exact_poly(np.abs(c), degree, np.abs(x)))
            assert abs(orc.eval_poly(degree, c, x) - float(ex)) <= 64 * 2.0 ** -53 * scale


# ------------------------------------------------------------- valid tolerance
def test_tolerance_closed_form_circle(orc):
    # f = x^2 + y^2 - 1 on [-2,2)^2 at 256: |df/dx| <= 2*2 = 4, delta = 1/64,
    # eps = (4 * 1/128 + 4 * 1/128) * (1 + 2^-30)
    eps = orc.valid_tolerance(2, [-1, 0, 0, 1, 0, 1], [-2, -2], [2, 2], [256, 256])
    assert Fraction(eps) == Fraction(1, 16) * (1 + Fraction(1, 2 ** 30))


def test_tolerance_linear_is_exact_sup(orc):
    # f = a + b x + c y: sup over a pixel of |f(p) - f(centre)| = |b| dx/2 + |c| dy/2
    a, b, c = 0.25, -3.0, 1.5
    lo, hi, res = [-1.0, 0.0], [1.0, 4.0], [8, 32]
    eps = orc.valid_tolerance(1, [a, b, c], lo, hi, res)
    want = (Fraction(3) * Fraction(2, 8) / 2 + Fraction(3, 2) * Fraction(4, 32) / 2)
    assert Fraction(eps) == want * (1 + Fraction(1, 2 ** 30))


def test_tolerance_is_valid_by_sampling(orc):
    """Eq. (continuity) at the pixel radius: |f(x) - f(c)| <= eps for x in the pixel."""
    rng = np.random.default_rng(3)
    for n in (1, 2, 3):
        m = math.comb(n + 3, 3)
        for _ in range(10):
            c = rng.normal(size=m)
            lo = rng.uniform(-3, 0, n)
            hi = lo + rng.uniform(0.5, 3, n)
            res = rng.integers(2, 40, n)
            eps = orc.valid_tolerance(3, c, lo, hi, res)
            d = (hi - lo) / res
            for _ in range(200):
                idx = np.array([rng.integers(0, r) for r in res])
                centre = lo + (idx + 0.5) * d
                x = centre + (rng.uniform(-0.5, 0.5, n) * d)
                diff = abs(float(exact_poly(c, 3, x)) - float(exact_poly(c, 3, centre)))
                assert diff <= eps


# --------------------------------------------------------------------- plots
def test_appendix_a_plot_exact(orc):
    """Appendix A: M1 = [|y - x^2| < 0.05] at pixel centres of Dim(-1.2,1.2,50),
    decided here in exact rational arithmetic (1-based centre (i - 1/2) * step)."""
    g = json.load(open(os.path.join(GOLDEN, "appendix_a.json")))
    lo, hi, r, tol = g["lower"], g["upper"], g["resolution"], g["tol"]
    m1 = orc.plot(2, g["m1_coeffs_graded_lex"], 0, tol, [lo, lo], [hi, hi], [r, r], strict=True)
    step = (Fraction(hi) - Fraction(lo)) / r
    close = 0
    for i in range(1, r + 1):
        for j in range(1, r + 1):
            x = Fraction(lo) + (i - Fraction(1, 2)) * step
            y = Fraction(lo) + (j - Fraction(1, 2)) * step
            v = abs(y - x * x)
            if abs(v - Fraction(tol)) < Fraction(1, 10 ** 12):
                close += 1
                continue
            assert m1[i - 1, j - 1] == int(v < Fraction(tol)), (i, j)
    assert close <= 4
    assert 0 < m1.sum() < r * r // 4


def test_appendix_a_product_is_circle(orc):
    """M1*M2 of Appendix A against numpy integer matmul, and the circle x^2+z^2=1:
    every (x, z) pixel whose y-column holds a common on pixel is on, nothing else."""
    g = json.load(open(os.path.join(GOLDEN, "appendix_a.json")))
    lo, hi, r, tol = g["lower"], g["upper"], g["resolution"], g["tol"]
    m1 = orc.plot(2, g["m1_coeffs_graded_lex"], 0, tol, [lo, lo], [hi, hi], [r, r], strict=True)
    m2 = orc.plot(2, g["m2_coeffs_graded_lex"], 0, tol, [lo, lo], [hi, hi], [r, r], strict=True)
    prod = orc.contract(orc.Arr(m1, (0, 1)), orc.Arr(m2, (1, 2)), (0, 2), [r, r, r])
    want = (m1.astype(np.int64) @ m2.astype(np.int64)) > 0
    assert np.array_equal(prod.data, want.astype(np.uint8))
    # the product pixels lie near the unit circle
    c = lo + (np.arange(r) + 0.5) * (hi - lo) / r
    xs, zs = np.nonzero(prod.data)
    rad = np.hypot(c[xs], c[zs])
    assert prod.data.sum() > 20 and np.all(np.abs(rad - 1.0) < 0.2)


def test_plot_kinds_and_strict(orc):
    # f = x on [-1,1) @ 8: centres -0.875 ... 0.875
    c = [0.0, 1.0]
    xs = -1 + (np.arange(8) + 0.5) * 0.25
    eq = orc.plot(1, c, W.KIND_EQ, 0.125, [-1], [1], [8])
    le = orc.plot(1, c, W.KIND_LE, 0.125, [-1], [1], [8])
    lt = orc.plot(1, c, W.KIND_LT, 0.125, [-1], [1], [8])
    eqs = orc.plot(1, c, W.KIND_EQ, 0.125, [-1], [1], [8], strict=True)
    assert eq.tolist() == (np.abs(xs) <= 0.125).astype(int).tolist()
    assert le.tolist() == (xs <= 0.125).astype(int).tolist()
    assert lt.tolist() == (xs < 0.125).astype(int).tolist()
    assert eqs.tolist() == (np.abs(xs) < 0.125).astype(int).tolist()
    # the boundary case: eps exactly |f(c)|
    e2 = orc.plot(1, c, W.KIND_EQ, 0.125, [-0.25], [0.25], [2])   # centres -0.125, 0.125
    e2s = orc.plot(1, c, W.KIND_EQ, 0.125, [-0.25], [0.25], [2], strict=True)
    assert e2.tolist() == [1, 1] and e2s.tolist() == [0, 0]


def test_plot_nonfinite_is_off(orc):
    # f = 1e300 * x^2 overflows to inf away from 0: those pixels must be off even for <=
    big = orc.plot(2, [0.0, 0.0, 1e300], W.KIND_LE, 1.0, [-1e10], [1e10], [4])
    assert big.tolist() == [0, 0, 0, 0]
    neg = orc.plot(2, [0.0, 0.0, -1e300], W.KIND_LE, 1.0, [-1e10], [1e10], [4])
    assert neg.tolist() == [0, 0, 0, 0]  # -inf is not finite either


def test_plot_axis_orientation(orc):
    # f(x, y) = x - 0.95 on [0,1)^2 @ 10 with eps 0.01: only the row x-index 9 is on
    p = orc.plot(1, [-0.95, 1.0, 0.0], 0, 0.01, [0, 0], [1, 1], [10, 10])
    assert p[9].all() and p[:9].sum() == 0


def test_accuracy_guarantees_sampled(orc):
    """Sec. 3.2, epsilon-accurate plot: (1) a pixel containing a zero is on,
    (3) on pixels have |f| <= 2 eps everywhere in the pixel."""
    rng = np.random.default_rng(4)
    for trial in range(6):
        c = rng.normal(size=10)
        lo, hi, r = np.array([-2.0, -2.0]), np.array([2.0, 2.0]), np.array([37, 29])
        eps = orc.valid_tolerance(3, c, lo, hi, r)
        p = orc.plot(3, c, 0, eps, lo, hi, r)
        d = (hi - lo) / r
        on = np.argwhere(p == 1)
        for (i, j) in on[rng.permutation(len(on))[:100]]:
            for _ in range(5):
                x = lo + (np.array([i, j]) + rng.uniform(0, 1, 2)) * d
                assert abs(float(exact_poly(c, 3, x))) <= 2 * eps
        # zeros on random horizontal lines (bisection in exact arithmetic)
        for _ in range(30):
            y = rng.uniform(-2, 2)
            xs = np.linspace(-2, 2, 400, endpoint=False)
            vals = [float(exact_poly(c, 3, (x, y))) for x in xs]
            for a, b, fa, fb in zip(xs[:-1], xs[1:], vals[:-1], vals[1:]):
                if fa == 0 or fa * fb < 0:
                    lo_, hi_ = a, b
                    for _ in range(60):
                        mid = 0.5 * (lo_ + hi_)
                        if float(exact_poly(c, 3, (lo_, y))) * float(exact_poly(c, 3, (mid, y))) <= 0:
                            hi_ = mid
                        else:
                            lo_ = mid
                    xr = 0.5 * (lo_ + hi_)
                    i = int(math.floor((xr + 2) / d[0]))
                    j = int(math.floor((y + 2) / d[1]))
                    if 0 <= i < r[0] and 0 <= j < r[1]:
                        assert p[i, j] == 1


# --------------------------------------------------------------------- GAM
def brute_gam(link_res, arrays, port_links, out_links):
    """Algorithm 1, written out a second time in plain Python."""
    out = np.zeros(tuple(link_res[l] for l in out_links), dtype=np.uint8)
    for e in itertools.product(*[range(r) for r in link_res]):
        a = 1
        for A, pl in zip(arrays, port_links):
            a &= int(A[tuple(e[l] for l in pl)])
        if a:
            out[tuple(e[l] for l in out_links)] = 1
    return out


def test_gam_matches_python_algorithm_1(orc):
    rng = np.random.default_rng(5)
    for trial in range(40):
        nl = int(rng.integers(1, 6))
        link_res = [int(v) for v in rng.integers(2, 5, nl)]
        na = int(rng.integers(1, 4))
        port_links = []
        for _ in range(na):
            k = int(rng.integers(0, min(3, nl) + 1))
            port_links.append([int(v) for v in rng.integers(0, nl, k)])
        nout = int(rng.integers(0, min(3, nl) + 1))
        out_links = [int(v) for v in rng.permutation(nl)[:nout]]
        arrays = [(rng.random(tuple(link_res[l] for l in pl)) < 0.5).astype(np.uint8)
                  for pl in port_links]
        got = orc.gam(link_res, arrays, port_links, out_links)
        assert np.array_equal(got, brute_gam(link_res, arrays, port_links, out_links))


def test_gam_special_cases_numpy(orc):
    """Sec. 3.3: matrix product, trace and Kronecker product as array multiplications."""
    rng = np.random.default_rng(6)
    A = (rng.random((5, 7)) < 0.3).astype(np.uint8)
    B = (rng.random((7, 4)) < 0.3).astype(np.uint8)
    got = orc.gam([5, 7, 4], [A, B], [[0, 1], [1, 2]], [0, 2])
    assert np.array_equal(got, ((A.astype(int) @ B.astype(int)) > 0).astype(np.uint8))
    S = (rng.random((6, 6)) < 0.2).astype(np.uint8)
    tr = orc.gam([6], [S], [[0, 0]], [])
    assert int(tr) == int(np.trace(S) > 0)
    K = orc.gam([5, 7, 7, 4], [A, B], [[0, 1], [2, 3]], [0, 2, 1, 3])
    assert np.array_equal(K.reshape(35, 28), np.kron(A, B))


def test_contract_pair_vs_numpy(orc):
    rng = np.random.default_rng(7)
    vres = [6, 5, 7, 4, 3]
    A = (rng.random((6, 5, 7)) < 0.25).astype(np.uint8)   # vars 0,1,2
    B = (rng.random((7, 5, 4)) < 0.25).astype(np.uint8)   # vars 2,1,3
    # batched (var 1 kept in both) contraction over var 2
    got = orc.contract(orc.Arr(A, (0, 1, 2)), orc.Arr(B, (2, 1, 3)), (1, 0, 3), vres)
    want = np.einsum("abc,cbd->bad", A.astype(int), B.astype(int)) > 0
    assert np.array_equal(got.data, want.astype(np.uint8))
    # Hadamard
    C = (rng.random((6, 5, 7)) < 0.5).astype(np.uint8)
    got = orc.contract(orc.Arr(A, (0, 1, 2)), orc.Arr(C, (0, 1, 2)), (0, 1, 2), vres)
    assert np.array_equal(got.data, A & C)
    # reduce a private axis
    got = orc.reduce(orc.Arr(A, (0, 1, 2)), (2, 0), vres)
    assert np.array_equal(got.data, A.max(axis=1).T)
    # diagonal read: X(v0, v0)
    D = (rng.random((6, 6)) < 0.5).astype(np.uint8)
    got = orc.contract(orc.Arr(D, (0, 0)), orc.Arr(np.ones((), np.uint8), ()), (0,), vres)
    assert np.array_equal(got.data, np.diag(D))


def test_contract_pair_vs_gam_random(orc):
    rng = np.random.default_rng(8)
    for trial in range(60):
        nv = int(rng.integers(1, 6))
        vres = [int(v) for v in rng.integers(2, 5, nv)]
        xv = [int(v) for v in rng.integers(0, nv, int(rng.integers(0, 4)))]
        yv = [int(v) for v in rng.integers(0, nv, int(rng.integers(0, 4)))]
        allv = sorted(set(xv) | set(yv))
        keep = [int(v) for v in rng.permutation(allv)[:int(rng.integers(0, len(allv) + 1))]]
        X = (rng.random(tuple(vres[v] for v in xv)) < 0.4).astype(np.uint8)
        Y = (rng.random(tuple(vres[v] for v in yv)) < 0.4).astype(np.uint8)
        got = orc.contract(orc.Arr(X, tuple(xv)), orc.Arr(Y, tuple(yv)), tuple(keep), vres)
        want = brute_gam(vres, [X, Y], [xv, yv], keep)
        assert np.array_equal(got.data, want)


def test_monotone_and_order_invariant(orc):
    """Thm. (associativity): every cluster order gives the same array; monotone."""
    rng = np.random.default_rng(9)
    sysm = W.chain(res=12, nrel=4, seed=11)
    ref = orc.solve(sysm.axes, sysm.rels, sysm.exposed)
    for order in itertools.permutations(range(4)):
        assert np.array_equal(orc.solve(sysm.axes, sysm.rels, sysm.exposed, order=order).data,
                              ref.data)
    # whole-network Algorithm 1 on the same plots
    plots = [orc.plot_relation(r, sysm.axes) for r in sysm.rels]
    vres = [a[2] for a in sysm.axes]
    got = orc.gam(vres, [p.data for p in plots], [list(p.vars) for p in plots],
                  list(sysm.exposed))
    assert np.array_equal(got, ref.data)
    # monotonicity: switching pixels on never switches an output pixel off
    bigger = [np.maximum(p.data, (rng.random(p.data.shape) < 0.1).astype(np.uint8))
              for p in plots]
    got2 = orc.gam(vres, bigger, [list(p.vars) for p in plots], list(sysm.exposed))
    assert np.all(got2 >= got)


def test_solve_ternary_orders_agree(orc):
    sysm = W.ternary(res=10)
    ref = orc.solve(sysm.axes, sysm.rels, sysm.exposed)
    for order in [(3, 2, 1, 0), (1, 3, 0, 2), (2, 0, 3, 1)]:
        assert np.array_equal(orc.solve(sysm.axes, sysm.rels, sysm.exposed, order=order).data,
                              ref.data)
    plots = [orc.plot_relation(r, sysm.axes) for r in sysm.rels]
    got = orc.gam([10] * 6, [p.data for p in plots], [list(p.vars) for p in plots], [0, 1, 2])
    assert np.array_equal(got, ref.data)


# ---------------------------------------------------- closed-form solution sets
def _pix(v, lo, hi, r):
    return int(math.floor((v - lo) / ((hi - lo) / r)))


def test_circle_parabola_no_false_negative(orc):
    """x^2 + y^2 = 1, y = z^2 - 1/2: every (x, z) on x^2 + (z^2 - 1/2)^2 = 1 is marked."""
    sysm = W.circle_parabola(res=96)
    out = orc.solve(sysm.axes, sysm.rels, sysm.exposed).data
    lo, hi, r = sysm.axes[0]
    hits = 0
    for z in np.linspace(-1.99, 1.99, 3001):
        y = z * z - 0.5
        if abs(y) > 1:
            continue
        for x in (math.sqrt(1 - y * y), -math.sqrt(1 - y * y)):
            assert out[_pix(x, lo, hi, r), _pix(z, lo, hi, r)] == 1
            hits += 1
    assert hits > 1000
    # and marked pixels are near the solution curve (soundness, loose)
    c = lo + (np.arange(r) + 0.5) * (hi - lo) / r
    xs, zs = np.nonzero(out)
    resid = np.abs(c[xs] ** 2 + (c[zs] ** 2 - 0.5) ** 2 - 1)
    assert resid.max() < 0.5


def test_circle_line_roots(orc):
    """R1: x^2 + y^2 - 1 = 0 and R2: y - (m x + c) = 0 share x and y; expose x.
    The roots of (1 + m^2) x^2 + 2 m c x + c^2 - 1 = 0 must be marked."""
    m, c0 = 0.7, 0.3
    r1 = W.Relation((0, 1), 2, [-1.0, 0.0, 0.0, 1.0, 0.0, 1.0])
    r2 = W.Relation((0, 1), 1, [-c0, -m, 1.0])
    axes = [(-2.0, 2.0, 200), (-2.0, 2.0, 200)]
    out = orc.solve(axes, [r1, r2], (0,)).data
    a, b, cc = 1 + m * m, 2 * m * c0, c0 * c0 - 1
    disc = math.sqrt(b * b - 4 * a * cc)
    roots = [(-b + disc) / (2 * a), (-b - disc) / (2 * a)]
    for x in roots:
        assert out[_pix(x, -2, 2, 200)] == 1
    # all marked x lie near a root
    cx = -2 + (np.nonzero(out)[0] + 0.5) * 0.02
    assert all(min(abs(v - q) for q in roots) < 0.1 for v in cx)


def test_circle_parabola_roots_exposed_x(orc):
    """x^2 + y^2 = 1, y = x^2 - 1/2 (both over x, y); expose x: x = +-(3/4)^(1/4)."""
    r1 = W.Relation((0, 1), 2, [-1.0, 0.0, 0.0, 1.0, 0.0, 1.0])
    r2 = W.Relation((0, 1), 2, [0.5, 0.0, 1.0, -1.0, 0.0, 0.0])
    axes = [(-2.0, 2.0, 160), (-2.0, 2.0, 160)]
    out = orc.solve(axes, [r1, r2], (0,)).data
    root = 0.75 ** 0.25
    for x in (root, -root):
        assert out[_pix(x, -2, 2, 160)] == 1
    cx = -2 + (np.nonzero(out)[0] + 0.5) * 0.025
    assert all(min(abs(v - root), abs(v + root)) < 0.1 for v in cx)


def test_entries_count_example():
    """Sec. 3.1: a pack with three ports of resolution 20 has 20^3 = 8000 entries."""
    assert np.zeros((20, 20, 20), np.uint8).size == 8000


# --------------------------------------------------------- cost-model oracle
def test_mlp_oracle_gradient_central_differences():
    """The oracle's analytic gradient against central differences of its loss."""
    from oracle import mlp as M
    rng = np.random.default_rng(21)
    sizes = M.layer_sizes(16, 12, 3)
    npar = sum(sizes[i + 1] * sizes[i] + sizes[i + 1] for i in range(len(sizes) - 1))
    p = rng.normal(size=npar) * 0.4
    X = rng.normal(size=(37, 16))
    T = rng.normal(size=37)
    L, g = M.loss_and_grad(p, sizes, X, T)
    assert abs(L - M.loss(p, sizes, X, T)) < 1e-12
    h = 1e-6
    for k in rng.choice(npar, 60, replace=False):
        e = np.zeros(npar)
        e[k] = h
        num = (M.loss(p + e, sizes, X, T) - M.loss(p - e, sizes, X, T)) / (2 * h)
        assert abs(num - g[k]) <= 1e-6 * max(1.0, abs(num)), k


def test_mlp_oracle_forward_by_hand():
    """A 1-input, one-hidden-unit network computed by hand."""
    from oracle import mlp as M
    sizes = [1, 1, 1]
    # W1 = 2, b1 = -1, W2 = 3, b2 = 0.5: y = 3 * relu(2x - 1) + 0.5
    p = np.array([2.0, -1.0, 3.0, 0.5])
    y = M.forward(p, sizes, np.array([[0.0], [1.0], [2.0]]))
    assert y.tolist() == [0.5, 3.5, 9.5]


def test_mlp_oracle_adam_first_steps():
    """Adam from zero moments: the bias corrections make the first step
    lr * g / (|g| + eps), i.e. lr * sign(g) for |g| >> eps; a constant gradient
    keeps that step size on later steps; a zero gradient does not move."""
    from oracle import mlp as M
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    p0 = np.array([1.0, 2.0, -1.0, 0.25])
    z = np.zeros(4)
    p1, m1, v1 = M.adam_step(p0, g, z, z, 1, 0.01)
    assert np.allclose(p1[:3], p0[:3] - 0.01 * np.sign(g[:3]), rtol=0, atol=1e-7)
    assert p1[3] == p0[3]
    p2, _, _ = M.adam_step(p1, g, m1, v1, 2, 0.01)
    assert np.allclose(p2[:3] - p1[:3], -0.01 * np.sign(g[:3]), rtol=0, atol=1e-7)


def test_solve_strategies_agree():
    """Smallest-result pairwise joining and left-to-right folding give the same
    array (associativity), on a tree-like random network."""
    import oracle
    net = W.random_networks(1, seed=9, nvars_range=(7, 8), nrel_range=(8, 9),
                            res_choices=(12,))[0]
    a = oracle.solve(net.axes, net.rels, net.exposed, smallest=True).data
    b = oracle.solve(net.axes, net.rels, net.exposed, smallest=False).data
    assert np.array_equal(a, b)
