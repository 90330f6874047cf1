"""GPU parity of expression relations (the paper's non-polynomial relations:
the input exemplar of Sec. 2.1, the butterfly and 3-D arrays examples of
Sec. 2.4).

The device evaluates +, -, *, / and sqrt correctly rounded, like the oracle,
but the elementary functions come from the CUDA math library, whose last bits
may differ from the C library's.  So a plot may differ from the oracle's only
at pixels whose |f| lies within that difference of eps: every differing pixel
must satisfy | d(f) - eps | <= TOL_REL * max(1, mag), d(f) the oracle's
distance to the target set and mag the largest magnitude the oracle's program
pushed at that pixel, and at most a 1e-4 share of the pixels may differ.
Whole solves are compared bit for bit (no plot pixel of these systems falls
in that band)."""
import math

import numpy as np
import pytest

import paper_1609_00061_gb300 as pa
from paper_1609_00061_gb300 import workloads as W
from paper_1609_00061_gb300.workloads import (Ex, abs_, atan_, cos_, cosh_, exp_, log_, sin_,
                                              sinh_, sqrt_, tan_, tanh_)

pytestmark = pytest.mark.gpu

# 2^-30 relative to the largest intermediate: far above the few-ulp
# differences of two math libraries after a short program, far below any
# formula or operand-order mistake
TOL_REL = 2.0 ** -30


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    e = pa.Engine(0)
    yield e
    e.close()


def centres(axes, v):
    lo, hi, r = axes[v]
    return lo + (np.arange(r) + 0.5) * ((hi - lo) / r)


def check_plot_band(orc, rel, axes, got, what=""):
    """The GPU plot against the oracle's: equal except inside the rounding band."""
    want = orc.plot_relation(rel, axes).data
    g = got.to_numpy()
    # plot_relation is over the ports; these relations have distinct ports
    assert g.shape == want.shape, what
    diff = np.argwhere(g != want)
    assert len(diff) <= 5 + 1e-4 * want.size, f"{what}: {len(diff)} pixels differ"
    ops, consts = rel.expr
    for idx in diff:
        pt = [centres(axes, rel.vars[p])[idx[p]] for p in range(len(rel.vars))]
        f, mag = orc.eval_expr(ops, consts, pt, with_mag=True)
        assert math.isfinite(f), (what, idx, f)
        d = abs(f) if rel.kind == W.KIND_EQ else f
        assert abs(d - rel.eps) <= TOL_REL * max(1.0, mag), (what, idx, f, rel.eps, mag)
    assert got.padding_clean(), what
    return len(diff)


# ------------------------------------------------------ random programs
UNARY = [abs_, sqrt_, exp_, log_, sin_, cos_, tan_, sinh_, cosh_, tanh_, atan_]


def random_expr(rng, arity, depth):
    """A random expression tree over the ports, of bounded depth."""
    if depth == 0 or rng.uniform() < 0.25:
        if rng.uniform() < 0.3:
            return Ex.const(float(np.round(rng.normal(), 3)))
        return Ex.port(int(rng.integers(arity)))
    kind = rng.uniform()
    if kind < 0.45:
        a, b = random_expr(rng, arity, depth - 1), random_expr(rng, arity, depth - 1)
        op = int(rng.integers(4))
        return [a + b, a - b, a * b, a / (b * b + 0.5)][op]
    if kind < 0.8:
        f = UNARY[int(rng.integers(len(UNARY)))]
        a = random_expr(rng, arity, depth - 1)
        if f in (sqrt_, log_):
            a = abs_(a) + 0.1
        if f in (exp_, sinh_, cosh_):
            a = tanh_(a) * 3.0
        return f(a)
    a = random_expr(rng, arity, depth - 1)
    return a ** int(rng.integers(-3, 4)) if rng.uniform() < 0.7 else abs_(a) ** 1.5


@pytest.mark.parametrize("seed", range(10))
def test_random_expression_plots(eng, orc, seed):
    rng = np.random.default_rng(9000 + seed)
    arity = int(rng.integers(1, 5))
    res = [int(rng.choice([2, 3, 31, 64, 65, 100, 127])) for _ in range(arity)]
    if arity >= 3:
        res = [min(r, 40) for r in res]
    axes = []
    for r in res:
        a, b = sorted(rng.uniform(-3, 3, 2))
        axes.append((float(a), float(b) + 0.1, r))
    e = random_expr(rng, arity, 4)
    # eps on the scale of the values, so that plots are neither empty nor full
    ops, consts = e.program()
    samples = [orc.eval_expr(ops, consts, rng.uniform([a[0] for a in axes],
                                                      [a[1] for a in axes])) for _ in range(64)]
    finite = [abs(v) for v in samples if math.isfinite(v)]
    eps = float(np.median(finite)) if finite else 0.5
    kind = int(rng.integers(3))
    rel = W.expr_relation(tuple(range(arity)), e, kind=kind, eps=eps)
    got = eng.plot(rel, axes)
    eng.sync()
    check_plot_band(orc, rel, axes, got, f"seed {seed}")


def test_strict_and_kinds(eng, orc):
    """f = x on [-1, 1) at 8: centres -0.875 .. 0.875, ties at eps = 0.125."""
    axes = [(-1.0, 1.0, 8)]
    for kind, strict, want in [(W.KIND_EQ, False, [0, 0, 0, 1, 1, 0, 0, 0]),
                               (W.KIND_EQ, True, [0, 0, 0, 0, 0, 0, 0, 0]),
                               (W.KIND_LE, False, [1, 1, 1, 1, 1, 0, 0, 0]),
                               (W.KIND_LE, True, [1, 1, 1, 1, 0, 0, 0, 0]),
                               (W.KIND_LT, False, [1, 1, 1, 1, 0, 0, 0, 0])]:
        rel = W.expr_relation((0,), Ex.port(0), kind=kind, eps=0.125)
        out = pa.BitArray.empty((0,), (8,))
        pa.pa_plot(eng.ctx, rel, axes, out, strict=strict)
        eng.sync()
        assert list(out.to_numpy()) == want, (kind, strict)
    # ties: centre 0.125 sits exactly on eps
    rel = W.expr_relation((0,), Ex.port(0) - 0.0, kind=W.KIND_EQ, eps=0.375)
    out = eng.plot(rel, axes)
    eng.sync()
    assert list(out.to_numpy()) == [0, 0, 1, 1, 1, 1, 0, 0]


def test_undefined_points_off(eng, orc):
    axes = [(-2.0, 2.0, 64), (-2.0, 2.0, 65)]
    x, y = Ex.port(0), Ex.port(1)
    rel = W.expr_relation((0, 1), log_(x) + 1.0 / y - tan_(x * 20.0), kind=W.KIND_LE, eps=1.0)
    got = eng.plot(rel, axes)
    eng.sync()
    check_plot_band(orc, rel, axes, got, "undefined")
    assert got.to_numpy()[:32].sum() == 0      # ln of a negative number: off


# ------------------------------------------------------ the paper's systems
@pytest.mark.parametrize("make", [lambda: W.butterfly(res=50, exposed=(1, 3), eps=0.2),
                                  lambda: W.butterfly(res=125),
                                  lambda: W.input_exemplar(), lambda: W.arrays_3d(res=75)],
                         ids=["butterfly50_xz", "butterfly125_wz", "exemplar", "arrays3d"])
def test_paper_examples(eng, orc, make):
    sy = make()
    for i, rel in enumerate(sy.rels):
        got = eng.plot(rel, sy.axes)
        eng.sync()
        check_plot_band(orc, rel, sy.axes, got, f"{sy.name} plot {i}")
    out, st = eng.solve(sy)
    eng.sync()
    want = orc.solve(sy.axes, sy.rels, sy.exposed).data
    assert np.array_equal(out.to_numpy(), want), sy.name
    assert out.padding_clean()
    assert want.sum() > 0, "the example has solutions in its box"


def test_mixed_and_batched(eng, orc):
    """Polynomial and expression relations in one system, and a batch of
    several expression systems; the kept program is reused only for the same
    constants."""
    circle = W.Relation((0, 1), 2, [-1.0, 0.0, 0.0, 1.0, 0.0, 1.0])
    y, z = Ex.port(0), Ex.port(1)
    r2 = W.expr_relation((1, 2), y - cos_(z * 2.0), eps=0.03)
    sy = W.System("mixed", [(-2.0, 2.0, 200)] * 3, [circle, r2], (0, 2))
    out, _ = eng.solve(sy)
    eng.sync()
    assert np.array_equal(out.to_numpy(), orc.solve(sy.axes, sy.rels, sy.exposed).data)
    # same structure, another constant: a new program, a new answer
    r2b = W.expr_relation((1, 2), y - cos_(z * 3.0), eps=0.03)
    sy2 = W.System("mixed2", sy.axes, [circle, r2b], (0, 2))
    out2, _ = eng.solve(sy2)
    eng.sync()
    assert np.array_equal(out2.to_numpy(), orc.solve(sy2.axes, sy2.rels, sy2.exposed).data)
    systems = [sy, sy2, W.butterfly(res=40), W.input_exemplar(eps=0.08)]
    outs, _ = eng.solve_batch(systems)
    eng.sync()
    for o, s in zip(outs, systems):
        assert np.array_equal(o.to_numpy(), orc.solve(s.axes, s.rels, s.exposed).data), s.name


def bisect(f, a, b, it=200):
    fa = f(a)
    for _ in range(it):
        m = 0.5 * (a + b)
        fm = f(m)
        if (fm < 0) == (fa < 0):
            a, fa = m, fm
        else:
            b = m
    return 0.5 * (a + b)


def butterfly_points():
    """Points (w, x, y, z) of the butterfly system's solution set, found by
    bisection on one variable at a time (Sec. 2.4 equations)."""
    pts = []
    for yv in np.linspace(-1.5, -0.3, 9):
        # Equation 3 in x, away from the poles of tan and the roots of the denominator
        g3 = lambda xv: math.tan(xv + yv) - (xv - 2) * (xv + 3) * yv * yv
        xs = np.linspace(-0.9, 0.9, 721)
        vals = [g3(v) for v in xs]
        for a, b, fa, fb in zip(xs, xs[1:], vals, vals[1:]):
            if fa * fb < 0 and abs(fa) < 50 and abs(fb) < 50:
                xv = bisect(g3, a, b)
                # Equation 2 in w (cosh(w) = 2 - y - ...: two roots, take w > 0)
                g2 = lambda wv: math.cosh(wv + 1e-3 * yv) + yv + 1e-4 * wv - 2
                if g2(0.0) < 0 < g2(2.9):
                    wv = bisect(g2, 0.0, 2.9)
                    # Equation 1 in z > 0
                    g1 = lambda zv: math.cos(math.log(zv * zv + 1e-3 * xv)) - xv + 1e-5 / zv
                    zs = np.linspace(0.2, 2.9, 541)
                    v1 = [g1(v) for v in zs]
                    for c, d, fc, fd in zip(zs, zs[1:], v1, v1[1:]):
                        if fc * fd < 0:
                            pts.append((wv, xv, yv, bisect(g1, c, d)))
                break
    return pts


def test_butterfly_no_false_negative(eng, orc):
    """Sec. 3.4: with tolerances valid at the solution points, each point's
    exposed pixel (w, z) is on.  Each relation's tolerance is set above the
    largest |f(centre)| over the pixels holding the points (measured with the
    oracle), so the plots mark those pixels and the product keeps them."""
    res = 125
    sy = W.butterfly(res=res)
    pts = butterfly_points()
    assert len(pts) >= 5
    d = 6.0 / res
    eps = []
    for rel in sy.rels:
        ops, consts = rel.expr
        need = 0.0
        for p in pts:
            c = [(-3.0 + (int((p[v] + 3.0) / d) + 0.5) * d) for v in rel.vars]
            need = max(need, abs(orc.eval_expr(ops, consts, c)))
        eps.append(need * 1.01 + 1e-12)
    rels = [W.Relation(r.vars, 0, r.coeffs, r.kind, e, r.expr) for r, e in zip(sy.rels, eps)]
    sy2 = W.System("butterfly_valid", sy.axes, rels, sy.exposed)
    out, _ = eng.solve(sy2)
    eng.sync()
    got = out.to_numpy()
    for p in pts:
        iw, iz = int((p[0] + 3.0) / d), int((p[3] + 3.0) / d)
        assert got[iw, iz] == 1, p
    assert np.array_equal(got, orc.solve(sy2.axes, sy2.rels, sy2.exposed).data)
