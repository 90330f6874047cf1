"""GPU parity of the corner-lattice sample rule (pa.h, pa_rule; an optional
mode beside the paper's centre rule of Sec. 3.2) against the oracle's corner
mode.

Polynomials and expressions made of correctly rounded operations are
evaluated at the lattice points in the same IEEE double order on both sides,
so their plots are compared bit for bit: ragged resolutions (one word, a
partial last word, several words), 1 to 3 distinct variables, a repeated
variable, every comparison kind, the strict flag, library-derived and given
tolerances, and the 2048 x 2048 chain plot at its full size.  Expressions
with elementary functions (the CUDA math library against the C library)
may differ only where a corner value lies within 2^-30 of a threshold."""
import math

import numpy as np
import pytest

import paper_1609_00061_gb300 as pa
from paper_1609_00061_gb300 import workloads as W
from paper_1609_00061_gb300.workloads import Ex, cos_, sqrt_

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    e = pa.Engine(0)
    yield e
    e.close()


def corner_rel(vars_, degree, coeffs, kind=W.KIND_EQ, eps=-1.0):
    return W.Relation(tuple(vars_), degree, coeffs, kind, eps, rule=W.RULE_CORNER)


def check_exact(eng, orc, rel, axes, strict=False, what=""):
    got = eng.plot(rel, axes, strict=strict)
    eng.sync()
    want = orc.plot_relation(rel, axes, strict=strict).data
    g = got.to_numpy()
    assert g.shape == want.shape, what
    bad = np.argwhere(g != want)
    assert len(bad) == 0, f"{what}: {len(bad)} pixels differ, first {bad[:4].tolist()}"
    assert got.padding_clean(), what
    return want


@pytest.mark.parametrize("seed", range(12))
def test_random_polynomial_plots(eng, orc, seed):
    rng = np.random.default_rng(3300 + seed)
    arity = 1 + seed % 3
    choices = [2, 3, 63, 64, 65, 127, 130, 200] if arity < 3 else [2, 5, 31, 64, 66]
    axes = []
    for _ in range(arity):
        a, b = sorted(rng.uniform(-3, 3, 2))
        axes.append((float(a), float(b) + 0.2, int(rng.choice(choices))))
    degree = int(rng.integers(1, 5))
    coeffs = rng.standard_normal(W.coeff_count(arity, degree))
    kind = [W.KIND_EQ, W.KIND_LE, W.KIND_LT][seed % 3 if seed < 9 else 0]
    eps = -1.0 if seed % 2 == 0 else float(rng.uniform(0.0, 0.3))
    strict = seed in (5, 10)
    rel = corner_rel(range(arity), degree, coeffs, kind, eps)
    want = check_exact(eng, orc, rel, axes, strict, f"seed {seed}")
    assert want.size > 0


def test_repeated_variable(eng, orc):
    """Ports (x, x, y): the corners are those of the (x, y) pixel."""
    rng = np.random.default_rng(12)
    axes = [(-2.0, 2.5, 130), (-1.5, 2.0, 70)]
    coeffs = rng.standard_normal(W.coeff_count(3, 3))
    for eps in (-1.0, 0.05):
        rel = corner_rel((0, 0, 1), 3, coeffs, eps=eps)
        want = check_exact(eng, orc, rel, axes, what=f"repeated eps {eps}")
        assert 0 < want.sum() < want.size
    rel = corner_rel((1, 0, 1), 3, coeffs, kind=W.KIND_LE, eps=0.0)
    check_exact(eng, orc, rel, axes, what="repeated (y, x, y)")


def test_linear_closed_form_on_gpu(eng, orc):
    """f = x - 0.3 on [-2, 2) at 16 pixels, eps = 0: only pixel 9 ([0.25,
    0.5)) is on, by its sign change; f = x - 0.25: pixels 8 and 9 (a corner
    value of exactly 0), none of them with the strict flag."""
    axes = [(-2.0, 2.0, 16)]
    out = eng.plot(corner_rel((0,), 1, [-0.3, 1.0], eps=0.0), axes)
    eng.sync()
    assert np.flatnonzero(out.to_numpy()).tolist() == [9]
    rel = corner_rel((0,), 1, [-0.25, 1.0], eps=0.0)
    out = eng.plot(rel, axes)
    eng.sync()
    assert np.flatnonzero(out.to_numpy()).tolist() == [8, 9]
    out = eng.plot(rel, axes, strict=True)
    eng.sync()
    assert out.to_numpy().sum() == 0


def test_chain_plot_full_size(eng, orc):
    """One relation of the 9-variable chain at its stated 2048 x 2048."""
    sy = W.chain(res=2048, nrel=8)
    r0 = sy.rels[3]
    rel = corner_rel(r0.vars, r0.degree, r0.coeffs)
    want = check_exact(eng, orc, rel, sy.axes, what="chain 2048^2")
    dens = want.mean()
    assert 0.0005 < dens < 0.1, dens


def test_ternary_plot(eng, orc):
    rng = np.random.default_rng(21)
    axes = [(-2.0, 2.0, 40), (-2.0, 2.0, 33), (-2.0, 2.0, 67)]
    coeffs = rng.standard_normal(W.coeff_count(3, 3))
    want = check_exact(eng, orc, corner_rel((0, 1, 2), 3, coeffs), axes, what="ternary")
    assert 0 < want.sum() < want.size


def test_exact_expression_plot(eng, orc):
    """An expression of correctly rounded operations only: bit for bit."""
    x, y = Ex.port(0), Ex.port(1)
    e = sqrt_(x * x + y * y + 0.5) - 1.3 + x / (y * y + 1.0) - x ** 3 * 0.1
    ops, consts = e.program()
    axes = [(-2.0, 2.0, 100), (-2.5, 1.5, 129)]
    for kind, eps in ((W.KIND_EQ, 0.0), (W.KIND_EQ, 0.02), (W.KIND_LT, 0.0)):
        rel = W.Relation((0, 1), 0, np.zeros(1), kind, eps, (ops, consts), rule=W.RULE_CORNER)
        want = check_exact(eng, orc, rel, axes, what=f"expr kind {kind} eps {eps}")
        assert 0 < want.sum() < want.size


def test_elementary_expression_band(eng, orc):
    """cos from two math libraries: a pixel may differ only when one of its
    corner values lies within 2^-30 (relative) of eps or of 0."""
    x, y = Ex.port(0), Ex.port(1)
    e = y - cos_(x * 3.0)
    ops, consts = e.program()
    axes = [(-2.0, 2.0, 257), (-1.5, 1.5, 190)]
    rel = W.Relation((0, 1), 0, np.zeros(1), W.KIND_EQ, 0.01, (ops, consts), rule=W.RULE_CORNER)
    got = eng.plot(rel, axes)
    eng.sync()
    want = orc.plot_relation(rel, axes).data
    g = got.to_numpy()
    d = [(lo + np.arange(r + 1) * ((hi - lo) / r)) for lo, hi, r in axes]
    for i, j in np.argwhere(g != want):
        vals = [orc.eval_expr(ops, consts, [d[0][i + a], d[1][j + b]])
                for a in (0, 1) for b in (0, 1)]
        assert any(abs(abs(v) - 0.01) <= 2.0 ** -30 * 4 or abs(v) <= 2.0 ** -30 * 4
                   for v in vals if math.isfinite(v)), (i, j, vals)
    assert (g != want).sum() <= 5
    assert got.padding_clean()


def test_solve_mixed_rules(eng, orc):
    """A chain whose relations alternate between the two rules, solved whole
    and in a batch with centre-rule systems: bit for bit against the oracle."""
    sy = W.chain(res=256, nrel=4)
    rels = [corner_rel(r.vars, r.degree, r.coeffs) if k % 2 == 0 else r
            for k, r in enumerate(sy.rels)]
    mixed = W.System("chain_mixed_rules", sy.axes, rels, sy.exposed)
    out, st = eng.solve(mixed)
    eng.sync()
    want = orc.solve(mixed.axes, mixed.rels, mixed.exposed).data
    assert np.array_equal(out.to_numpy(), want)
    assert want.sum() > 0
    allc = W.System("chain_corner", sy.axes,
                    [corner_rel(r.vars, r.degree, r.coeffs) for r in sy.rels], sy.exposed)
    systems = [mixed, sy, allc, W.chain(res=128, nrel=3, seed=5)]
    outs, _ = eng.solve_batch(systems)
    eng.sync()
    for o, s in zip(outs, systems):
        assert np.array_equal(o.to_numpy(), orc.solve(s.axes, s.rels, s.exposed).data), s.name
    assert outs[2].to_numpy().sum() > 0
