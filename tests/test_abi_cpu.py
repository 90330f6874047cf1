"""CPU checks of the C interface: the library loads, exports what include/pa.h
declares, and its host-only entry points (tolerance, planner, tree cost, argument
checks) behave as the paper and the oracle say.  No kernel runs here."""
import json
import os
import re

import numpy as np
import pytest

import paper_1609_00061_gb300 as pa
from paper_1609_00061_gb300 import _native
from paper_1609_00061_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module")
def lib():
    _native.build()
    return _native.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pa_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_native.EXPORTS)


def test_array_words(lib):
    assert pa.pa_array_words([]) == 1
    assert pa.pa_array_words([256, 256]) == 256 * 4
    assert pa.pa_array_words([3, 65]) == 3 * 2
    assert pa.pa_array_words([2048]) == 32


def test_create_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pa.PaError) as e:
        pa.pa_create(0, 0)
    assert e.value.status == 5


def test_tolerance_matches_oracle_bitwise(orc):
    rng = W.SplitMix64(77)
    for trial in range(40):
        arity = int(rng.integers(1, 4, 1)[0])
        degree = int(rng.integers(0, 5, 1)[0])
        nv = arity + 1
        axes = []
        for v in range(nv):
            a, b = sorted(-5 + 10 * rng.uniform(2))
            axes.append((a, b + 0.01, int(rng.integers(2, 3000, 1)[0])))
        vars_ = [int(v) for v in rng.integers(0, nv - 1, arity)]
        rule = trial % 2
        rel = W.Relation(vars_, degree, rng.normal(W.coeff_count(arity, degree)), rule=rule)
        got = pa.pa_valid_tolerance(rel, axes)
        want = orc.relation_eps(rel, axes)
        assert got == want, (trial, got, want)


def test_corner_rule_arguments():
    """The corner rule's tolerance is twice the centre rule's (full pixel
    width); a rule outside pa_rule is rejected before any GPU work."""
    axes = [(-2.0, 2.0, 64), (-1.0, 3.0, 48)]
    c = np.array([0.5, 1.0, -2.0, 0.25, 0.0, 1.5])
    e0 = pa.pa_valid_tolerance(W.Relation((0, 1), 2, c), axes)
    e1 = pa.pa_valid_tolerance(W.Relation((0, 1), 2, c, rule=W.RULE_CORNER), axes)
    assert e1 == 2.0 * e0 > 0
    with pytest.raises(pa.PaError) as e:
        pa.pa_valid_tolerance(W.Relation((0, 1), 2, c, rule=2), axes)
    assert e.value.status == 1


def test_tree_cost_paper_example(lib):
    """Sec. 3.5 cluster-tree example: Cost_T = 2r^5 + 2r^4 + r^3, parallel 2r^5."""
    g = json.load(open(os.path.join(GOLDEN, "cluster_tree_example.json")))
    names = sorted({l for p in g["packs"].values() for l in p} | set(g["outer"]))
    lid = {n: i for i, n in enumerate(names)}
    order = ["A", "B", "C", "D", "E", "F", "G"]
    packs = [[lid[l] for l in g["packs"][p]] for p in order]
    outer = [lid[l] for l in g["outer"]]
    slot = {p: i for i, p in enumerate(order)}
    clusters = []

    def build(node):
        if isinstance(node, str):
            return slot[node]
        kids = [build(c) for c in node]
        clusters.append(kids)
        return len(order) + len(clusters) - 1

    build(g["tree"])
    for r in (3, 5, 7, 10):
        s, p = pa.pa_tree_cost([r] * len(names), packs, outer, clusters)
        want_s = sum(c * r ** k for k, c in enumerate(g["cost_coeffs_r0_to_r5"]))
        want_p = sum(c * r ** k for k, c in enumerate(g["parallel_cost_coeffs_r0_to_r5"]))
        assert s == want_s and p == want_p


def test_tree_cost_matrix_triple(lib):
    """Sec. 3.5: MNP unclustered costs n^4, clustered (MN)P costs 2n^3."""
    n = 9
    packs = [[0, 1], [1, 2], [2, 3]]
    s, _ = pa.pa_tree_cost([n] * 4, packs, [0, 3], [[0, 1, 2]])
    assert s == n ** 4
    s, p = pa.pa_tree_cost([n] * 4, packs, [0, 3], [[0, 1], [3, 2]])
    assert s == 2 * n ** 3 and p == 2 * n ** 3


def test_tree_cost_speedup_inequality(lib):
    """Prop. speedup (Sec. 3.5): a nontrivial cluster never costs more."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        nl = int(rng.integers(4, 8))
        res = [int(v) for v in rng.integers(2, 6, nl)]
        packs = [[int(v) for v in rng.choice(nl, int(rng.integers(1, 4)), replace=False)]
                 for _ in range(int(rng.integers(3, 6)))]
        outer = [int(v) for v in rng.choice(nl, 1)]
        flat, _ = pa.pa_tree_cost(res, packs, outer, [list(range(len(packs)))])
        two, _ = pa.pa_tree_cost(res, packs, outer, [[0, 1], list(range(2, len(packs))) + [len(packs)]])
        # nontrivial clusters (properly internal and external links exist) are never worse
        inner = set(packs[0]) | set(packs[1])
        rest = set(outer).union(*[set(p) for p in packs[2:]])
        if inner - rest and rest - inner:
            assert two <= flat


def test_plan_order_chain_and_ternary(lib):
    s = W.chain(res=64, nrel=5)
    pairs, ops, peak = pa.pa_plan_order(s.axes, s.rels, s.exposed)
    assert len(pairs) == 4
    assert ops == 4 * 64 ** 3 and peak == 64 * 64
    t = W.ternary(res=32)
    pairs, ops, peak = pa.pa_plan_order(t.axes, t.rels, t.exposed)
    # greedy reading: R1 (v1,v4,v5) with R2 (v4,v5,v6) first (smallest result v1,v6)
    assert pairs[0] == (0, 1)
    assert peak <= 32 ** 3


def test_invalid_arguments_host(lib):
    bad = W.Relation((0, 1), 1, [0.0, 1.0, 1.0])
    with pytest.raises(pa.PaError) as e:
        pa.pa_valid_tolerance(bad, [(0.0, 1.0, 1), (0.0, 1.0, 4)])   # res < 2
    assert e.value.status == 1
    with pytest.raises(pa.PaError):
        pa.pa_valid_tolerance(bad, [(1.0, 0.0, 4), (0.0, 1.0, 4)])   # lo > hi
    with pytest.raises(pa.PaError):
        pa.pa_plan_order([(0, 1, 4)], [W.Relation((0, 3), 1, [0.0, 1.0, 1.0])], (0,))


def test_solve_argument_reuse():
    """The binding reuses the last call's marshalled arguments only while the
    same objects hold the same values; coefficient arrays are pointed at, so a
    change in place is seen without re-marshalling, and any other change (or a
    coefficient array that needed converting) builds new arguments."""
    s = W.chain(res=64, nrel=3)
    a1 = pa._network_args(s.axes, s.rels, s.exposed)
    assert pa._network_args(s.axes, s.rels, s.exposed) is a1
    s.rels[0].coeffs[0] += 1.0
    assert pa._network_args(s.axes, s.rels, s.exposed) is a1
    assert a1.c_rels[0].coeffs[0] == s.rels[0].coeffs[0]
    s.rels[1].eps = 0.5
    a2 = pa._network_args(s.axes, s.rels, s.exposed)
    assert a2 is not a1 and a2.c_rels[1].eps == 0.5
    s.rels[1].rule = W.RULE_CORNER
    a2b = pa._network_args(s.axes, s.rels, s.exposed)
    assert a2b is not a2 and a2b.c_rels[1].rule == W.RULE_CORNER
    a2 = a2b
    s.rels[1].vars = (2, 1)
    a3 = pa._network_args(s.axes, s.rels, s.exposed)
    assert a3 is not a2 and list(a3.c_rels[1].vars)[:2] == [2, 1]
    s.axes[2] = (-1.0, 1.0, 64)
    a4 = pa._network_args(s.axes, s.rels, s.exposed)
    assert a4 is not a3 and a4.c_axes[2].lo == -1.0
    a5 = pa._network_args(s.axes, s.rels, (0, 2))
    assert a5 is not a4 and list(a5.c_exposed)[:2] == [0, 2]
    s.rels[2].coeffs = s.rels[2].coeffs.astype(np.float32)
    a6 = pa._network_args(s.axes, s.rels, (0, 2))
    assert pa._network_args(s.axes, s.rels, (0, 2)) is not a6
    assert a6.c_rels[2].coeffs[1] == float(s.rels[2].coeffs[1])


def test_expression_relation_checks(lib):
    """Expression relations (Sec. 2.1, Sec. 2.4): programs are checked on the
    host before any launch; the library derives tolerances for polynomials only."""
    from paper_1609_00061_gb300.workloads import Ex, cos_
    axes = [(-2.0, 2.0, 16), (-2.0, 2.0, 16)]
    x, y = Ex.port(0), Ex.port(1)
    good = W.expr_relation((0, 1), cos_(x) - y, eps=0.1)
    pairs, ops, _ = pa.pa_plan_order(axes, [good], (0,))
    assert pairs == [] and ops == 0
    with pytest.raises(pa.PaError) as e:
        pa.pa_valid_tolerance(good, axes)
    assert e.value.status == 2

    def prog(ops, consts=(), eps=0.1, arity=2):
        return W.Relation(tuple(range(arity)), 0, np.zeros(1), 0, eps,
                          (np.array(ops, np.int32), np.array(consts, np.float64)))

    bad = [prog([W.X_ADD]),                                   # stack underflow
           prog([W.X_VAR, W.X_VAR]),                          # two values left
           prog([W.X_VAR + 256 * 5]),                         # port 5 of 2
           prog([W.X_CONST + 256 * 1], [1.0]),                # constant 1 of 1
           prog([W.X_VAR, 99]),                               # unknown instruction
           prog([W.X_VAR, W.X_POWI + 256 * 65]),              # power out of range
           prog([W.X_VAR], eps=-1.0),                         # no derived tolerance
           prog([W.X_CONST], [float("nan")]),                 # NaN constant
           prog([W.X_VAR] * 17 + [W.X_ADD] * 16)]             # 17 stack values
    for k, r in enumerate(bad):
        with pytest.raises(pa.PaError) as e:
            pa.pa_plan_order(axes, [r], (0,))
        assert e.value.status == 1, k
    ok = prog([W.X_VAR] * 16 + [W.X_ADD] * 15)                # exactly 16 values
    pa.pa_plan_order(axes, [ok], (0,))
