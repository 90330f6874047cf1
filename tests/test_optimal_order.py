"""Optimal cluster trees (Sec. 3.5, cost polynomials minimised over cluster
trees).  The oracle's brute force (oracle/clusters.py) is pinned first --
the paper's cluster-tree example, the matrix-triple costs, tree counts and a
chain's closed form -- and then the library's exact planner
(PA_ORDER_OPTIMAL, a dynamic program over subsets) is checked against it:
same least cost on every random network small enough to enumerate, never
more than greedy, and its own tree's cost recomputed independently."""
import json
import math
import os

import numpy as np
import pytest

from oracle import clusters as C

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# -------------------------------------------------------- pins of the oracle
def test_oracle_tree_cost_paper_example():
    g = json.load(open(os.path.join(GOLDEN, "cluster_tree_example.json")))
    names = sorted({l for p in g["packs"].values() for l in p} | set(g["outer"]))
    lid = {n: i for i, n in enumerate(names)}
    order = ["A", "B", "C", "D", "E", "F", "G"]
    packs = [tuple(lid[l] for l in g["packs"][p]) for p in order]
    outer = [lid[l] for l in g["outer"]]

    def conv(node):
        return order.index(node) if isinstance(node, str) else tuple(conv(c) for c in node)

    tree = conv(g["tree"])
    # the paper compares parallel costs as polynomials in r; evaluated at a
    # number, the maximum over children agrees with that order once r >= 3
    for r in (3, 7, 10):
        s, p = C.tree_cost(tree, packs, outer, [r] * len(names))
        assert s == sum(c * r ** k for k, c in enumerate(g["cost_coeffs_r0_to_r5"]))
        assert p == sum(c * r ** k for k, c in enumerate(g["parallel_cost_coeffs_r0_to_r5"]))


def test_oracle_matrix_triple():
    """Sec. 3.5: the product MNP unclustered costs n^4, clustered 2 n^3."""
    n = 11
    packs, outer = [(0, 1), (1, 2), (2, 3)], (0, 3)
    assert C.tree_cost((0, 1, 2), packs, outer, [n] * 4) == (n ** 4, n ** 4)
    assert C.tree_cost(((0, 1), 2), packs, outer, [n] * 4) == (2 * n ** 3, 2 * n ** 3)
    best = C.min_cost(packs, outer, [n] * 4, binary=False)
    assert best[0] == 2 * n ** 3


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_oracle_tree_counts(n):
    """(2n-3)!! binary trees; cluster trees: 1, 1, 4, 26, 236, 2752 (Schroeder's
    fourth problem, the number of total partitions of n labelled items)."""
    nb = sum(1 for _ in C.binary_trees(range(n)))
    assert nb == (math.prod(range(1, 2 * n - 2, 2)) if n > 1 else 1)
    nc = sum(1 for _ in C.cluster_trees(range(n)))
    assert nc == [1, 1, 4, 26, 236, 2752][n - 1]


@pytest.mark.parametrize("L,r", [(2, 5), (4, 7), (6, 3)])
def test_oracle_chain_closed_form(L, r):
    """A chain of L binary relations with its two ends exposed: every pairwise
    tree whose clusters are contiguous costs (L-1) r^3, and no tree is cheaper."""
    packs = [(k, k + 1) for k in range(L)]
    best = C.min_cost(packs, (0, L), [r] * (L + 1))
    assert best[0] == (L - 1) * r ** 3
    left = 0
    for k in range(1, L):
        left = (left, k)
    assert C.tree_cost(left, packs, (0, L), [r] * (L + 1))[0] == (L - 1) * r ** 3


def test_oracle_bounds_between_tree_families():
    """Binary trees are cluster trees, so the least cost over all cluster trees
    is at most the least binary cost; every binary cluster costs at most
    r^(all links), so the least binary cost is at most (n - 1) times that; and
    the root of any tree counts the outer links, so no tree costs less than
    r^(outer links)."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        n, nl = int(rng.integers(2, 6)), int(rng.integers(3, 7))
        packs = [tuple(sorted(set(int(x) for x in rng.integers(0, nl, int(rng.integers(1, 4))))))
                 for _ in range(n)]
        outer = tuple(sorted(set(int(x) for x in rng.integers(0, nl, 2))))
        res = [int(x) for x in rng.integers(2, 9, nl)]
        best = C.min_cost(packs, outer, res)[0]
        general = C.min_cost(packs, outer, res, binary=False)[0]
        used = set(l for p in packs for l in p) | set(outer)
        assert math.prod(res[l] for l in outer) <= general <= best
        assert best <= (n - 1) * math.prod(res[l] for l in used)


# ----------------------------------------------- the library against the oracle
pa = pytest.importorskip("paper_1609_00061_gb300")
W = pytest.importorskip("paper_1609_00061_gb300.workloads")


def random_network(rng, nrel, nvars, res_choices=(2, 3, 5, 8)):
    rels = []
    for _ in range(nrel):
        ar = int(rng.integers(1, 4))
        vs = [int(v) for v in rng.choice(nvars, size=min(ar, nvars), replace=False)]
        rels.append(W.Relation(vs, 1, np.ones(W.coeff_count(len(vs), 1))))
    used = sorted({v for r in rels for v in r.vars})
    ne = int(rng.integers(0, min(3, len(used)) + 1))
    exposed = tuple(int(v) for v in rng.choice(used, size=ne, replace=False))
    axes = [(-1.0, 1.0, int(res_choices[int(rng.integers(len(res_choices)))]))
            for _ in range(nvars)]
    return W.System("rand", axes, rels, exposed)


@pytest.mark.parametrize("seed", range(12))
def test_optimal_matches_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    nrel = [2, 3, 4, 5, 6, 7][seed % 6]
    sy = random_network(rng, nrel, int(rng.integers(3, 8)))
    pairs, ops, peak = pa.pa_plan_order(sy.axes, sy.rels, sy.exposed, order="optimal")
    packs, outer, res = C.network_packs(sy)
    best = C.min_cost(packs, outer, res)
    assert ops == best[0], (seed, ops, best)
    # the tree the library chose costs what it reports, by the oracle's own sum
    tree = C.pairs_to_tree(pairs, nrel)
    s, p = C.tree_cost(tree, packs, outer, res)
    assert s == ops
    assert p == best[1], "ties go to the smaller parallel cost"
    _, gops, _ = pa.pa_plan_order(sy.axes, sy.rels, sy.exposed, order="greedy")
    assert ops <= gops


def test_optimal_on_workload_networks():
    """Networks of the random-network workload (12-20 relations): the exact
    planner is never worse than greedy and its reported cost is its tree's."""
    nets = W.random_networks(24, seed=W.SEED_BASE + 5)
    ratios = []
    for sy in nets:
        pairs, ops, _ = pa.pa_plan_order(sy.axes, sy.rels, sy.exposed, order="optimal")
        _, gops, _ = pa.pa_plan_order(sy.axes, sy.rels, sy.exposed, order="greedy")
        packs, outer, res = C.network_packs(sy)
        assert C.tree_cost(C.pairs_to_tree(pairs, len(sy.rels)), packs, outer, res)[0] == ops
        assert ops <= gops
        ratios.append(gops / ops)
    print(f"greedy / optimal naive cost: median {np.median(ratios):.3f}, max {max(ratios):.3f}")


def test_optimal_chain_is_closed_form():
    sy = W.chain(res=64, nrel=8)
    _, ops, _ = pa.pa_plan_order(sy.axes, sy.rels, sy.exposed, order="optimal")
    assert ops == 7 * 64 ** 3
