"""Cluster-tree costs by brute force (Sec. 3.5, "Cluster trees" and the cost
polynomials Cost and Cost^infinity).

TEST INFRASTRUCTURE ONLY: the tests call this module to check the library's
planner; nothing in the product path imports it.

A wiring diagram here is a list of inner packs, each a tuple of link ids (its
ports' links), the outer pack's links, and a resolution per link.  A cluster
tree is a nested tuple whose leaves are pack indices: (0, (1, 2)) joins pack 0
with the cluster of packs 1 and 2.  The cost of one cluster is
r^(links of its children), a child contributing its own intermediate pack:
for a leaf its links, for a cluster the links of its packs that also touch
something outside it (another pack or the outer pack).  The root cluster also
counts the outer pack's links.  The serial cost sums over the clusters; the
parallel cost of a cluster is its own cost plus the largest parallel cost of
its children.

Everything is plain Python: enumerate every tree, evaluate it, take the
minimum.  It is exponential and meant for a handful of packs.
"""
from __future__ import annotations

import math
from itertools import combinations


def leaves(tree):
    if isinstance(tree, int):
        return [tree]
    out = []
    for c in tree:
        out.extend(leaves(c))
    return out


def intermediate_pack(tree, packs, outer):
    """Links of the packs inside `tree` that touch a pack outside it or the outer pack."""
    inside = set(leaves(tree))
    if isinstance(tree, int):
        return list(dict.fromkeys(packs[tree]))
    touch_out = set(outer)
    for p, links in enumerate(packs):
        if p not in inside:
            touch_out.update(links)
    out = []
    for p in leaves(tree):
        for l in packs[p]:
            if l in touch_out and l not in out:
                out.append(l)
    return out


def tree_cost(tree, packs, outer, link_res):
    """(serial, parallel) cost of a cluster tree whose root is `tree`."""

    def go(t, root):
        if isinstance(t, int):
            return 0.0, 0.0
        links = set()
        serial, below = 0.0, 0.0
        for c in t:
            links.update(intermediate_pack(c, packs, outer))
            s, p = go(c, False)
            serial += s
            below = max(below, p)
        if root:
            links.update(outer)
        own = math.prod(link_res[l] for l in links)
        return serial + own, own + below

    return go(tree, True)


def binary_trees(items):
    """Every binary tree (unordered children) over the given leaves."""
    items = list(items)
    if len(items) == 1:
        yield items[0]
        return
    first, rest = items[0], items[1:]
    # split into a part holding `first` and a non-empty remainder
    for k in range(0, len(rest)):
        for left_rest in combinations(rest, k):
            right = [x for x in rest if x not in left_rest]
            for lt in binary_trees([first, *left_rest]):
                for rt in binary_trees(right):
                    yield (lt, rt)


def set_partitions(items):
    """Every partition of `items` into non-empty blocks."""
    items = list(items)
    if not items:
        yield []
        return
    first, rest = items[0], items[1:]
    for part in set_partitions(rest):
        for i in range(len(part)):
            yield part[:i] + [[first] + part[i]] + part[i + 1:]
        yield [[first]] + part


def cluster_trees(items):
    """Every cluster tree (clusters of two or more children) over the leaves."""
    items = list(items)
    if len(items) == 1:
        yield items[0]
        return
    for part in set_partitions(items):
        if len(part) < 2:
            continue

        def expand(blocks):
            if not blocks:
                yield ()
                return
            for sub in cluster_trees(blocks[0]):
                for tail in expand(blocks[1:]):
                    yield (sub,) + tail

        yield from expand(part)


def min_cost(packs, outer, link_res, binary=True):
    """Least serial cost over every binary (or every) cluster tree, with the
    parallel cost of a least-serial tree that has the smallest parallel cost."""
    gen = binary_trees if binary else cluster_trees
    best = None
    for t in gen(range(len(packs))):
        s, p = tree_cost(t, packs, outer, link_res)
        if best is None or (s, p) < best[:2]:
            best = (s, p, t)
    return best


def network_packs(system):
    """A relation network as a wiring diagram: links are variables, inner packs
    the relations' distinct variables, the outer pack the exposed variables."""
    packs = [tuple(dict.fromkeys(r.vars)) for r in system.rels]
    link_res = [a[2] for a in system.axes]
    return packs, tuple(system.exposed), link_res


def pairs_to_tree(pairs, nrel):
    """The tree of a join list (slots 0..nrel-1 are relations, join t makes slot nrel+t)."""
    slot = {i: i for i in range(nrel)}
    for t, (a, b) in enumerate(pairs):
        slot[nrel + t] = (slot[a], slot[b])
    return slot[nrel + len(pairs) - 1] if pairs else 0
