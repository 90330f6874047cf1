"""Training workflow of the learned join-order cost model.

The solver logs, for every join it runs one launch at a time, the 16 features
the library computes for the join and the measured microseconds
(Engine.log_joins).  Logs over many join orders of many training networks
train the cost model (CostModel.train, on the GPU); PA_ORDER_LEARNED then uses
the model to rank candidate orders, with the greedy order as fallback and judge.
"""
from __future__ import annotations

import math

import numpy as np

# Networks the batch benchmark and the tests solve: the greedy order's largest
# intermediate at most 2^30 bits and its naive cost (sum of r^Lambda) at most
# 1e13 pixel-ops.
MAX_PEAK_BITS = 1 << 30
MAX_PIXEL_OPS = 1e13


def usable_networks(nets, max_peak_bits=MAX_PEAK_BITS, max_pixel_ops=MAX_PIXEL_OPS):
    """The networks whose greedy plan stays within the limits above (host only)."""
    from . import pa_plan_order
    keep = []
    for n in nets:
        _, ops, peak = pa_plan_order(n.axes, n.rels, n.exposed)
        if peak <= max_peak_bits and ops <= max_pixel_ops:
            keep.append(n)
    return keep


def join_sequence_shapes(system, pairs):
    """Per join of a pair sequence: (kept variables, r^Lambda, result bits).
    Slots 0..nrel-1 are the relations; join t creates slot nrel + t."""
    vres = [a[2] for a in system.axes]
    slots = [list(dict.fromkeys(r.vars)) for r in system.rels]
    live = list(range(len(slots)))
    out = []
    for a, b in pairs:
        live.remove(a)
        live.remove(b)
        need = set(system.exposed)
        for s in live:
            need.update(slots[s])
        union = list(dict.fromkeys(slots[a] + slots[b]))
        keep = [v for v in union if v in need]
        cost = math.prod(vres[v] for v in union)
        bits = math.prod(vres[v] for v in keep)
        slots.append(keep)
        live.append(len(slots) - 1)
        out.append((keep, cost, bits))
    return out


def random_order(system, rng, max_bits=1 << 26, tries=50):
    """A random valid join sequence (pairs sharing a variable preferred) whose
    intermediates stay below max_bits, or None."""
    for _ in range(tries):
        slots = [set(r.vars) for r in system.rels]
        live = list(range(len(slots)))
        pairs = []
        ok = True
        while len(live) > 1:
            cand = [(a, b) for i, a in enumerate(live) for b in live[i + 1:]
                    if slots[a] & slots[b]]
            if not cand:
                cand = [(a, b) for i, a in enumerate(live) for b in live[i + 1:]]
            a, b = cand[int(rng.integers(len(cand)))]
            pairs.append((a, b))
            live.remove(a)
            live.remove(b)
            slots.append(slots[a] | slots[b])
            live.append(len(slots) - 1)
        shapes = join_sequence_shapes(system, pairs)
        if max(s[2] for s in shapes) > max_bits:
            ok = False
        if ok:
            return pairs
    return None


def collect_logs(engine, systems, orders_per_system=4, seed=0, max_bits=1 << 26):
    """Features and log2(us)/8 targets from the greedy order, the
    least-naive-cost order, the left-to-right order and random orders of
    every system."""
    rng = np.random.default_rng(seed)
    X, T, D = [], [], []
    for sy in systems:
        from . import pa_plan_order
        runs = [("greedy", None), ("left", None)]
        p_opt, _, peak = pa_plan_order(sy.axes, sy.rels, sy.exposed, "optimal")
        if peak <= max_bits:
            runs.append(("given", p_opt))
        for _ in range(orders_per_system):
            p = random_order(sy, rng, max_bits)
            if p is not None:
                runs.append(("given", p))
        for order, pairs in runs:
            if order == "left":
                shapes = join_sequence_shapes(sy, [(0, 1)] + [(len(sy.rels) + t, t + 2)
                                                             for t in range(len(sy.rels) - 2)])
                if max(s[2] for s in shapes) > max_bits:
                    continue
            f, us, dens, _ = engine.log_joins(sy, order=order, pairs=pairs)
            X.append(f)
            T.append(np.log2(np.maximum(us, 1e-3)) / 8.0)
            D.append(dens)
    return np.concatenate(X), np.concatenate(T), np.concatenate(D)
