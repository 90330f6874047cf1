"""GPU parity at the sizes the workloads state, through the same calls the
benchmark times.

- Batched chains: the whole 4096-system batch (2-6 binary cubics, 64..1024
  pixels per axis, random sub-boxes of [-4, 4)) is planned with autotuned
  rates and replayed as one CUDA graph; a seeded sample of its systems, the
  heaviest ones included, is compared bit for bit with the oracle (Sec. 3.6
  applied to each system).  The sample is also solved on its own with each
  contraction path forced.
- Random relation networks (10-16 variables, 12-20 relations of arity 2-3,
  128/256/512 pixels per axis): the batch of every usable network is replayed
  with the greedy order and with a trained cost model's orders; a sample whose
  oracle cost stays within seconds is compared bit for bit.
- Full-size plots: the eight 2048 x 2048 plots of the chain workload and the
  four 256^3 plots of the ternary workload, through pa_plot (Sec. 3.2,
  sample-in-center plot), against the oracle's plots pixel for pixel.
"""
import math

import numpy as np
import pytest

import paper_1609_00061_gb300 as pa
from paper_1609_00061_gb300 import learned as L
from paper_1609_00061_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    e = pa.Engine(0)
    e.autotune()
    yield e
    e.close()


_ORACLE = {}


def oracle_out(orc, key, sy):
    if key not in _ORACLE:
        _ORACLE[key] = orc.solve(sy.axes, sy.rels, sy.exposed).data
    return _ORACLE[key]


def check(out, want, what):
    got = out.to_numpy()
    assert got.shape == want.shape, what
    diff = int((got != want).sum())
    assert diff == 0, f"{what}: {diff} of {want.size} pixels differ"
    assert out.padding_clean(), what


def oracle_cost(sy):
    """Pixel-ops of the oracle's own solve (left fold up to four relations,
    smallest-result pairing beyond), computed from shapes only."""
    vres = [a[2] for a in sy.axes]
    slots = [list(dict.fromkeys(r.vars)) for r in sy.rels]
    total = 0.0
    if len(slots) <= 4:
        acc = []
        for pos, s in enumerate(slots):
            total += math.prod(vres[v] for v in dict.fromkeys(acc + s))
            later = set(sy.exposed).union(*[set(x) for x in slots[pos + 1:]])
            acc = [v for v in dict.fromkeys(acc + s) if v in later]
        return total
    live = slots
    while len(live) > 1:
        best = None
        for i in range(len(live)):
            for j in range(i + 1, len(live)):
                later = set(sy.exposed)
                for k, a in enumerate(live):
                    if k not in (i, j):
                        later.update(a)
                keep = [v for v in dict.fromkeys(live[i] + live[j]) if v in later]
                size = math.prod(vres[v] for v in keep)
                if best is None or size < best[0]:
                    best = (size, i, j, keep)
        _, i, j, keep = best
        total += math.prod(vres[v] for v in dict.fromkeys(live[i] + live[j]))
        live = [a for k, a in enumerate(live) if k not in (i, j)] + [keep]
    return total


# ------------------------------------------------------------ batched chains
@pytest.fixture(scope="module")
def chains():
    return W.batched_chains(nsys=4096, seed=W.SEED_BASE + 4)


def chain_sample(systems, n_random=32, n_heavy=16):
    cost = [sum(math.prod(sy.axes[v][2] for v in r.vars) for r in sy.rels) for sy in systems]
    heavy = list(np.argsort(cost)[::-1][:n_heavy])
    rng = np.random.default_rng(0x160900061)
    rest = [k for k in range(len(systems)) if k not in heavy]
    pick = sorted(int(k) for k in heavy) + sorted(int(k) for k in
                                                  rng.choice(rest, n_random, replace=False))
    return pick


def test_batched_chains_full_batch_sample(eng, orc, chains):
    """The benchmark's 4096-system batch, one graph replay, 48 systems checked."""
    b = eng.batch(chains)
    for o in b.outs:
        o.words.fill_(-1)     # the replay must write every word
    b.run()
    eng.sync()
    st = b.stats()
    assert st["n_joins"] == sum(len(s.rels) - 1 for s in chains)
    assert st["n_mma"] > 0, "the batch should send its largest joins to the tensor cores"
    for k in chain_sample(chains):
        check(b.outs[k], oracle_out(orc, ("chain", k), chains[k]), f"system {k}")
    b.close()


@pytest.mark.parametrize("path", ["auto", "mma", "rowor"])
def test_batched_chains_sample_each_path(eng, orc, chains, path):
    pick = chain_sample(chains)
    sample = [chains[k] for k in pick]
    eng.set_path(path)
    try:
        b = eng.batch(sample)
        b.run()
        eng.sync()
        st = b.stats()
        if path == "auto":
            assert st["n_mma"] >= 1, "the sample holds a join of the tensor-core path"
            assert st["n_mma"] < st["n_joins"], "and joins of the row-OR path"
        for k, o in zip(pick, b.outs):
            check(o, oracle_out(orc, ("chain", k), chains[k]), f"system {k} ({path})")
        b.close()
    finally:
        eng.set_path("auto")


# ---------------------------------------------------------- random networks
@pytest.fixture(scope="module")
def networks():
    return L.usable_networks(W.random_networks(512, seed=W.SEED_BASE + 5))


def network_sample(nets, budget=1.2e11, per_net=2.5e10):
    """Networks of every resolution whose oracle solve stays cheap, cheapest
    first per resolution, up to `budget` oracle pixel-ops in all."""
    by_res = {}
    for k, n in enumerate(nets):
        c = oracle_cost(n)
        if c <= per_net:
            by_res.setdefault(n.axes[0][2], []).append((c, k))
    pick, total = [], 0.0
    for res in sorted(by_res):
        for c, k in sorted(by_res[res])[:6]:
            if total + c <= budget:
                pick.append(k)
                total += c
    return sorted(pick)


@pytest.fixture(scope="module")
def model(eng):
    train = L.usable_networks(W.random_networks(16, seed=W.SEED_BASE + 50))
    X, T, _ = L.collect_logs(eng, train, orders_per_system=2, seed=2)
    m = pa.CostModel(eng, hidden=128, nlayers=3, seed=W.SEED_BASE + 5)
    m.train(X, T, epochs=60, batch=256, lr=2e-3)
    yield m
    m.close()


@pytest.mark.parametrize("order", ["greedy", "learned"])
def test_networks_full_batch_sample(eng, orc, networks, model, order):
    """Every usable network in one graph-replayed batch; a sample at 128, 256
    and 512 pixels checked, K-chunked row-OR joins included."""
    pick = network_sample(networks)
    assert len(pick) >= 10
    assert {networks[k].axes[0][2] for k in pick} >= {128, 256}
    b = eng.batch(networks, order=order, model=model if order == "learned" else None)
    b.run()
    eng.sync()
    for k in pick:
        check(b.outs[k], oracle_out(orc, ("net", k), networks[k]), f"network {k} ({order})")
    b.close()
    # the sample alone under the automatic path: row-OR joins whose K range is
    # split over several tiles, and (greedy) each path used
    sample = [networks[k] for k in pick]
    outs, st = eng.solve_batch(sample, order=order,
                               model=model if order == "learned" else None)
    eng.sync()
    for k, o in zip(pick, outs):
        check(o, oracle_out(orc, ("net", k), networks[k]), f"network {k} ({order}, sample)")


def test_networks_sample_has_k_chunked_joins(networks):
    """At least one join of the sample contracts more B rows than one row-OR
    tile holds (K = 65536 bits: two latent variables at 256 pixels)."""
    pick = network_sample(networks)
    big_k = 0
    for k in pick:
        n = networks[k]
        pairs, _, _ = pa.pa_plan_order(n.axes, n.rels, n.exposed)
        vres = [a[2] for a in n.axes]
        for keep, cost, bits in L.join_sequence_shapes(n, pairs):
            kbits = cost / max(1.0, bits)
            big_k += kbits >= 65536
    assert big_k >= 1


# -------------------------------------------------------------- full plots
def test_chain_plots_2048_full(eng, orc):
    sy = W.chain()
    for i, rel in enumerate(sy.rels):
        got = eng.plot(rel, sy.axes)
        eng.sync()
        want = orc.plot_relation(rel, sy.axes).data
        check(got, want, f"chain plot {i}")


def test_ternary_plots_256_full(eng, orc):
    sy = W.ternary()
    for i, rel in enumerate(sy.rels):
        got = eng.plot(rel, sy.axes)
        eng.sync()
        want = orc.plot_relation(rel, sy.axes).data
        check(got, want, f"ternary plot {i}")


def test_batched_plots_in_one_launch_full(eng, orc):
    """All eight 2048^2 chain plots in the one plot launch of a solve: the
    final output of a one-relation-per-system batch is the plot itself."""
    sy = W.chain()
    systems = [W.System(f"plot{i}", sy.axes, [rel], rel.vars) for i, rel in enumerate(sy.rels)]
    outs, st = eng.solve_batch(systems)
    eng.sync()
    assert st["n_joins"] == 0 and st["n_plots"] == 8
    for i, (o, rel) in enumerate(zip(outs, sy.rels)):
        check(o, orc.plot_relation(rel, sy.axes).data, f"batched chain plot {i}")
