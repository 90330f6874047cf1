"""GPU parity of the batched entry points: many independent systems of uneven
size solved in shared launches (pa_solve_batch) and replayed from one CUDA
graph (pa_batch_create / pa_batch_run), each output equal bit for bit to the
oracle's solve of that system alone."""
import numpy as np
import pytest

import paper_1609_00061_gb300 as pa
from paper_1609_00061_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    e = pa.Engine(0)
    yield e
    e.close()


def small_chains(n, seed, res_choices):
    return W.batched_chains(nsys=n, seed=seed, res_choices=res_choices, min_len=2, max_len=6)


def check_all(outs, systems, orc):
    for k, (o, sy) in enumerate(zip(outs, systems)):
        want = orc.solve(sy.axes, sy.rels, sy.exposed).data
        got = o.to_numpy()
        assert got.shape == want.shape, k
        assert np.array_equal(got, want), f"system {k}: {int((got != want).sum())} pixels differ"
        assert o.padding_clean(), k


def test_solve_batch_uneven_ragged(eng, orc):
    """Odd resolutions (ragged words) and random sub-boxes, 40 chains in one call."""
    systems = small_chains(40, 11, [37, 64, 65, 100, 127, 130, 200])
    outs, st = eng.solve_batch(systems)
    eng.sync()
    check_all(outs, systems, orc)
    assert st["n_plots"] == sum(len(s.rels) for s in systems)
    # every tree level of every system shares launches: far fewer than one per join
    assert st["n_launches"] < st["n_joins"]


def test_solve_batch_multiple_of_64(eng, orc):
    systems = small_chains(24, 12, [64, 128, 192, 256])
    outs, st = eng.solve_batch(systems)
    eng.sync()
    check_all(outs, systems, orc)


def test_batch_graph_replay(eng, orc):
    systems = small_chains(30, 13, [64, 96, 128, 160])
    b = eng.batch(systems)
    for _ in range(3):
        for o in b.outs:
            o.words.fill_(-1)      # replays must rewrite every word
        b.run()
        eng.sync()
        check_all(b.outs, systems, orc)
    st = b.stats()
    assert st["n_joins"] == sum(len(s.rels) - 1 for s in systems)
    b.close()


def test_solve_batch_mixed_systems(eng, orc):
    """Different shapes in one batch: circle/parabola, a ternary network, a
    single relation, a system with nothing exposed, a loop."""
    rng = W.SplitMix64(77)
    systems = [W.circle_parabola(res=100), W.ternary(res=20),
               W.System("single", [(-2, 2, 90), (-1, 1, 33)],
                        [W.Relation((0, 1), 3, rng.normal(10))], (1,)),
               W.System("exists", [(-2, 2, 70)] * 3,
                        [W.Relation((0, 1), 2, [-1, 0, 0, 1, 0, 1]),
                         W.Relation((1, 2), 2, [0.5, 1, 0, 0, 0, -1])], ()),
               W.System("loop", [(-2, 2, 80), (-2, 2, 81)],
                        [W.Relation((0, 0, 1), 2, rng.normal(10)),
                         W.Relation((0, 1), 2, rng.normal(6))], (1,)),
               W.chain(res=150, nrel=5, seed=5)]
    outs, st = eng.solve_batch(systems)
    eng.sync()
    check_all(outs, systems, orc)


def test_batch_matches_single_solves(eng):
    systems = small_chains(16, 14, [64, 128, 256])
    outs, _ = eng.solve_batch(systems)
    for o, sy in zip(outs, systems):
        single, _ = eng.solve(sy)
        eng.sync()
        assert np.array_equal(o.to_numpy(), single.to_numpy())


def test_batch_rejects_bad_system(eng):
    systems = small_chains(3, 15, [64])
    bad = W.System("bad", [(0.0, 1.0, 1)], [W.Relation((0,), 1, [0.0, 1.0])], (0,))
    outs = [pa.BitArray.empty(s.exposed, [s.axes[v][2] for v in s.exposed]) for s in systems]
    outs.append(pa.BitArray.empty((0,), (1,)))
    with pytest.raises(pa.PaError) as e:
        pa.pa_solve_batch(eng.ctx, systems + [bad], outs)
    assert e.value.status == 1
