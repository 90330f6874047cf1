"""GPU parity of the layout kernels behind a cluster (Sec. 3.5): the word-gather
and 64 x 64 bit-transpose reshapes, the outer-product kernel of clusters that
sum nothing, and the masked-dot kernel of clusters that keep no axis of one
operand alone.  Every result equals the oracle's bit for bit, padding clean."""
import numpy as np
import pytest

import paper_1609_00061_gb300 as pa
from paper_1609_00061_gb300 import workloads as W

from test_gpu_parity import check_same, pack, rand_bits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    e = pa.Engine(0)
    yield e
    e.close()


LAYOUT_CASES = [
    # (X vars, Y vars, keep, res by var)
    ((0, 1), (1, 0), (0, 1), {0: 320, 1: 576}),             # transpose, several tiles
    ((0, 1), (1, 0), (0, 1), {0: 300, 1: 333}),             # transpose, ragged J and L
    ((0, 1, 2), (2, 0, 1), (0, 1, 2), {0: 5, 1: 130, 2: 200}),  # transpose, other axis
    ((0, 1), (1, 0), (0, 1), {0: 2048, 1: 1536}),           # transpose, large
    ((1, 0, 2), (1, 2, 3), (0, 3), {0: 40, 1: 64, 2: 128, 3: 50}),  # word gather, 2 packed axes
    ((0, 4, 1), (1, 2), (0, 2), {0: 30, 1: 130, 2: 70, 4: 7}),  # word gather + reduction
    ((0, 1), (1, 2), (0, 1, 2), {0: 70, 1: 90, 2: 130}),    # outer with a batch axis
    ((0,), (1,), (0, 1), {0: 100, 1: 200}),                 # outer, no batch
    ((0, 1), (1,), (0, 1), {0: 77, 1: 150}),                # outer, operands swapped
    ((0, 1, 2), (0, 2), (0, 1), {0: 9, 1: 100, 2: 200}),    # batched masked dot
    ((0, 1), (0, 1), (0,), {0: 130, 1: 70}),                # dot, no M axis
    ((0, 1), (0, 1), (), {0: 64, 1: 640}),                  # dot to a scalar
    ((2, 0, 1), (1, 2, 3), (3, 0), {0: 17, 1: 64, 2: 3, 3: 65}),  # mixed
    ((0, 4), (0, 1), (0, 1), {0: 100, 1: 70, 4: 130}),      # private packed axis: row OR
    ((0, 4, 5), (0, 1), (1, 0), {0: 33, 1: 65, 4: 3, 5: 200}),  # row OR over two axes
]


@pytest.mark.parametrize("case", range(len(LAYOUT_CASES)))
@pytest.mark.parametrize("density", [0.03, 0.4])
def test_layout_cases(eng, orc, case, density):
    xv, yv, keep, rmap = LAYOUT_CASES[case]
    rng = np.random.default_rng(1000 + 10 * case + int(density * 100))
    X = rand_bits(rng, tuple(rmap[v] for v in xv), density)
    Y = rand_bits(rng, tuple(rmap[v] for v in yv), density)
    vres = [rmap.get(v, 1) for v in range(max(rmap) + 1)]
    want = orc.contract(orc.Arr(X, xv), orc.Arr(Y, yv), keep, vres).data
    got = eng.contract(pack(X, xv), pack(Y, yv), keep)
    eng.sync()
    check_same(got, want, str(LAYOUT_CASES[case]))


@pytest.mark.parametrize("res_choices", [(64, 128, 192), (48, 96, 130)])
def test_networks_layouts(eng, orc, res_choices):
    """Random tree-like networks of binary and ternary relations: intermediates
    with several packed axes pass through every reshape mode."""
    nets = W.random_networks(10, seed=4242 + res_choices[0], nvars_range=(6, 8),
                             nrel_range=(7, 10), res_choices=res_choices)
    outs, _ = eng.solve_batch(nets)
    eng.sync()
    for o, sy in zip(outs, nets):
        want = orc.solve(sy.axes, sy.rels, sy.exposed).data
        check_same(o, want, sy.name)
