"""GPU parity of the counting-semiring cluster (pa_contract_count): the arrays
of the method may take values in the natural numbers to count solutions
instead of marking them (Sec. 2.2, footnote on plots).  The tensor-core path
without its > 0 threshold gives every count exactly (each is an integer of at
most K, exact in FP32 up to 2^24), compared element by element with the
oracle's plain loop."""
import numpy as np
import pytest

import paper_1609_00061_gb300 as pa
from paper_1609_00061_gb300 import workloads as W

from test_gpu_parity import pack, rand_bits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    e = pa.Engine(0)
    yield e
    e.close()


CASES = [
    # (X vars, Y vars, keep, res by var)
    ((0, 1), (1, 2), (0, 2), {0: 128, 1: 128, 2: 256}),      # one tile
    ((0, 1), (1, 2), (0, 2), {0: 129, 1: 130, 2: 257}),      # past every tile edge
    ((0, 1), (1, 2), (0, 2), {0: 1, 1: 3, 2: 1}),            # degenerate
    ((0, 1), (1, 2), (2, 0), {0: 70, 1: 300, 2: 100}),       # transposed keep order
    ((0, 1, 2), (0, 2, 3), (0, 1, 3), {0: 3, 1: 200, 2: 150, 3: 300}),  # batch axis
    ((0, 1, 2), (0, 2, 3), (3, 0, 1), {0: 2, 1: 40, 2: 50, 3: 70}),     # batch, permuted
    ((0, 1, 2), (1, 2, 3), (0, 3), {0: 64, 1: 30, 2: 40, 3: 65}),       # two summed axes
    ((1, 0), (1, 2), (0, 2), {0: 90, 1: 200, 2: 64}),        # A's summed axis first
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("density", [0.02, 0.5])
def test_contract_count(eng, orc, case, density):
    xv, yv, keep, rmap = CASES[case]
    rng = np.random.default_rng(8100 + 10 * case + int(density * 100))
    X = rand_bits(rng, tuple(rmap[v] for v in xv), density)
    Y = rand_bits(rng, tuple(rmap[v] for v in yv), density)
    vres = [rmap.get(v, 1) for v in range(max(rmap) + 1)]
    want = orc.contract_count(orc.Arr(X, xv), orc.Arr(Y, yv), keep, vres)
    got = eng.contract_count(pack(X, xv), pack(Y, yv), keep)
    eng.sync()
    got = got.cpu().numpy().view(np.uint32).astype(np.uint64)
    assert got.shape == want.shape
    assert np.array_equal(got, want), f"{int((got != want).sum())} counts differ"


def test_count_full_rows(eng, orc):
    """All-ones operands: every count is K = 4096 (exact), and one more K row
    of zeros changes nothing."""
    X = np.ones((200, 4097), dtype=np.uint8)
    X[:, -1] = 0
    Y = np.ones((4097, 130), dtype=np.uint8)
    got = eng.contract_count(pack(X, (0, 1)), pack(Y, (1, 2)), (0, 2))
    eng.sync()
    assert np.all(got.cpu().numpy() == 4096)


def test_count_chain_join(eng, orc):
    """Two plots of the chain workload at 512: the number of shared v2
    pixels behind every (v1, v3) pixel, against the oracle; its support is the
    Boolean product."""
    sy = W.chain(res=512, nrel=2)
    a = eng.plot(sy.rels[0], sy.axes)
    b = eng.plot(sy.rels[1], sy.axes)
    got = eng.contract_count(a, b, (0, 2))
    boolean = eng.contract(a, b, (0, 2))
    eng.sync()
    pa_ = orc.plot_relation(sy.rels[0], sy.axes)
    pb = orc.plot_relation(sy.rels[1], sy.axes)
    want = orc.contract_count(pa_, pb, (0, 2), [512] * 3)
    g = got.cpu().numpy().view(np.uint32).astype(np.uint64)
    assert np.array_equal(g, want)
    assert np.array_equal(boolean.to_numpy(), (want > 0).astype(np.uint8))


def test_count_unsupported(eng):
    X = pack(np.ones((4, 5), np.uint8), (0, 1))
    Y = pack(np.ones((5, 6), np.uint8), (1, 2))
    Z = pack(np.ones((4, 5), np.uint8), (0, 1))
    for A, B, keep in [(X, Y, (0,)),        # v2 private to B
                       (X, Z, (0, 1)),      # nothing summed
                       (X, Y, (0, 1, 2))]:  # nothing summed (outer)
        with pytest.raises(pa.PaError) as e:
            eng.contract_count(A, B, keep)
        assert e.value.status == 2
