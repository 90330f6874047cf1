"""GPU parity of the tensor-core contraction path (0/1 E4M3 tcgen05 products,
FP32 accumulation, > 0): forced on every matrix-form cluster, it gives the same
bits as the oracle on single clusters, whole networks and batches; the
autotuner's rates are measured and the automatic choice stays bit-exact."""
import math

import numpy as np
import pytest

import paper_1609_00061_gb300 as pa
from paper_1609_00061_gb300 import workloads as W

from test_gpu_layouts import LAYOUT_CASES
from test_gpu_parity import CASES, check_same, pack, rand_bits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    e = pa.Engine(0)
    e.set_path("mma")
    yield e
    e.close()


MMA_CASES = [
    # (X vars, Y vars, keep, res by var): shapes around the 128 x 256 x 128 tiles
    ((0, 1), (1, 2), (0, 2), {0: 128, 1: 128, 2: 256}),     # exactly one tile
    ((0, 1), (1, 2), (0, 2), {0: 129, 1: 129, 2: 257}),     # one past every tile edge
    ((0, 1), (1, 2), (0, 2), {0: 1, 1: 3, 2: 1}),           # degenerate sizes
    ((0, 1), (1, 2), (0, 2), {0: 300, 1: 1000, 2: 40}),     # narrow N (64-column tiles)
    ((0, 1), (1, 2), (0, 2), {0: 70, 1: 70, 2: 100}),       # 128-column tiles
    ((0, 1, 2), (0, 2, 3), (0, 1, 3), {0: 3, 1: 200, 2: 150, 3: 300}),  # batch axis
    ((0, 1), (1, 2), (0, 2), {0: 1024, 1: 1024, 2: 1024}),  # several tiles each way
    # few output tiles and a long K: K split over several CTAs per tile, their
    # partial results OR-ed into C (a ragged last K block, a batch axis, and
    # two summed variables of 256 x 64)
    ((0, 1), (1, 2), (0, 2), {0: 200, 1: 5000, 2: 300}),
    ((0, 1, 2), (0, 2, 3), (0, 1, 3), {0: 3, 1: 100, 2: 3000, 3: 64}),
    ((0, 1, 2), (1, 2, 3), (0, 3), {0: 64, 1: 256, 2: 64, 3: 100}),
]


@pytest.mark.parametrize("case", range(len(CASES) + len(LAYOUT_CASES) + len(MMA_CASES)))
@pytest.mark.parametrize("density", [0.02, 0.5])
def test_contract_mma(eng, orc, case, density):
    allc = CASES + LAYOUT_CASES + MMA_CASES
    xv, yv, keep, rmap = allc[case]
    rng = np.random.default_rng(7000 + 10 * case + int(density * 100))
    X = rand_bits(rng, tuple(rmap[v] for v in xv), density)
    Y = rand_bits(rng, tuple(rmap[v] for v in yv), density)
    vres = [rmap.get(v, 1) for v in range(max(rmap) + 1)]
    want = orc.contract(orc.Arr(X, xv), orc.Arr(Y, yv), keep, vres).data
    got = eng.contract(pack(X, xv), pack(Y, yv), keep)
    eng.sync()
    check_same(got, want, str(allc[case]))


def test_full_rows_all_ones(eng, orc):
    """All-ones operands with K = 4096: every count is K (exact in FP32)."""
    X = np.ones((200, 4096), dtype=np.uint8)
    Y = np.ones((4096, 130), dtype=np.uint8)
    want = orc.contract(orc.Arr(X, (0, 1)), orc.Arr(Y, (1, 2)), (0, 2), [200, 4096, 130]).data
    got = eng.contract(pack(X, (0, 1)), pack(Y, (1, 2)), (0, 2))
    eng.sync()
    check_same(got, want)


@pytest.mark.parametrize("sysm", [W.circle_parabola(res=256), W.chain(res=333, nrel=5, seed=11),
                                  W.ternary(res=50)], ids=lambda s: s.name)
def test_solve_mma(eng, orc, sysm):
    out, _ = eng.solve(sysm)
    eng.sync()
    want = orc.solve(sysm.axes, sysm.rels, sysm.exposed).data
    check_same(out, want, sysm.name)


def test_chain_2048_mma_full(eng, orc):
    """The 2048-pixel chain (7 Boolean 2048^3 joins) on the tensor cores."""
    sysm = W.chain()
    out, _ = eng.solve(sysm)
    eng.sync()
    want = orc.solve(sysm.axes, sysm.rels, sysm.exposed).data
    check_same(out, want, sysm.name)


def test_batch_mma(eng, orc):
    systems = W.batched_chains(nsys=24, seed=31, res_choices=[64, 100, 192, 256], min_len=2,
                               max_len=5)
    b = eng.batch(systems)
    b.run()
    eng.sync()
    for o, sy in zip(b.outs, systems):
        want = orc.solve(sy.axes, sy.rels, sy.exposed).data
        check_same(o, want, sy.name)
    b.close()


def test_networks_mma(eng, orc):
    nets = W.random_networks(6, seed=977, nvars_range=(6, 8), nrel_range=(7, 9),
                             res_choices=(64, 96, 128))
    outs, _ = eng.solve_batch(nets)
    eng.sync()
    for o, sy in zip(outs, nets):
        want = orc.solve(sy.axes, sy.rels, sy.exposed).data
        check_same(o, want, sy.name)


def test_autotune_and_auto_path(orc):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    e = pa.Engine(0)
    default = pa.pa_get_rates(e.ctx)
    rates = e.autotune()
    assert all(math.isfinite(v) and v > 0 for v in rates.values())
    assert pa.pa_get_rates(e.ctx) == rates
    # the tensor path must be far faster per multiply-add than the row-OR per word
    assert rates["mma_macs_per_us"] > 100 * rates["rowor_words_per_us"]
    pa.pa_set_rates(e.ctx, default)
    assert pa.pa_get_rates(e.ctx) == default
    with pytest.raises(pa.PaError):
        pa.pa_set_rates(e.ctx, {"rowor_words_per_us": 0.0, "rowor_words_per_us_dense": 1.0,
                                "mma_macs_per_us": 1.0})
    with pytest.raises(pa.PaError):
        e.set_path(7)
    pa.pa_set_rates(e.ctx, rates)
    sysm = W.chain(res=1024, nrel=4, seed=12)
    out, _ = e.solve(sysm)
    e.sync()
    want = orc.solve(sysm.axes, sysm.rels, sysm.exposed).data
    check_same(out, want, sysm.name)
    e.close()
