"""GPU parity: every array the CUDA path produces must equal the oracle's, bit
for bit (plots, single clusters, whole networks), and padding bits must be 0."""
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


def pack(bits: np.ndarray, vars_, device=0) -> pa.BitArray:
    """Host marshalling: uint8 pixels -> the pa_array word layout on the GPU."""
    import torch
    res = tuple(int(r) for r in bits.shape)
    if len(res) == 0:
        w = np.array([int(bits) & 1], dtype=np.uint64)
    else:
        rw = (res[-1] + 63) // 64
        rows = bits.reshape(-1, res[-1]).astype(np.uint8)
        padded = np.zeros((rows.shape[0], rw * 64), dtype=np.uint8)
        padded[:, :res[-1]] = rows
        w = np.packbits(padded, axis=1, bitorder="little").view(np.uint64).reshape(-1)
    t = torch.from_numpy(w.view(np.int64).copy()).to(f"cuda:{device}")
    return pa.BitArray(t, tuple(vars_), res)


def check_same(got: pa.BitArray, want: np.ndarray, what=""):
    g = got.to_numpy()
    assert g.shape == want.shape, what
    diff = int((g != want).sum())
    assert diff == 0, f"{what}: {diff} of {want.size} pixels differ"
    assert got.padding_clean(), what


# ----------------------------------------------------------------- plots
def random_relation(rng, nvars, arity, degree, kind=0, eps=-1.0, allow_repeat=False):
    if allow_repeat:
        vs = [int(v) for v in rng.integers(0, nvars - 1, arity)]
    else:
        perm = np.argsort(rng.uniform(nvars))
        vs = [int(v) for v in perm[:arity]]
    return W.Relation(vs, degree, rng.normal(W.coeff_count(arity, degree)), kind, eps)


@pytest.mark.parametrize("res", [2, 3, 63, 64, 65, 127, 200, 333])
def test_plot_binary_ragged(eng, orc, res):
    rng = W.SplitMix64(1000 + res)
    axes = [(-2.5, 1.75, res), (-1.0, 3.0, res + 1)]
    for trial in range(4):
        rel = random_relation(rng, 2, 2, 3)
        check_same(eng.plot(rel, axes), orc.plot_relation(rel, axes).data, f"res {res} t{trial}")


@pytest.mark.parametrize("arity,degree,res", [(1, 5, 1000), (3, 3, 37), (3, 2, 64), (4, 2, 13),
                                              (2, 0, 70), (2, 6, 90), (5, 2, 7), (8, 1, 3)])
def test_plot_arity_degree(eng, orc, arity, degree, res):
    rng = W.SplitMix64(2000 + 31 * arity + degree)
    axes = [(-1.5 - 0.1 * v, 1.5 + 0.2 * v, res + (v % 3)) for v in range(arity + 1)]
    for kind in (W.KIND_EQ, W.KIND_LE, W.KIND_LT):
        rel = random_relation(rng, arity + 1, arity, degree, kind)
        check_same(eng.plot(rel, axes), orc.plot_relation(rel, axes).data, f"kind {kind}")


def test_plot_strict_and_given_eps(eng, orc):
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "appendix_a.json")))
    axes = [(g["lower"], g["upper"], g["resolution"])] * 3
    for coeffs, vs in ((g["m1_coeffs_graded_lex"], (0, 1)), (g["m2_coeffs_graded_lex"], (1, 2))):
        rel = W.Relation(vs, 2, coeffs, W.KIND_EQ, g["tol"])
        check_same(eng.plot(rel, axes, strict=True), orc.plot_relation(rel, axes, strict=True).data)
        check_same(eng.plot(rel, axes), orc.plot_relation(rel, axes).data)


def test_plot_exact_ties(eng, orc):
    """|f(c)| equal to eps exactly at many pixels: <= keeps them, < drops them."""
    # f = x - y on a dyadic grid: centres differ by exact multiples of 1/8
    axes = [(0.0, 4.0, 32), (0.0, 4.0, 32)]
    rel = W.Relation((0, 1), 1, [0.0, 1.0, -1.0], W.KIND_EQ, 0.25)
    check_same(eng.plot(rel, axes), orc.plot_relation(rel, axes).data)
    check_same(eng.plot(rel, axes, strict=True), orc.plot_relation(rel, axes, strict=True).data)
    assert eng.plot(rel, axes).to_numpy().sum() > eng.plot(rel, axes, strict=True).to_numpy().sum()


def test_plot_repeated_variable(eng, orc):
    """A variable on two ports: the plot is the diagonal (Sec. 3.1, loops)."""
    rng = W.SplitMix64(3000)
    axes = [(-2.0, 2.0, 150), (-1.0, 1.0, 70)]
    for vs in ((0, 0), (1, 0, 1), (0, 1, 0, 1)):
        rel = W.Relation(vs, 3, rng.normal(W.coeff_count(len(vs), 3)))
        full = orc.plot_relation(rel, axes)
        # reduce the oracle's port-wise plot to the diagonal over distinct variables
        dv = []
        for v in vs:
            if v not in dv:
                dv.append(v)
        diag = orc.reduce(full, tuple(dv), [a[2] for a in axes])
        check_same(eng.plot(rel, axes), diag.data, str(vs))


@pytest.mark.parametrize("vs,degree", [((0, 1, 2, 0, 1, 2, 0, 1), 3), ((2, 0, 1, 2), 4),
                                       ((0, 1, 2, 3, 4, 5, 6), 3), ((0, 1, 2, 3, 4, 5, 6, 7), 2)])
def test_plot_deep_nesting(eng, orc, vs, degree):
    """Seven and eight ports: the nested FP64 sums of the pa.h evaluation order at
    depths 5 to 7, on the row path (distinct variables) and the per-pixel path
    (repeated ones)."""
    rng = W.SplitMix64(3100 + len(vs) + 10 * degree)
    nv = max(vs) + 1
    axes = [(-1.2 - 0.05 * v, 1.1 + 0.1 * v, 3 + (v % 3) if nv > 3 else 4 + v) for v in range(nv)]
    coeffs = rng.normal(W.coeff_count(len(vs), degree))
    for kind in (W.KIND_EQ, W.KIND_LE):
        # eps = 1 leaves a mix of on and off pixels on these coarse grids
        rel = W.Relation(vs, degree, coeffs, kind, 1.0)
        full = orc.plot_relation(rel, axes)
        assert 0 < int(full.data.sum()) < full.data.size
        dv = []
        for v in vs:
            if v not in dv:
                dv.append(v)
        want = full if len(dv) == len(vs) else orc.reduce(full, tuple(dv), [a[2] for a in axes])
        check_same(eng.plot(rel, axes), want.data, f"{vs} kind {kind}")


def test_plot_large_values_and_overflow(eng, orc):
    """Coefficients near FP32 overflow and FP64 overflow: the exact FP64 path decides."""
    axes = [(-1e3, 1e3, 300), (-1e2, 1e2, 129)]
    for scale in (1e30, 1e36, 1e300):
        rel = W.Relation((0, 1), 3, np.linspace(-1, 1, 10) * scale, W.KIND_LE, 1e-3 * scale)
        check_same(eng.plot(rel, axes), orc.plot_relation(rel, axes).data, str(scale))
    rel = W.Relation((0, 1), 2, [1.0, 0, 0, 1e-30, 0, -1e-30], W.KIND_EQ, 1e-40)
    check_same(eng.plot(rel, axes), orc.plot_relation(rel, axes).data, "tiny")


# ------------------------------------------------------------- contraction
def rand_bits(rng, shape, density):
    return (rng.random(shape) < density).astype(np.uint8)


CASES = [
    # (X vars, Y vars, keep, res by var)
    ((0, 1), (1, 2), (0, 2), {0: 70, 1: 130, 2: 65}),        # matmul, ragged
    ((0, 1), (1, 2), (2, 0), {0: 64, 1: 64, 2: 64}),          # transposed output
    ((0, 1, 2), (2, 1, 3), (1, 0, 3), {0: 9, 1: 5, 2: 77, 3: 40}),  # batched
    ((0, 1, 2), (0, 1, 2), (0, 1, 2), {0: 7, 1: 9, 2: 100}),  # Hadamard
    ((0, 1, 2), (0, 1), (2, 0), {0: 11, 1: 13, 2: 70}),       # Hadamard + reduce
    ((0, 1), (2, 3), (0, 2, 1, 3), {0: 5, 1: 6, 2: 7, 3: 66}),  # Kronecker
    ((0, 1), (0, 1), (), {0: 40, 1: 90}),                      # full contraction
    ((0, 1, 4), (1, 2, 5), (0, 2), {0: 33, 1: 65, 2: 31, 4: 3, 5: 4}),  # private axes
    ((0, 1), (1,), (0,), {0: 100, 1: 200}),                    # matrix-vector
    ((1,), (1, 2), (2,), {1: 129, 2: 300}),                    # vector-matrix
    ((0, 1, 2), (1, 2, 3), (0, 3), {0: 16, 1: 16, 2: 16, 3: 16}),  # K = two axes
    ((0, 1, 2), (2, 3), (0, 1, 3), {0: 20, 1: 20, 2: 2000, 3: 3}),  # long K, narrow N
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("density", [0.02, 0.3])
def test_contract_cases(eng, orc, case, density):
    xv, yv, keep, rmap = CASES[case]
    rng = np.random.default_rng(100 * case + int(density * 100))
    X = rand_bits(rng, tuple(rmap[v] for v in xv), density)
    Y = rand_bits(rng, tuple(rmap[v] for v in yv), density)
    vres = [rmap.get(v, 1) for v in range(max(rmap) + 1)]
    want = orc.contract(orc.Arr(X, xv), orc.Arr(Y, yv), keep, vres).data
    got = eng.contract(pack(X, xv), pack(Y, yv), keep)
    check_same(got, want, str(CASES[case]))


def test_contract_padding_garbage_ignored(eng, orc):
    """Bits beyond the last pixel of a caller's row must not change the result."""
    import torch
    rng = np.random.default_rng(5)
    X = rand_bits(rng, (50, 70), 0.2)
    Y = rand_bits(rng, (70, 33), 0.2)
    xa, ya = pack(X, (0, 1)), pack(Y, (1, 2))
    # set every padding bit of X's rows (bits 70..127 of each row)
    w = xa.words.view(torch.int64).reshape(50, 2)
    w[:, 1] |= torch.tensor(np.array([~((1 << 6) - 1)], dtype=np.int64)[0], device=w.device)
    want = orc.contract(orc.Arr(X, (0, 1)), orc.Arr(Y, (1, 2)), (0, 2), [50, 70, 33]).data
    check_same(eng.contract(xa, ya, (0, 2)), want)


# -------------------------------------------------------------- networks
def solve_both(eng, orc, sysm, **kw):
    out, st = eng.solve(sysm, **kw)
    eng.sync()
    want = orc.solve(sysm.axes, sysm.rels, sysm.exposed, strict=kw.get("strict", False)).data
    check_same(out, want, sysm.name)
    return out, st


def test_solve_circle_parabola_full(eng, orc):
    """Config 1 at its full size (256^3 box, one latent variable)."""
    out, st = solve_both(eng, orc, W.circle_parabola(res=256))
    assert st["n_joins"] == 1 and st["pixel_ops_dense"] == 256 ** 3


def test_solve_circle_parabola_no_false_negative(eng):
    sysm = W.circle_parabola(res=256)
    out, _ = eng.solve(sysm)
    got = out.to_numpy()
    lo, hi, r = sysm.axes[0]
    for z in np.linspace(-1.99, 1.99, 2001):
        y = z * z - 0.5
        if abs(y) > 1:
            continue
        for x in (np.sqrt(1 - y * y), -np.sqrt(1 - y * y)):
            assert got[int((x - lo) / ((hi - lo) / r)), int((z - lo) / ((hi - lo) / r))] == 1


@pytest.mark.parametrize("res", [64, 200, 333])
def test_solve_chain_ragged(eng, orc, res):
    solve_both(eng, orc, W.chain(res=res, nrel=8))


def test_solve_orders_identical(eng, orc):
    sysm = W.chain(res=150, nrel=6, seed=99)
    want = orc.solve(sysm.axes, sysm.rels, sysm.exposed).data
    for order, pairs in (("greedy", None), ("left", None), ("optimal", None),
                         ("given", [(4, 5), (2, 3), (0, 1), (6, 7), (8, 9)])):
        out, _ = eng.solve(sysm, order=order, pairs=pairs)
        check_same(out, want, order)


def test_solve_optimal_order_networks(eng, orc):
    """The least-naive-cost tree (Sec. 3.5) on random networks, single solves
    and one batch: the same bits as the oracle's own order (Sec. 3.3,
    associativity), for a naive cost never above greedy's."""
    nets = W.random_networks(6, seed=515, nvars_range=(8, 12), nrel_range=(10, 18),
                             res_choices=(48, 64, 100))
    outs, st = eng.solve_batch(nets, order="optimal")
    _, st_g = eng.solve_batch(nets, order="greedy")
    eng.sync()
    assert st["pixel_ops_dense"] <= st_g["pixel_ops_dense"]
    for o, sy in zip(outs, nets):
        want = orc.solve(sy.axes, sy.rels, sy.exposed).data
        check_same(o, want, sy.name)
        single, _ = eng.solve(sy, order="optimal")
        check_same(single, want, sy.name + " single")


@pytest.mark.parametrize("res", [16, 50, 64])
def test_solve_ternary(eng, orc, res):
    solve_both(eng, orc, W.ternary(res=res))


def test_solve_edge_cases(eng, orc):
    rng = W.SplitMix64(4242)
    # single relation, reduce to one exposed variable
    s1 = W.System("single", [(-2, 2, 100), (-1, 1, 77)], [random_relation(rng, 2, 2, 3)], (1,))
    solve_both(eng, orc, s1)
    # nothing exposed: one bit (does a solution exist?)
    s0 = W.System("exists", [(-2, 2, 90)] * 3,
                  [W.Relation((0, 1), 2, [-1, 0, 0, 1, 0, 1]),
                   W.Relation((1, 2), 2, [0.5, 1, 0, 0, 0, -1])], ())
    solve_both(eng, orc, s0)
    # no solution at all: x^2 + y^2 + 1 = 0
    sn = W.System("empty", [(-2, 2, 70)] * 2, [W.Relation((0, 1), 2, [1, 0, 0, 1, 0, 1])], (0, 1))
    out, _ = solve_both(eng, orc, sn)
    assert out.to_numpy().sum() == 0
    # exposed variable in no relation: broadcast along it
    sb = W.System("broadcast", [(-2, 2, 70), (-2, 2, 90), (0, 1, 5)],
                  [random_relation(rng, 2, 2, 3)], (2, 0))
    solve_both(eng, orc, sb)
    # exposed order reversed, strict comparison
    sr = W.chain(res=96, nrel=3)
    sr.exposed = (3, 0)
    solve_both(eng, orc, sr)
    solve_both(eng, orc, W.chain(res=96, nrel=3), strict=True)
    # relation with a repeated variable inside a network
    sl = W.System("loop", [(-2, 2, 80), (-2, 2, 81)],
                  [W.Relation((0, 0, 1), 2, rng.normal(10)), random_relation(rng, 2, 2, 2)], (1,))
    solve_both(eng, orc, sl)


def test_invalid_arguments_gpu(eng):
    sysm = W.chain(res=64, nrel=2)
    bad = pa.BitArray.empty((0,), (64,))
    with pytest.raises(pa.PaError) as e:
        pa.pa_solve_network(eng.ctx, sysm.axes, sysm.rels, sysm.exposed, bad)
    assert e.value.status == 1
    with pytest.raises(pa.PaError):
        pa.pa_solve_network(eng.ctx, sysm.axes, sysm.rels, sysm.exposed,
                            pa.BitArray.empty((0, 2), (64, 64)), order="given", pairs=[(0, 0)])


# ------------------------------------------------------- full-size workloads
def test_chain_2048_full(eng, orc):
    """Config 2 at full size: 8 binary cubics at 2048 per axis, 7 latent variables."""
    solve_both(eng, orc, W.chain(res=2048, nrel=8))


def test_ternary_256_full(eng, orc):
    """Config 3 at full size: four ternary cubics at 256 per axis."""
    solve_both(eng, orc, W.ternary(res=256))
