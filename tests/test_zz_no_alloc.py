"""pa_solve_network_static: the solve for callers that cannot let the library
allocate memory (real-time loops that cannot take cudaFree's device-wide
synchronisation, serving processes whose GPU memory is budgeted by someone
else).  Its workspace is a fixed device array; its results must equal those of
pa_solve_network bit for bit, call after call, since every call reuses the
same array."""
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
    torch.cuda.set_device(0)
    e = pa.Engine(0)
    yield e
    e.close()


def reference(eng, sysm, **kw):
    out, _ = eng.solve(sysm, **kw)
    eng.sync()
    return out.to_numpy()


@pytest.mark.parametrize("make", [lambda: W.circle_parabola(res=256),
                                  lambda: W.chain(res=200, nrel=8),
                                  lambda: W.chain(res=2048, nrel=8)])
def test_static_matches_allocating_solve_twice(eng, make):
    sysm = make()
    want = reference(eng, sysm)
    for call in range(2):
        out = pa.BitArray.empty(sysm.exposed, [sysm.axes[v][2] for v in sysm.exposed])
        out.words.fill_(-1)
        st = pa.pa_solve_network_static(sysm.axes, sysm.rels, sysm.exposed, out)
        eng.sync()
        got = out.to_numpy()
        assert np.array_equal(got, want), f"call {call}: {int((got != want).sum())} pixels differ"
        assert out.padding_clean()
        assert 0 < st["workspace_bytes"] <= 16 << 20


def test_static_two_systems_back_to_back(eng):
    """The array keeps the previous call's contents: a different system right
    after must still come out exact."""
    a, b = W.chain(res=333, nrel=4, seed=3), W.ternary(res=40)
    wa, wb = reference(eng, a), reference(eng, b)
    for sysm, want in ((a, wa), (b, wb), (a, wa)):
        out = pa.BitArray.empty(sysm.exposed, [sysm.axes[v][2] for v in sysm.exposed])
        pa.pa_solve_network_static(sysm.axes, sysm.rels, sysm.exposed, out)
        eng.sync()
        assert np.array_equal(out.to_numpy(), want)


def test_static_rejects_oversized_system(eng):
    sysm = W.ternary(res=512)   # its four 512^3-bit plots alone take 64 MiB
    out = pa.BitArray.empty(sysm.exposed, [sysm.axes[v][2] for v in sysm.exposed])
    with pytest.raises(pa.PaError) as e:
        pa.pa_solve_network_static(sysm.axes, sysm.rels, sysm.exposed, out)
    assert e.value.status == 3


def test_static_rejects_learned_order(eng):
    """The learned order needs a context's cost model: refused, not replaced."""
    sysm = W.chain(res=64, nrel=3, seed=4)
    out = pa.BitArray.empty(sysm.exposed, [sysm.axes[v][2] for v in sysm.exposed])
    with pytest.raises(pa.PaError) as e:
        pa.pa_solve_network_static(sysm.axes, sysm.rels, sysm.exposed, out, order="learned")
    assert e.value.status == 1
