"""Failure paths and probes on the GPU, made without faulting it: a bounded
device wait that nothing completes runs out and is reported by pa_sync as
PA_ERR_TIMEOUT (the context stays usable); a workspace cap below a call's
needs gives PA_ERR_OOM before any launch; and the pipe-throughput probes that
give the kernels' rooflines return plausible per-SM rates."""
import numpy as np
import pytest

import paper_1609_00061_gb300 as pa
from paper_1609_00061_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_context_survives(orc):
    """A device wait that nothing completes gives up after its limit; pa_sync
    reports PA_ERR_TIMEOUT once, and the context keeps solving correctly."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    e = pa.Engine(0)
    pa.pa_wait_selftest(e.ctx, 2_000_000)      # 2 ms
    with pytest.raises(pa.PaError) as err:
        e.sync()
    assert err.value.status == 6
    e.sync()                                    # the error word was cleared
    sy = W.chain(res=100, nrel=3, seed=7)
    out, _ = e.solve(sy)
    e.sync()
    assert np.array_equal(out.to_numpy(), orc.solve(sy.axes, sy.rels, sy.exposed).data)
    e.close()


def test_workspace_cap_gives_oom():
    """A context whose workspace cap is below what a call needs returns
    PA_ERR_OOM before any launch, and serves smaller calls afterwards."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    e = pa.Engine(0, workspace_cap=1 << 20)
    big = W.chain(res=2048, nrel=8)
    with pytest.raises(pa.PaError) as err:
        e.solve(big)
    assert err.value.status == 4
    small = W.chain(res=64, nrel=3, seed=2)
    out, st = e.solve(small)
    e.sync()
    assert st["workspace_bytes"] <= 1 << 20
    e.close()


def test_measured_peaks_plausible():
    """The pipe probes: a GB300 SM issues at most 128 lane-operations per clock
    per pipe class, loads at most 128 shared-memory bytes per clock, and the
    clock reads between 0.5 and 2.2 GHz."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    e = pa.Engine(0)
    p = pa.pa_measure_peaks(e.ctx)
    e.close()
    print(p)
    assert p["sms"] >= 100
    assert 0.5e9 < p["sm_clock_hz"] < 2.2e9
    assert 16 <= p["lop3_per_clk_sm"] <= 128 * 1.05
    assert 32 <= p["smem_bytes_per_clk_sm"] <= 128 * 1.05
    assert 64 <= p["fp32_flops_per_clk_sm"] <= 256 * 1.05
    assert 0 < p["fp64_flops_per_clk_sm"] <= 256
