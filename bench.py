"""Benchmark: Boolean-contraction throughput of the pixel array method on GB300.

One step = one whole solve (pa_solve_network) of the chain network: 9 variables
in [-3, 3) at 2048 pixels per axis, 8 binary cubics R_k(v_k, v_{k+1}) with N(0,1)
coefficients, v1 and v9 exposed: 8 plots, the join order, 7 Boolean 2048^3
contractions.  The metric is dense-equivalent Boolean pixel-ops per second
(the naive cost r^Lambda of every join, Sec. 3.5) for the whole job.  Each step
is a full call: the library relaunches the program it planned for the same
arguments on the previous call, but still uploads the call's descriptors and
coefficients and runs every plot and contraction kernel.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank solves its own instance (seed + rank): weak scaling,
no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Boolean contraction Gpixel-ops/s"
UNIT = "Gpixel-ops/s"
WORKLOAD = ("chain8_r2048: 9 vars in [-3,3) at 2048 px/axis, 8 binary cubics with N(0,1) "
            "coefficients (seed 0x160900061+2), v1,v9 exposed; 8 plots + 7 Boolean 2048^3 joins")


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------ clocks sampler
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
            return
        # nvidia-smi takes the host (and a driver query) while it starts:
        # wait for its first sample, so that the timed steps run with the
        # sampler already in its loop
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------ reference arm
def run_reference(args, rank):
    """The CPU oracle timed as it stands on the host cores (bounded sample)."""
    if rank != 0:
        return
    import oracle
    from paper_1609_00061_gb300 import workloads as W
    oracle.build()
    sample = reference_sample(W)
    for _ in range(args.warmup):
        oracle.solve(sample.axes, sample.rels, sample.exposed)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.solve(sample.axes, sample.rels, sample.exposed)
        times.append(time.perf_counter() - t0)
    ops = sample_ops(sample)
    ms = 1e3 * sum(times) / len(times)
    val = ops / (ms / 1e3) / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample.meta["sample"]},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample.meta["sample"]},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reference_sample(W):
    """The first 256 of 2048 rows of v1 (same pixels, same coefficients) with the
    first two relations: one 256x2048x2048 join, about a second of oracle work."""
    full = W.chain(res=2048, nrel=8)
    lo, hi, r = full.axes[0]
    axes = [(lo, lo + (hi - lo) * 256 / 2048, 256)] + list(full.axes[1:3])
    s = W.System("chain_sample", axes, full.rels[:2], (0, 2))
    s.meta["sample"] = ("chain8_r2048 rows 0..255 of v1, relations R1,R2: 2 plots + one "
                        "256x2048x2048 join per step")
    return s


def sample_ops(s):
    vres = [a[2] for a in s.axes]
    ops = 1.0
    for v in set(s.rels[0].vars) | set(s.rels[1].vars):
        ops *= vres[v]
    return ops


def cpu_baseline():
    """The oracle as it stands on the host cores: the chain sample on every core
    (the headline figure) and on one core, and the circle-parabola (256) and
    ternary (256^3 arrays) workloads in full on every core."""
    import oracle
    from paper_1609_00061_gb300 import workloads as W
    oracle.build()
    cores = oracle.num_threads()
    s = reference_sample(W)

    def timed(sy, max_s, max_n):
        oracle.solve(sy.axes, sy.rels, sy.exposed)
        t0 = time.perf_counter()
        n = 0
        while True:
            oracle.solve(sy.axes, sy.rels, sy.exposed)
            n += 1
            if time.perf_counter() - t0 > max_s or n >= max_n:
                break
        return (time.perf_counter() - t0) / n, n

    dt, n = timed(s, 10.0, 20)
    out = {"value": sample_ops(s) / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": s.meta["sample"] + f", {n} repetitions"}
    oracle.set_num_threads(1)
    try:
        dt1, n1 = timed(s, 3.0, 2)
    finally:
        oracle.set_num_threads(cores)
    out["single_core"] = {"value": sample_ops(s) / dt1 / 1e9, "unit": UNIT, "cores": 1,
                          "repetitions": n1}
    other = {}
    for sy in (W.circle_parabola(res=256), W.ternary(res=256)):
        d, k = timed(sy, 5.0, 3)
        other[sy.name] = {"ms_per_solve": d * 1e3, "cores": cores, "repetitions": k,
                          "pixel_ops_per_solve": solve_ops(sy)}
    out["other_workloads"] = other
    return out


def solve_ops(sy):
    """Naive cost sum r^Lambda of the library's greedy plan (host planning only)."""
    import paper_1609_00061_gb300 as pa
    return pa.pa_plan_order(sy.axes, sy.rels, sy.exposed)[1]


# ------------------------------------------------------------------ our arm
def fp8_tflops():
    return 2.0 * (load_peaks().get("bf16_tflops") or 1900.0)


def kernel_rooflines(kernels, stats_step, steps, sysm, pk):
    """Roofline of every kernel with a defined algorithmic work, largest share
    first; pk: the pipe peaks pa_measure_peaks measured on this GPU.  The
    contraction gets three lines: the 32-bit logic pipe on the OR work it
    executed (the bit path's roofline), the shared-memory load bandwidth on
    the table words it read, and HBM on its operand bytes."""
    out, extra = [], []
    total = sum(v[1] for k, v in kernels.items() if k != "words_or") or 1.0
    words = kernels.get("words_or", (0, 0.0))[0]
    for name, (launches, ms) in kernels.items():
        if name == "words_or" or launches == 0 or ms <= 0:
            continue
        t = ms / 1e3 / launches
        share = ms / total
        if name == "rowor_kernel":
            wl = words / launches
            # every executed table word is one 64-bit OR: two 32-bit LOP3
            ops = 2.0 * wl
            ach = ops / t / 1e9
            peak = pk["lop3_ops_per_s"] / 1e9
            out.append({"kernel": name, "bound": "alu", "achieved": ach, "peak": peak,
                        "unit": "Gop/s", "frac": ach / peak, "traffic": None,
                        "limit": f"32-bit LOP3 pipe, measured by pa_measure_peaks "
                                 f"({pk['lop3_per_clk_sm']:.1f} per SM per clock at "
                                 f"{pk['sm_clock_hz'] / 1e6:.0f} MHz)",
                        "work_per_launch": f"{wl:.4g} 64-bit table words OR-ed (2 LOP3 each), "
                                           f"counted by the kernel",
                        "share": share})
            b = 8.0 * wl
            extra.append({"kernel": name, "bound": "smem", "achieved": b / t / 1e9,
                          "peak": pk["smem_bytes_per_s"] / 1e9, "unit": "GB/s",
                          "frac": (b / t) / pk["smem_bytes_per_s"],
                          "limit": "shared-memory loads, measured by pa_measure_peaks",
                          "work_per_launch": f"{b:.4g} bytes of table words read",
                          "share": share})
            # algorithmic bytes of a Boolean r x r x r product: the bit-packed A
            # and B read once and C written once, 3 r^2 / 8 bytes
            r = sysm.axes[0][2]
            joins = (stats_step["n_joins"] - stats_step.get("n_mma", 0)) * steps
            hb = 3.0 * r * r / 8.0 * joins / launches
            hpk = load_peaks().get("hbm_gbs") or 6800.0
            extra.append({"kernel": name, "bound": "hbm", "achieved": hb / t / 1e9, "peak": hpk,
                          "unit": "GB/s", "frac": hb / t / 1e9 / hpk,
                          "limit": "HBM copy bandwidth, MEASURED_PEAKS.json",
                          "work_per_launch": f"{hb:.4g} bytes: A, B read and C written once, "
                                            f"{joins / launches:.3g} joins of {r}^3",
                          "share": share})
        elif name == "mma_bool_kernel":
            # 2 flops per multiply-add of the unpadded clusters (M x N x K each)
            macs = stats_step.get("mma_macs", 0.0) * steps / launches
            ach = 2.0 * macs / t / 1e12
            peak = fp8_tflops()
            out.append({"kernel": name, "bound": "tensor", "achieved": ach, "peak": peak,
                        "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                        "limit": "dense FP8 tensor rate: measured bf16 burst x 2 (nominal "
                                 "FP8/BF16 ratio), MEASURED_PEAKS.json",
                        "work_per_launch": f"{macs:.4g} multiply-adds",
                        "share": share})
        elif name == "plot_kernel":
            # algorithmic work per pixel: the row polynomial sum_j g_j y^j, D FMAs
            D = max(r.degree for r in sysm.rels)
            pix = stats_step["pixels_plotted"] * steps / launches
            ach = 2.0 * D * pix / t / 1e12
            peak = pk["fp32_flops_per_s"] / 1e12
            out.append({"kernel": name, "bound": "alu", "achieved": ach, "peak": peak,
                        "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                        "limit": "FP32 FMA, measured by pa_measure_peaks",
                        "work_per_launch": f"{pix:.4g} pixels x {2 * D} flops",
                        "share": share})
    out.sort(key=lambda r: -r["share"])
    return out, extra


def run_batched(eng, pa, W, dev, reps=5):
    """4096 independent chains of 2-6 binary cubics, 64-1024 px per axis, random
    sub-boxes of [-4, 4): one CUDA-graph replay of the planned batch versus one
    pa_solve_network call per system (greedy order both ways)."""
    import torch
    systems = W.batched_chains(nsys=4096, seed=W.SEED_BASE + 4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = eng.batch(systems)
    plan_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    b.run()
    torch.cuda.synchronize()
    fresh_s = time.perf_counter() - t0
    b.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        b.run()
    e1.record(stream)
    torch.cuda.synchronize()
    graph_s = e0.elapsed_time(e1) / 1e3 / reps
    st = b.stats()
    # plain: one call per system
    outs = b.outs
    for sy, o in zip(systems[:64], outs[:64]):
        pa.pa_solve_network(eng.ctx, sy.axes, sy.rels, sy.exposed, o)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for sy, o in zip(systems, outs):
        pa.pa_solve_network(eng.ctx, sy.axes, sy.rels, sy.exposed, o)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    b.close()
    return {"workload": "4096 chains of 2-6 binary cubics, 64..1024 px per axis (multiples of 64), "
                        "random sub-boxes of [-4,4), seed 0x160900061+4",
            "systems": len(systems), "batched_systems_per_s": len(systems) / graph_s,
            "batched_ms": graph_s * 1e3, "plain_systems_per_s": len(systems) / plain_s,
            "plain_ms": plain_s * 1e3, "speedup": plain_s / graph_s,
            "graph_launches": st["n_launches"], "joins": st["n_joins"],
            "tensor_core_joins": int(st["n_mma"]),
            "pixel_ops_dense": st["pixel_ops_dense"],
            "batched_gpixel_ops_per_s": st["pixel_ops_dense"] / graph_s / 1e9,
            "plan_and_capture_s": plan_s,
            "fresh_batch_systems_per_s": len(systems) / fresh_s,
            "fresh_batch_s": fresh_s,
            "workspace_bytes": st["workspace_bytes"],
            "timing": "batched: CUDA events around graph replays (blob copy included); "
                      "plain: host clock around the per-system calls, synchronised"}


def run_learned(eng, pa, W, n_eval=512, n_train=64, reps=3):
    """Random relation networks (10-16 variables, 12-20 relations of arity 2-3,
    128/256/512 px per axis, 2-3 exposed): the cost model is trained on solver
    logs of disjoint training networks, then the evaluation networks are solved
    (a) one pa_solve_network call each, greedy order; (b) as one graph-captured
    batch, greedy order; (c) as one graph-captured batch, least-naive-cost
    order (PA_ORDER_OPTIMAL); (d) as one graph-captured batch, learned order.
    Before (d) the solver logs the greedy order of every evaluation network
    (pa_join_log), so the judge compares a candidate's predicted time with
    greedy's measured one."""
    import torch
    from paper_1609_00061_gb300 import learned as L

    usable = L.usable_networks
    t0 = time.perf_counter()
    # training networks of both wirings (disjoint seeds from the evaluation sets)
    train = usable(W.random_networks(n_train, seed=W.SEED_BASE + 50))
    train += usable(W.random_networks(n_train // 2, seed=W.SEED_BASE + 51, window=8))
    X, T, D = L.collect_logs(eng, train, orders_per_system=3, seed=2)
    model = pa.CostModel(eng, hidden=128, nlayers=3, seed=W.SEED_BASE + 5)
    hist = model.train(X, T, epochs=150, batch=256, lr=2e-3)
    train_s = time.perf_counter() - t0
    drawn = W.random_networks(n_eval, seed=W.SEED_BASE + 5)
    nets = usable(drawn)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    for n in nets:
        eng.log_joins(n)          # greedy's measured join times, for the judge
    torch.cuda.synchronize()
    judge_log_s = time.perf_counter() - t0

    def time_batch(order, nets=nets):
        t0 = time.perf_counter()
        b = eng.batch(nets, order=order, model=model if order == "learned" else None)
        b.run()
        torch.cuda.synchronize()
        fresh = time.perf_counter() - t0
        b.run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            b.run()
        e1.record(stream)
        torch.cuda.synchronize()
        st = b.stats()
        st["fresh_s"] = fresh
        b.close()
        return e0.elapsed_time(e1) / 1e3 / reps, st

    g_s, g_st = time_batch("greedy")
    o_s, o_st = time_batch("optimal")
    l_s, l_st = time_batch("learned")
    _, learned_flags, pred = eng.plan_learned(model, nets)
    # the same generator with relations drawn from windows of 8 consecutive
    # variables instead of 4: looser wirings, where the greedy order is far
    # from the least naive cost on a fifth of the networks
    wide = usable(W.random_networks(256, seed=W.SEED_BASE + 6, window=8))
    for n in wide:
        eng.log_joins(n)
    torch.cuda.synchronize()
    wg_s, wg_st = time_batch("greedy", wide)
    wo_s, wo_st = time_batch("optimal", wide)
    wl_s, wl_st = time_batch("learned", wide)
    _, wide_flags, _ = eng.plan_learned(model, wide)
    outs = [pa.BitArray.empty(n.exposed, [n.axes[v][2] for v in n.exposed], eng.device)
            for n in nets]
    for n, o in zip(nets[:16], outs[:16]):
        pa.pa_solve_network(eng.ctx, n.axes, n.rels, n.exposed, o)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for n, o in zip(nets, outs):
        pa.pa_solve_network(eng.ctx, n.axes, n.rels, n.exposed, o)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t1
    model.close()
    return {"workload": "random relation networks: 10-16 vars, 12-20 relations of arity 2-3, "
                        "cubics N(0,1), 128/256/512 px per axis, 2-3 exposed, seed 0x160900061+5",
            "networks": len(nets), "networks_drawn": len(drawn),
            "networks_dropped": len(drawn) - len(nets),
            "drop_rule": f"greedy plan's largest intermediate > 2^30 bits or sum of r^Lambda "
                         f"> {L.MAX_PIXEL_OPS:.0e} pixel-ops",
            "train_networks": len(train), "train_samples": int(len(T)),
            "train_loss_first_last": [hist[0], hist[-1]], "train_s": train_s,
            "plain_greedy_systems_per_s": len(nets) / plain_s,
            "batched_greedy_systems_per_s": len(nets) / g_s,
            "batched_optimal_systems_per_s": len(nets) / o_s,
            "batched_learned_systems_per_s": len(nets) / l_s,
            "learned_vs_plain": plain_s / l_s, "learned_vs_batched_greedy": g_s / l_s,
            "optimal_vs_batched_greedy": g_s / o_s,
            "learned_orders_kept": int(sum(learned_flags)),
            "judge_log_s": judge_log_s,
            "fresh_batch_s": {"greedy": g_st["fresh_s"], "optimal": o_st["fresh_s"],
                              "learned": l_st["fresh_s"]},
            "tensor_core_joins_greedy": int(g_st["n_mma"]),
            "tensor_core_joins_optimal": int(o_st["n_mma"]),
            "tensor_core_joins_learned": int(l_st["n_mma"]),
            "pixel_ops_dense_greedy": g_st["pixel_ops_dense"],
            "pixel_ops_dense_optimal": o_st["pixel_ops_dense"],
            "pixel_ops_dense_learned": l_st["pixel_ops_dense"],
            "graph_launches": {"greedy": g_st["n_launches"], "optimal": o_st["n_launches"],
                               "learned": l_st["n_launches"]},
            "wide_windows": {
                "workload": "the same generator, relations from windows of 8 consecutive "
                            "variables, seed 0x160900061+6, 256 drawn",
                "networks": len(wide),
                "batched_greedy_systems_per_s": len(wide) / wg_s,
                "batched_optimal_systems_per_s": len(wide) / wo_s,
                "batched_learned_systems_per_s": len(wide) / wl_s,
                "learned_vs_batched_greedy": wg_s / wl_s,
                "optimal_vs_batched_greedy": wg_s / wo_s,
                "learned_orders_kept": int(sum(wide_flags)),
                "pixel_ops_dense": {"greedy": wg_st["pixel_ops_dense"],
                                    "optimal": wo_st["pixel_ops_dense"],
                                    "learned": wl_st["pixel_ops_dense"]}},
            "timing": "batched: CUDA events around graph replays; plain: host clock, "
                      "synchronised; fresh: host clock around planning, capture and the "
                      "first replay"}


def run_other(eng, pa, W, pk, reps=50):
    """The other workloads through the same calls: the circle-parabola system
    (256) and the ternary network (256^3 arrays) solved whole; the butterfly
    of Sec. 2.4 (expression relations) at the paper's printed size and at 2048
    pixels per axis; and one counting-semiring cluster of two 2048^2 chain
    plots on the tensor cores.  CUDA events on the launching stream."""
    import torch
    stream = torch.cuda.current_stream()

    def time_calls(fn, n):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    out = {}
    for sy in (W.circle_parabola(res=256), W.ternary(res=256), W.butterfly(res=125),
               W.butterfly(res=2048)):
        o = pa.BitArray.empty(sy.exposed, [sy.axes[v][2] for v in sy.exposed], eng.device)
        st = {}

        def solve(sy=sy, o=o):
            st.update(pa.pa_solve_network(eng.ctx, sy.axes, sy.rels, sy.exposed, o))
        ms = time_calls(solve, reps)
        rec = {"ms_per_solve": ms, "pixel_ops_dense": st["pixel_ops_dense"],
               "gpixel_ops_per_s": st["pixel_ops_dense"] / (ms / 1e3) / 1e9,
               "pixels_plotted": st["pixels_plotted"], "launches": st["n_launches"]}
        if sy.name.startswith("butterfly"):
            pa.pa_profile_enable(eng.ctx, True)
            for _ in range(5):
                solve()
            kern = pa.pa_profile_read(eng.ctx)
            pa.pa_profile_enable(eng.ctx, False)
            n, kms = kern.get("plot_expr_kernel", (0, 0.0))
            if n:
                rec["plot_expr_gpixels_per_s"] = st["pixels_plotted"] / (kms / n / 1e3) / 1e9
        out[sy.name] = rec
    # one counting cluster: two plots of the chain workload at 2048
    ch = W.chain(res=2048, nrel=2)
    a = eng.plot(ch.rels[0], ch.axes)
    b = eng.plot(ch.rels[1], ch.axes)
    cnt = torch.empty(2048 * 2048, dtype=torch.int32, device=f"cuda:{eng.device}")
    ms = time_calls(lambda: pa.pa_contract_count(eng.ctx, a, b, (0, 2), cnt), reps)
    tf = 2.0 * 2048 ** 3 / (ms / 1e3) / 1e12
    out["count_2048cube"] = {"ms": ms, "tflops": tf, "peak_tflops": fp8_tflops(),
                             "frac": tf / fp8_tflops(),
                             "what": "pa_contract_count of two 2048^2 chain plots (counting "
                                     "semiring, tensor cores): 2 M N K flops per call, the "
                                     "operand expansion and the permute-free epilogue included"}
    return out


def rank_system(W, rank):
    """The chain instance rank `rank` solves: same shape on every rank, its own
    coefficients (seed + rank), so per-rank work is fixed as ranks are added."""
    return W.chain(res=2048, nrel=8, seed=W.SEED_BASE + 2 + rank)


def whole_job(local, units_per_rank, world, dist=None, device="cpu"):
    """The slowest rank's duration (max over ranks) and the whole-job rate:
    every rank processed units_per_rank units, so the job processed
    world x units_per_rank in that time.  Returns (duration, rate per unit of
    duration)."""
    import torch
    t = torch.tensor([float(local)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tmax = float(t.item())
    return tmax, world * units_per_rank / tmax


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1609_00061_gb300 as pa
    from paper_1609_00061_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = local_rank
    eng = pa.Engine(dev)
    # the autotuner measures both contraction paths on this GPU; the automatic
    # path choice then weighs each cluster with those rates
    rates = eng.autotune()
    eng.set_path(args.path)
    # the pipes' peaks on this GPU: the denominators of the kernels' rooflines
    peaks_live = pa.pa_measure_peaks(eng.ctx)
    sysm = rank_system(W, rank)
    # one logged solve measures the densities of this system's intermediates,
    # which the automatic path choice then prefers to its independence estimate
    _, _, observed, _ = eng.log_joins(sysm)
    eng.sync()
    out = pa.BitArray.empty(sysm.exposed, [sysm.axes[v][2] for v in sysm.exposed], dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=f"cuda:{dev}")

    def step():
        return pa.pa_solve_network(eng.ctx, sysm.axes, sysm.rels, sysm.exposed, out)

    for _ in range(max(3, args.warmup)):
        st = step()
    torch.cuda.synchronize()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    def timed_steps(profile):
        """K steps, each bracketed by CUDA events on the launching stream.  With
        profile, the library also brackets every launch with its own events
        (per-kernel durations for the roofline); those events cost time of
        their own, so the headline value comes from the pass without them."""
        if profile:
            pa.pa_profile_enable(eng.ctx, True)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(k)         # 256 MiB write: L2 (129 MB) holds nothing of the last step
            starts[k].record(stream)
            st = step()
            ends[k].record(stream)
        torch.cuda.synchronize()
        kern = None
        if profile:
            kern = pa.pa_profile_read(eng.ctx)
            pa.pa_profile_enable(eng.ctx, False)
        per_step = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        if not profile:
            step_ms.extend(per_step)
        return sum(per_step) / args.steps, st, kern

    step_ms = []
    clocks = Clocks(dev)
    clocks.start()
    for _ in range(3):  # untimed, with the sampler running and the flush loaded
        flush.fill_(0)
        step()
    torch.cuda.synchronize()
    ms, st, _ = timed_steps(False)
    ms_prof, _, kernels = timed_steps(True)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ops = st["pixel_ops_dense"]
    ms_max, ops_per_ms = whole_job(ms, ops, world, dist, f"cuda:{dev}")
    value = ops_per_ms * 1e3 / 1e9

    # host cost of one call (the program is kept, so this is argument checks,
    # the descriptor upload and the graph launch): three calls enqueued right
    # after a synchronisation, host clock, before the device could hold the
    # host back (the library's staging ring lets the host run four calls
    # ahead); the median of 50 such groups
    groups = []
    for _ in range(50):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            step()
        groups.append((time.perf_counter() - t0) / 3 * 1e6)
    torch.cuda.synchronize()
    host_us = statistics.median(groups)

    # end to end through the public call: host coefficients in, output words out
    host_out = torch.empty(out.words.numel(), dtype=torch.int64, pin_memory=True)
    h2d = sum(r.coeffs.nbytes for r in sysm.rels) + 20 * len(sysm.axes)
    for _ in range(2):
        step()
        host_out.copy_(out.words, non_blocking=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        step()
        host_out.copy_(out.words, non_blocking=True)
        stream.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    _, ops_per_s = whole_job(e2e_s, ops, world, dist, f"cuda:{dev}")
    e2e_value = ops_per_s / 1e9

    if rank != 0:
        eng.close()
        return
    rl, rl_extra = kernel_rooflines(kernels, st, args.steps, sysm, peaks_live)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "flushed between steps (256 MiB write)",
                   "pixel_ops_per_step": ops, "parallelism": f"independent systems x{world}",
                   "contract_path": args.path, "tensor_core_joins": int(st["n_mma"]),
                   "autotuned_rates": rates,
                   "host_us_per_call": host_us,
                   "step_ms_min_median_max": [min(step_ms), statistics.median(step_ms),
                                              max(step_ms)],
                   "step_ms_first": step_ms[:5],
                   "observed_join_densities": [round(float(x), 5) for x in observed]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": int(out.words.numel() * 8)},
        "gpu_launches": int(st["n_launches"]) * args.steps,
        "peaks": {"hbm_gbs": load_peaks().get("hbm_gbs"), "fp8_tflops_derived": fp8_tflops()},
        "clocks": clk,
        "roofline": (rl[0] if rl else None),
        "roofline_other": rl[1:] + rl_extra,
        "measured_peaks": peaks_live,
        "kernels": {k: {"launches": v[0], "ms_total": v[1]} for k, v in kernels.items()
                    if k != "words_or"},
        "kernel_timing": "per-launch CUDA events on the launching stream, over a second pass "
                         f"of the same {args.steps} steps ({ms_prof:.4f} ms per step with "
                         "those events); value and ms_per_step come from the pass without them",
        "stats": st,
    }
    if not args.no_batched:
        line["batched"] = run_batched(eng, pa, W, dev)
        line["learned"] = run_learned(eng, pa, W)
        line["other_workloads"] = run_other(eng, pa, W, peaks_live)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    eng.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--path", default="auto", choices=["auto", "rowor", "mma"],
                    help="contraction path of matrix-form clusters")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
