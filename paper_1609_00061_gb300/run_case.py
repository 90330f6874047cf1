"""Run one named case of the engine and print its timing: the entry point that
kernel profiles (ncu) are taken on.

    python -m paper_1609_00061_gb300.run_case contract --res 2048 --density 0.02 --path mma
    python -m paper_1609_00061_gb300.run_case chain --res 2048 --path auto
    python -m paper_1609_00061_gb300.run_case networks --count 40 --path auto

contract: one Boolean matrix product X[r][r] x Y[r][r] of random bits of the
given density (seeded), `--reps` times after two warm-up calls.
chain: the 9-variable chain of 8 binary cubics at `--res` pixels per axis
(with --path auto, one logged solve first measures its intermediates'
densities for the path choice).
networks: `--count` random relation networks (10-16 variables, 12-20
relations, 128/256/512 pixels per axis), planned once as a batch and replayed.
"""
from __future__ import annotations

import argparse
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["contract", "chain", "networks"])
    ap.add_argument("--res", type=int, default=2048)
    ap.add_argument("--density", type=float, default=0.02)
    ap.add_argument("--count", type=int, default=40)
    ap.add_argument("--path", default="auto", choices=["auto", "rowor", "mma"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=1)
    args = ap.parse_args(argv)

    import torch

    import paper_1609_00061_gb300 as pa
    from paper_1609_00061_gb300 import workloads as W

    eng = pa.Engine(0)
    eng.set_path(args.path)
    if args.case == "contract":
        rng = np.random.default_rng(args.seed)
        r = args.res

        def rand_bits(vars_):
            bits = (rng.random((r, r)) < args.density).astype(np.uint8)
            words = np.packbits(bits, axis=1, bitorder="little").view(np.uint64).reshape(-1)
            t = torch.from_numpy(words.view(np.int64).copy()).cuda()
            return pa.BitArray(t, vars_, (r, r))

        X, Y = rand_bits((0, 1)), rand_bits((1, 2))

        def run():
            eng.contract(X, Y, (0, 2))
    elif args.case == "chain":
        sysm = W.chain(res=args.res, nrel=8)
        if args.path == "auto":
            eng.log_joins(sysm)

        def run():
            eng.solve(sysm)
    else:
        nets = W.random_networks(args.count, seed=W.SEED_BASE + 5)
        nets = [n for n in nets if pa.pa_plan_order(n.axes, n.rels, n.exposed)[2] <= (1 << 30)]
        batch = eng.batch(nets)
        run = batch.run
    for _ in range(2):
        run()
    eng.sync()
    t0 = time.perf_counter()
    for _ in range(args.reps):
        run()
    eng.sync()
    dt = (time.perf_counter() - t0) / args.reps
    print(f"{args.case} path={args.path}: {dt * 1e6:.1f} us per run (host clock, synchronised)")
    eng.close()


if __name__ == "__main__":
    main()
