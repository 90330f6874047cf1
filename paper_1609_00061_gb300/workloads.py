"""Seeded synthetic relation systems shaped like the pixel array method's workloads.

This module only draws inputs: variable boxes and resolutions, polynomial
coefficients and wirings.  It holds none of the method's arithmetic (no
plotting, tolerance or contraction), so the CUDA library and the CPU oracle can
both be fed from it without sharing any computation.

Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; the output mix with the
constants of Vigna's public-domain ``splitmix64.c``), 53-bit uniform doubles,
and Box-Muller for N(0, 1) coefficients.  Seeds are 0x160900061 + workload index.

Polynomial coefficient order (shared convention of the library's C interface):
graded lexicographic -- total degree 0, 1, ..., D; inside one degree the exponent
tuples (e_1, ..., e_n) in descending lexicographic order.  For two variables and
degree 3: 1, x, y, x^2, xy, y^2, x^3, x^2 y, x y^2, y^3.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from math import comb

import numpy as np

KIND_EQ, KIND_LE, KIND_LT = 0, 1, 2
SEED_BASE = 0x160900061

_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream: state += golden gamma; output = mix(state)."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self, n: int) -> np.ndarray:
        idx = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + idx * np.uint64(self.GAMMA)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * self.GAMMA) & _M64
        return z

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) with 53 random bits each."""
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        """n N(0,1) draws by Box-Muller (cosine branch), two uniforms per draw."""
        u = self.uniform(2 * n).reshape(n, 2)
        r = np.sqrt(-2.0 * np.log(1.0 - u[:, 0]))
        return r * np.cos(2.0 * np.pi * u[:, 1])

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """n integers uniform on [lo, hi] (inclusive)."""
        span = hi - lo + 1
        return lo + np.floor(self.uniform(n) * span).astype(np.int64)


def coeff_count(n: int, degree: int) -> int:
    return comb(n + degree, degree)


@dataclass
class Relation:
    """f(x_vars) S 0 with f a polynomial; S is =, <= or < by ``kind``."""
    vars: tuple
    degree: int
    coeffs: np.ndarray
    kind: int = KIND_EQ
    eps: float = -1.0          # < 0: the solver derives a valid tolerance

    def __post_init__(self):
        self.vars = tuple(int(v) for v in self.vars)
        self.coeffs = np.ascontiguousarray(self.coeffs, dtype=np.float64)
        assert len(self.coeffs) == coeff_count(len(self.vars), self.degree)


@dataclass
class System:
    """Relations over variables 0..nvars-1 with a box and resolution per variable."""
    name: str
    axes: list                 # per variable: (lo, hi, res), range [lo, hi)
    rels: list
    exposed: tuple
    meta: dict = field(default_factory=dict)

    @property
    def nvars(self) -> int:
        return len(self.axes)


def random_cubic(rng: SplitMix64, arity: int, degree: int = 3) -> np.ndarray:
    return rng.normal(coeff_count(arity, degree))


def circle_parabola(res: int = 256, lo: float = -2.0, hi: float = 2.0) -> System:
    """x^2 + y^2 - 1 = 0 and y - z^2 + 1/2 = 0 over [-2, 2)^3; y latent, (x, z) exposed."""
    r1 = Relation((0, 1), 2, [-1.0, 0.0, 0.0, 1.0, 0.0, 1.0])
    r2 = Relation((1, 2), 2, [0.5, 1.0, 0.0, 0.0, 0.0, -1.0])
    axes = [(lo, hi, res)] * 3
    return System(f"circle_parabola_r{res}", axes, [r1, r2], (0, 2))


def chain(res: int = 2048, nrel: int = 8, lo: float = -3.0, hi: float = 3.0,
          seed: int = SEED_BASE + 2) -> System:
    """nrel binary cubics R_k(v_k, v_{k+1}) with N(0,1) coefficients; ends exposed."""
    rng = SplitMix64(seed)
    rels = [Relation((k, k + 1), 3, random_cubic(rng, 2)) for k in range(nrel)]
    axes = [(lo, hi, res)] * (nrel + 1)
    return System(f"chain{nrel}_r{res}", axes, rels, (0, nrel))


def ternary(res: int = 256, lo: float = -2.0, hi: float = 2.0,
            seed: int = SEED_BASE + 3) -> System:
    """Four ternary cubics on overlapping triples of six variables:
    R1(v1,v4,v5), R2(v4,v5,v6), R3(v6,v2,v3), R4(v1,v2,v3); (v1,v2,v3) exposed
    (0-based ids 0..5 for v1..v6)."""
    rng = SplitMix64(seed)
    wiring = [(0, 3, 4), (3, 4, 5), (5, 1, 2), (0, 1, 2)]
    rels = [Relation(w, 3, random_cubic(rng, 3)) for w in wiring]
    axes = [(lo, hi, res)] * 6
    return System(f"ternary_r{res}", axes, rels, (0, 1, 2))


def batched_chains(nsys: int = 4096, seed: int = SEED_BASE + 4, res_choices=None,
                   min_len: int = 2, max_len: int = 6) -> list:
    """Independent chains of L ~ U{min_len..max_len} binary cubics over L+1
    variables; per variable a resolution drawn from ``res_choices`` (default
    64, 128, ..., 1024) and a sub-box [lo, hi) of [-4, 4) with hi - lo >= 0.5."""
    rng = SplitMix64(seed)
    if res_choices is None:
        res_choices = [64 * k for k in range(1, 17)]
    res_choices = list(res_choices)
    out = []
    for s in range(nsys):
        L = int(rng.integers(min_len, max_len, 1)[0])
        axes = []
        for _ in range(L + 1):
            r = int(res_choices[int(rng.integers(0, len(res_choices) - 1, 1)[0])])
            while True:
                a, b = sorted(float(v) for v in (-4.0 + 8.0 * rng.uniform(2)))
                if b - a >= 0.5:
                    break
            axes.append((a, b, r))
        rels = [Relation((k, k + 1), 3, random_cubic(rng, 2)) for k in range(L)]
        out.append(System(f"batch{s}", axes, rels, (0, L)))
    return out


def random_network(rng: SplitMix64, nvars_range=(10, 16), nrel_range=(12, 20),
                   res_choices=(128, 256, 512), nexp_range=(2, 3), lo=-2.0, hi=2.0,
                   window=4) -> System:
    """A random relation network: nrel relations of arity 2-3 (cubics with N(0,1)
    coefficients) over nvars variables on a line, each relation drawing its
    variables from a window of `window` consecutive ones (so the network stays
    tree-like), every variable used at least once, 2-3 exposed variables."""
    nv = int(rng.integers(nvars_range[0], nvars_range[1], 1)[0])
    nr = int(rng.integers(nrel_range[0], nrel_range[1], 1)[0])
    res = int(res_choices[int(rng.integers(0, len(res_choices) - 1, 1)[0])])
    rels = []
    # a path through all variables first, so every one is used and linked
    for k in range(nv - 1):
        if len(rels) >= nr:
            break
        if k + 2 < nv and rng.uniform(1)[0] < 0.35:
            vs = (k, k + 1, k + 2)
        else:
            vs = (k, k + 1)
        rels.append(Relation(vs, 3, random_cubic(rng, len(vs))))
    covered = set(v for r in rels for v in r.vars)
    for v in range(nv):
        if v not in covered:
            rels.append(Relation((v - 1, v), 3, random_cubic(rng, 2)))
    while len(rels) < nr:
        s0 = int(rng.integers(0, max(0, nv - window), 1)[0])
        ar = int(rng.integers(2, 3, 1)[0])
        pool = list(range(s0, min(nv, s0 + window)))
        vs = []
        while len(vs) < ar:
            v = pool[int(rng.integers(0, len(pool) - 1, 1)[0])]
            if v not in vs:
                vs.append(v)
        rels.append(Relation(tuple(vs), 3, random_cubic(rng, ar)))
    ne = int(rng.integers(nexp_range[0], nexp_range[1], 1)[0])
    exposed = []
    while len(exposed) < ne:
        v = int(rng.integers(0, nv - 1, 1)[0])
        if v not in exposed:
            exposed.append(v)
    axes = [(lo, hi, res)] * nv
    return System(f"net_v{nv}_r{len(rels)}_res{res}", axes, rels, tuple(exposed))


def random_networks(n: int, seed: int = SEED_BASE + 5, **kw) -> list:
    rng = SplitMix64(seed)
    return [random_network(rng, **kw) for _ in range(n)]


def workload(name: str, **kw):
    """Named workloads: 'circle_parabola', 'chain', 'ternary', 'batched_chains'."""
    return {"circle_parabola": circle_parabola, "chain": chain, "ternary": ternary,
            "batched_chains": batched_chains}[name](**kw)
