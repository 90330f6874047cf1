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
# Sample rules (include/pa.h, pa_rule): the paper's pixel centres, or the grid corners.
RULE_CENTER, RULE_CORNER = 0, 1
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
    """f(x_vars) S 0 with f a polynomial (coefficients in graded lex order) or,
    when ``expr`` is given, an expression program (see ``Ex``); S is =, <= or <
    by ``kind``."""
    vars: tuple
    degree: int
    coeffs: np.ndarray
    kind: int = KIND_EQ
    eps: float = -1.0          # < 0: the solver derives a valid tolerance (polynomials)
    expr: tuple = None         # (int32 instructions, float64 constants) or None
    rule: int = 0              # RULE_CENTER (the paper's) or RULE_CORNER

    def __post_init__(self):
        self.vars = tuple(int(v) for v in self.vars)
        self.coeffs = np.ascontiguousarray(self.coeffs, dtype=np.float64)
        if self.expr is None:
            assert len(self.coeffs) == coeff_count(len(self.vars), self.degree)
        else:
            ops, consts = self.expr
            self.expr = (np.ascontiguousarray(ops, dtype=np.int32),
                         np.ascontiguousarray(consts, dtype=np.float64))


# ------------------------------------------------------ expression programs
# Instruction codes of the postfix expression programs (include/pa.h, pa_expr).
X_CONST, X_VAR, X_ADD, X_SUB, X_MUL, X_DIV, X_NEG, X_ABS, X_SQRT, X_EXP, X_LOG = range(11)
X_SIN, X_COS, X_TAN, X_SINH, X_COSH, X_TANH, X_ATAN, X_POWI, X_POW = range(11, 20)


class Ex:
    """An expression of a relation's ports, built with Python operators and the
    functions below, written out as the postfix program the library runs.
    Only the program is built here; nothing is evaluated.

        x, y = Ex.port(0), Ex.port(1)
        rel = expr_relation((vx, vy), x ** 2 + 3 * abs_(x - y) - 5, eps=0.05)
    """

    def __init__(self, code):
        self.code = code          # list of (op, arg) with constants as floats

    @staticmethod
    def port(p):
        return Ex([(X_VAR, int(p))])

    @staticmethod
    def const(c):
        return Ex([(X_CONST, float(c))])

    @staticmethod
    def wrap(v):
        return v if isinstance(v, Ex) else Ex.const(v)

    def _bin(self, other, op, swap=False):
        a, b = (Ex.wrap(other), self) if swap else (self, Ex.wrap(other))
        return Ex(a.code + b.code + [(op, 0)])

    def __add__(self, o): return self._bin(o, X_ADD)
    def __radd__(self, o): return self._bin(o, X_ADD, True)
    def __sub__(self, o): return self._bin(o, X_SUB)
    def __rsub__(self, o): return self._bin(o, X_SUB, True)
    def __mul__(self, o): return self._bin(o, X_MUL)
    def __rmul__(self, o): return self._bin(o, X_MUL, True)
    def __truediv__(self, o): return self._bin(o, X_DIV)
    def __rtruediv__(self, o): return self._bin(o, X_DIV, True)
    def __neg__(self): return Ex(self.code + [(X_NEG, 0)])

    def __pow__(self, o):
        if isinstance(o, int):
            return Ex(self.code + [(X_POWI, o)])
        return self._bin(o, X_POW)

    def program(self):
        """(int32 instructions, float64 constants): op | (arg << 8) per instruction."""
        consts, ops = [], []
        for op, arg in self.code:
            if op == X_CONST:
                key = np.float64(arg).tobytes()
                idx = next((i for i, c in enumerate(consts) if np.float64(c).tobytes() == key),
                           None)
                if idx is None:
                    idx = len(consts)
                    consts.append(arg)
                arg = idx
            ops.append(op + 256 * int(arg))
        return (np.array(ops, dtype=np.int32), np.array(consts, dtype=np.float64))


def _fn(op):
    return lambda e: Ex(Ex.wrap(e).code + [(op, 0)])


abs_, sqrt_, exp_, log_, sin_, cos_, tan_ = (_fn(X_ABS), _fn(X_SQRT), _fn(X_EXP), _fn(X_LOG),
                                             _fn(X_SIN), _fn(X_COS), _fn(X_TAN))
sinh_, cosh_, tanh_, atan_ = _fn(X_SINH), _fn(X_COSH), _fn(X_TANH), _fn(X_ATAN)


def expr_relation(vars_, e: Ex, kind: int = KIND_EQ, eps: float = 0.05) -> Relation:
    """The relation e(ports) S 0 over the given variables (port p reads vars_[p])."""
    return Relation(tuple(vars_), 0, np.zeros(1), kind, eps, Ex.wrap(e).program())


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


def butterfly(res: int = 50, lo: float = -3.0, hi: float = 3.0, eps: float = 0.05,
              exposed=(0, 3)) -> System:
    """The butterfly example of Sec. 2.4: variables w, x, y, z (ids 0..3) in
    [-3, 3) at `res` pixels, (w, z) exposed;
      cos(ln(z^2 + 1e-3 x)) - x + 1e-5 / z = 0,
      cosh(w + 1e-3 y) + y + 1e-4 w - 2 = 0,
      tan(x + y) / ((x - 2)(x + 3) y^2) - 1 = 0.
    The paper times it at resolution 50 with x and z exposed (exposed=(1, 3))
    and prints the plot at 125 with (w, z) exposed; it states no tolerance, so
    eps is a parameter."""
    w, x, y, z = (Ex.port(p) for p in range(4))
    e1 = cos_(log_(z ** 2 + 1e-3 * x)) - x + 1e-5 / z
    e2 = cosh_(w + 1e-3 * y) + y + 1e-4 * w - 2.0
    e3 = tan_(x + y) / ((x - 2.0) * (x + 3.0) * y ** 2) - 1.0
    rels = [expr_relation((0, 1, 2, 3), e1, eps=eps), expr_relation((0, 1, 2, 3), e2, eps=eps),
            expr_relation((0, 1, 2, 3), e3, eps=eps)]
    # each relation reads only its own variables: ports not used by the
    # expression are dropped from its variable list below
    rels = [_used_ports(r) for r in rels]
    return System(f"butterfly_r{res}", [(lo, hi, res)] * 4, rels, tuple(exposed))


def _used_ports(rel: Relation) -> Relation:
    """The same relation over only the ports its program reads (renumbered)."""
    ops, consts = rel.expr
    used = sorted({int(o) >> 8 for o in ops if (int(o) & 0xff) == X_VAR})
    remap = {p: i for i, p in enumerate(used)}
    new_ops = np.array([(o & 0xff) + 256 * remap[o >> 8] if (o & 0xff) == X_VAR else o
                        for o in (int(v) for v in ops)], dtype=np.int32)
    return Relation(tuple(rel.vars[p] for p in used), 0, rel.coeffs, rel.kind, rel.eps,
                    (new_ops, consts))


def input_exemplar(eps: float = 0.05) -> System:
    """The input exemplar of Sec. 2.1: u, v, x, y in [-2, 2) at 50 and w, z in
    [-1, 1) at 80 (ids u0 v1 w2 x3 y4 z5), (v, z) exposed;
      x^2 + 3|x - y| - 5 = 0,  y^2 v^3 - w^5 <= 0,  cos(u + z x) - w^2 = 0."""
    x, y = Ex.port(0), Ex.port(1)
    r1 = expr_relation((3, 4), x ** 2 + 3.0 * abs_(x - y) - 5.0, eps=eps)
    y2, v2, w2 = Ex.port(0), Ex.port(1), Ex.port(2)
    r2 = expr_relation((4, 1, 2), y2 ** 2 * v2 ** 3 - w2 ** 5, KIND_LE, eps=eps)
    u3, z3, x3, w3 = Ex.port(0), Ex.port(1), Ex.port(2), Ex.port(3)
    r3 = expr_relation((0, 5, 3, 2), cos_(u3 + z3 * x3) - w3 ** 2, eps=eps)
    axes = [(-2.0, 2.0, 50), (-2.0, 2.0, 50), (-1.0, 1.0, 80), (-2.0, 2.0, 50), (-2.0, 2.0, 50),
            (-1.0, 1.0, 80)]
    return System("input_exemplar", axes, [r1, r2, r3], (1, 5))


def arrays_3d(res: int = 75, eps: float = 0.05) -> System:
    """The 3-D arrays example of Sec. 2.4: v, x, z in [-3, 3) and w, y in
    [-2.5, 2.5) at `res` (ids v0 w1 x2 y3 z4), (w, y) exposed;
      tan(y + w) + exp(x) - 2 = 0,  x^3 + cos(ln(y^2)) - 1.5 v = 0,
      w + z + 0.1 v - 0.5 = 0."""
    y, w, x = Ex.port(0), Ex.port(1), Ex.port(2)
    r1 = expr_relation((3, 1, 2), tan_(y + w) + exp_(x) - 2.0, eps=eps)
    x2, y2, v2 = Ex.port(0), Ex.port(1), Ex.port(2)
    r2 = expr_relation((2, 3, 0), x2 ** 3 + cos_(log_(y2 ** 2)) - 1.5 * v2, eps=eps)
    w3, z3, v3 = Ex.port(0), Ex.port(1), Ex.port(2)
    r3 = expr_relation((1, 4, 0), w3 + z3 + 0.1 * v3 - 0.5, eps=eps)
    axes = [(-3.0, 3.0, res), (-2.5, 2.5, res), (-3.0, 3.0, res), (-2.5, 2.5, res),
            (-3.0, 3.0, res)]
    return System(f"arrays3d_r{res}", axes, [r1, r2, r3], (1, 3))


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
