"""Pixel-array oracle: plain CPU statement of the pixel array method.

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only callers.
It shares no code with the CUDA library (``paper_1609_00061_gb300``) and neither
package imports the other.

The arithmetic lives in ``pa_oracle.c`` (plain C, ``-O2 -ffp-contract=off``);
this module only marshals numpy arrays into it and strings the pairwise
contractions of a network together.

Arrays are ``Arr`` objects: one byte per pixel (0/1), numpy shape = the
resolutions of the array's variables, axes in the order of ``Arr.vars``.

Functions (passages of Spivak et al., arXiv 1609.00061):
  valid_tolerance   Sec. 3.2, Eq. (continuity): a valid tolerance for a polynomial
  plot              Sec. 3.2, sample-in-center plot
  eval_expr, plot_expr  expression relations (Sec. 2.1, Sec. 2.4) and their plot
  plot_corner       the corner-lattice sample rule (an optional mode, not the
                    paper's rule) with valid_tolerance(corner=True)
  gam               Sec. 3.3, Algorithm 1 (all arrays at once; tiny grids)
  contract          Sec. 3.3 Eq. (GAM) on one two-array cluster (Sec. 3.5)
  contract_count    the same cluster over the counting semiring (Sec. 2.2, footnote)
  reduce            Eq. (GAM) with one array: OR over the dropped variables
  solve             the whole method: plots, then one cluster after another
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pa_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libpa_oracle.so")
_lib = None

KIND_EQ, KIND_LE, KIND_LT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile pa_oracle.c into oracle/_build/libpa_oracle.so (gcc, no FMA)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-std=c99",
           "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int)
        f64p = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.or_coeff_count.restype = ctypes.c_int64
        lib.or_coeff_count.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.or_coeff_index.restype = ctypes.c_int64
        lib.or_coeff_index.argtypes = [ctypes.c_int, ctypes.c_int, i32p]
        lib.or_eval_poly.restype = ctypes.c_double
        lib.or_eval_poly.argtypes = [ctypes.c_int, ctypes.c_int, f64p, f64p]
        lib.or_valid_tolerance.restype = ctypes.c_double
        lib.or_valid_tolerance.argtypes = [ctypes.c_int, ctypes.c_int, f64p, f64p, f64p, i32p]
        lib.or_valid_tolerance_corner.restype = ctypes.c_double
        lib.or_valid_tolerance_corner.argtypes = [ctypes.c_int, ctypes.c_int, f64p, f64p, f64p,
                                                  i32p]
        lib.or_plot_corner.restype = ctypes.c_int
        lib.or_plot_corner.argtypes = [ctypes.c_int, i32p, ctypes.c_int, ctypes.c_int, f64p,
                                       ctypes.c_int, i32p, f64p, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_int, f64p, f64p, i32p, u8p]
        lib.or_plot.restype = ctypes.c_int
        lib.or_plot.argtypes = [ctypes.c_int, ctypes.c_int, f64p, ctypes.c_int, ctypes.c_double,
                                ctypes.c_int, f64p, f64p, i32p, u8p]
        lib.or_gam.restype = ctypes.c_int
        lib.or_gam.argtypes = [ctypes.c_int, i32p, ctypes.c_int, i32p, i32p,
                               ctypes.POINTER(u8p), ctypes.c_int, i32p, u8p]
        lib.or_contract_pair.restype = ctypes.c_int
        lib.or_contract_pair.argtypes = [ctypes.c_int, i32p, u8p, ctypes.c_int, i32p, u8p,
                                         ctypes.c_int, i32p, i32p, u8p]
        lib.or_eval_expr.restype = ctypes.c_double
        lib.or_eval_expr.argtypes = [ctypes.c_int, i32p, f64p, f64p, f64p]
        lib.or_plot_expr.restype = ctypes.c_int
        lib.or_plot_expr.argtypes = [ctypes.c_int, ctypes.c_int, i32p, f64p, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int, f64p, f64p, i32p, u8p]
        lib.or_contract_count.restype = ctypes.c_int
        lib.or_contract_count.argtypes = [ctypes.c_int, i32p, u8p, ctypes.c_int, i32p, u8p,
                                          ctypes.c_int, i32p, i32p,
                                          ctypes.POINTER(ctypes.c_uint64)]
        lib.or_num_threads.restype = ctypes.c_int
        lib.or_set_num_threads.restype = None
        lib.or_set_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def num_threads() -> int:
    return int(_L().or_num_threads())


def set_num_threads(n: int) -> None:
    """Threads the oracle's loops use from now on."""
    _L().or_set_num_threads(int(n))


# ----------------------------------------------------------------- polynomials
def coeff_count(n: int, degree: int) -> int:
    return int(_L().or_coeff_count(n, degree))


def coeff_index(exps, degree: int) -> int:
    """Index of exponent tuple ``exps`` in the graded lex coefficient order of
    polynomials of total degree <= ``degree`` (-1 when the degree is too high)."""
    e, ep = _i32(exps)
    return int(_L().or_coeff_index(len(e), degree, ep))


def eval_poly(degree: int, coeffs, x) -> float:
    c, cp = _f64(coeffs)
    xx, xp = _f64(x)
    return float(_L().or_eval_poly(len(xx), degree, cp, xp))


# ------------------------------------------------------------------- plotting
@dataclass
class Arr:
    """A Boolean array over named variables (one uint8 per pixel)."""
    data: np.ndarray
    vars: tuple


def valid_tolerance(degree: int, coeffs, lo, hi, res, corner: bool = False) -> float:
    """A valid tolerance for the centre rule, or (corner) for the corner rule."""
    c, cp = _f64(coeffs)
    l, lp = _f64(lo)
    h, hp = _f64(hi)
    r, rp = _i32(res)
    fn = _L().or_valid_tolerance_corner if corner else _L().or_valid_tolerance
    return float(fn(len(r), degree, cp, lp, hp, rp))


def plot(degree: int, coeffs, kind: int, eps: float, lo, hi, res, strict: bool = False) -> np.ndarray:
    """Sample-in-center plot over the box prod [lo_p, hi_p) at resolutions res."""
    c, cp = _f64(coeffs)
    l, lp = _f64(lo)
    h, hp = _f64(hi)
    r, rp = _i32(res)
    assert len(c) == coeff_count(len(r), degree)
    out = np.zeros(tuple(int(v) for v in r), dtype=np.uint8)
    rc = _L().or_plot(len(r), degree, cp, int(kind), float(eps), int(bool(strict)), lp, hp, rp,
                      _u8(out))
    assert rc == 0
    return out


def eval_expr(ops, consts, x, with_mag: bool = False):
    """An expression relation's value at the point x (one coordinate per port);
    with_mag: also the largest magnitude of any value the program pushed."""
    o, op = _i32(ops)
    c, cp = _f64(consts if len(consts) else [0.0])
    xx, xp = _f64(x)
    mag = ctypes.c_double()
    f = float(_L().or_eval_expr(len(o), op, cp, xp, ctypes.byref(mag)))
    return (f, mag.value) if with_mag else f


def plot_expr(ops, consts, kind: int, eps: float, lo, hi, res, strict: bool = False) -> np.ndarray:
    """Sample-in-center plot of an expression relation over its ports."""
    o, op = _i32(ops)
    c, cp = _f64(consts if len(consts) else [0.0])
    l, lp = _f64(lo)
    h, hp = _f64(hi)
    r, rp = _i32(res)
    out = np.zeros(tuple(int(v) for v in r), dtype=np.uint8)
    rc = _L().or_plot_expr(len(r), len(o), op, cp, int(kind), float(eps), int(bool(strict)), lp, hp,
                           rp, _u8(out))
    assert rc == 0
    return out


RULE_CENTER, RULE_CORNER = 0, 1


def plot_corner(port_var, nv, kind: int, eps: float, lo, hi, res, strict: bool = False,
                degree: int = 0, coeffs=(), expr=None) -> np.ndarray:
    """Corner-lattice plot over the nv distinct variables; port_var[p] is the
    distinct variable port p reads.  A polynomial (degree, coeffs) or an
    expression program expr = (ops, consts)."""
    pv, pvp = _i32(port_var)
    l, lp = _f64(lo)
    h, hp = _f64(hi)
    r, rp = _i32(res)
    assert len(r) == nv
    if expr is None:
        c, cp = _f64(coeffs)
        assert len(c) == coeff_count(len(pv), degree)
        o, op = _i32([0])
        k, kp = _f64([0.0])
        nops = 0
    else:
        c, cp = _f64([0.0])
        o, op = _i32(expr[0])
        k, kp = _f64(expr[1] if len(expr[1]) else [0.0])
        nops = len(o)
    out = np.zeros(tuple(int(v) for v in r), dtype=np.uint8)
    rc = _L().or_plot_corner(len(pv), pvp, nv, int(degree), cp, nops, op, kp, int(kind),
                             float(eps), int(bool(strict)), lp, hp, rp, _u8(out))
    assert rc == 0
    return out


def relation_eps(rel, axes) -> float:
    """Tolerance of a relation: its own when given (>= 0), else a valid one
    for the relation's sample rule."""
    if rel.eps >= 0:
        return float(rel.eps)
    assert getattr(rel, "expr", None) is None, "expression relations carry their own eps"
    lo = [axes[v][0] for v in rel.vars]
    hi = [axes[v][1] for v in rel.vars]
    res = [axes[v][2] for v in rel.vars]
    corner = getattr(rel, "rule", RULE_CENTER) == RULE_CORNER
    return valid_tolerance(rel.degree, rel.coeffs, lo, hi, res, corner=corner)


def plot_relation(rel, axes, strict: bool = False) -> Arr:
    """Plot a relation over its ports (a repeated variable gives a repeated
    port); under the corner rule, over its distinct variables."""
    lo = [axes[v][0] for v in rel.vars]
    hi = [axes[v][1] for v in rel.vars]
    res = [axes[v][2] for v in rel.vars]
    eps = relation_eps(rel, axes)
    if getattr(rel, "rule", RULE_CENTER) == RULE_CORNER:
        dv = []
        for v in rel.vars:
            if v not in dv:
                dv.append(v)
        pv = [dv.index(v) for v in rel.vars]
        data = plot_corner(pv, len(dv), rel.kind, eps, [axes[v][0] for v in dv],
                           [axes[v][1] for v in dv], [axes[v][2] for v in dv], strict,
                           degree=rel.degree, coeffs=rel.coeffs,
                           expr=getattr(rel, "expr", None))
        return Arr(data, tuple(dv))
    if getattr(rel, "expr", None) is not None:
        ops, consts = rel.expr
        return Arr(plot_expr(ops, consts, rel.kind, eps, lo, hi, res, strict), tuple(rel.vars))
    return Arr(plot(rel.degree, rel.coeffs, rel.kind, eps, lo, hi, res, strict), tuple(rel.vars))


# ---------------------------------------------------------------- GAM
def gam(link_res, arrays, port_links, out_links) -> np.ndarray:
    """Algorithm 1 verbatim: all arrays at once over every link entry."""
    lr, lrp = _i32(link_res)
    nd, ndp = _i32([len(p) for p in port_links])
    flat = [l for p in port_links for l in p]
    pl, plp = _i32(flat if flat else [0])
    ol, olp = _i32(list(out_links) if len(out_links) else [0])
    arrs = [np.array(a, dtype=np.uint8, order="C") for a in arrays]
    for a, p in zip(arrs, port_links):
        assert a.shape == tuple(link_res[l] for l in p)
    ptrs = (ctypes.POINTER(ctypes.c_uint8) * max(1, len(arrs)))(*[_u8(a) for a in arrs])
    out = np.zeros(tuple(link_res[l] for l in out_links), dtype=np.uint8)
    rc = _L().or_gam(len(lr), lrp, len(arrs), ndp, plp, ptrs, len(out_links), olp, _u8(out))
    assert rc == 0
    return out


def contract(X: Arr, Y: Arr, keep, vres) -> Arr:
    """One two-array cluster: OR over every variable of X or Y not in ``keep``."""
    keep = tuple(int(v) for v in keep)
    xv, xvp = _i32(X.vars if X.vars else [0])
    yv, yvp = _i32(Y.vars if Y.vars else [0])
    kv, kvp = _i32(keep if keep else [0])
    vr, vrp = _i32(vres)
    xd = np.array(X.data, dtype=np.uint8, order="C")
    yd = np.array(Y.data, dtype=np.uint8, order="C")
    out = np.zeros(tuple(int(vres[v]) for v in keep), dtype=np.uint8)
    rc = _L().or_contract_pair(len(X.vars), xvp, _u8(xd), len(Y.vars), yvp, _u8(yd),
                               len(keep), kvp, vrp, _u8(out))
    assert rc == 0
    return Arr(out, keep)


def contract_count(X: Arr, Y: Arr, keep, vres) -> np.ndarray:
    """One cluster over the counting semiring: the number of values of the
    summed variables with X and Y both on (uint64 array shaped by keep)."""
    keep = tuple(int(v) for v in keep)
    xv, xvp = _i32(X.vars if X.vars else [0])
    yv, yvp = _i32(Y.vars if Y.vars else [0])
    kv, kvp = _i32(keep if keep else [0])
    vr, vrp = _i32(vres)
    xd = np.array(X.data, dtype=np.uint8, order="C")
    yd = np.array(Y.data, dtype=np.uint8, order="C")
    out = np.zeros(tuple(int(vres[v]) for v in keep), dtype=np.uint64)
    rc = _L().or_contract_count(len(X.vars), xvp, _u8(xd), len(Y.vars), yvp, _u8(yd), len(keep),
                                kvp, vrp, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    assert rc == 0
    return out


def reduce(X: Arr, keep, vres) -> Arr:
    """Eq. (GAM) with a single array: OR over the variables not in ``keep``."""
    one = Arr(np.ones((), dtype=np.uint8), ())
    return contract(X, one, keep, vres)


def solve(axes, rels, exposed, strict: bool = False, order=None, smallest: bool = None) -> Arr:
    """The pixel array method end to end (Sec. 3.6).

    Plots every relation, then joins arrays two at a time, summing out each
    variable as soon as no array still to be joined and no exposed variable
    uses it.  Any cluster tree gives the same result (Sec. 3.3, associativity);
    the tree only decides how large the intermediate arrays get:
      - order given: fold the plots into a running product in that order;
      - otherwise, with few relations (<= 4) fold left to right;
      - otherwise join, at every step, the two arrays whose result is smallest
        (so that loosely coupled networks stay small)."""
    vres = [int(a[2]) for a in axes]
    exposed = tuple(int(v) for v in exposed)
    plots = [plot_relation(r, axes, strict) for r in rels]
    if smallest is None:
        smallest = order is None and len(plots) > 4
    one = Arr(np.ones((), dtype=np.uint8), ())
    if not smallest:
        seq = list(range(len(plots))) if order is None else list(order)
        acc = one
        for pos, i in enumerate(seq):
            later = set(exposed)
            for j in seq[pos + 1:]:
                later.update(plots[j].vars)
            have = []
            for v in tuple(acc.vars) + tuple(plots[i].vars):
                if v in later and v not in have:
                    have.append(v)
            acc = contract(acc, plots[i], tuple(have), vres)
        return contract(acc, one, exposed, vres)
    live = list(plots)
    while len(live) > 1:
        best = None
        for i in range(len(live)):
            for j in range(i + 1, len(live)):
                later = set(exposed)
                for k, a in enumerate(live):
                    if k != i and k != j:
                        later.update(a.vars)
                keep = []
                for v in tuple(live[i].vars) + tuple(live[j].vars):
                    if v in later and v not in keep:
                        keep.append(v)
                size = 1
                for v in keep:
                    size *= vres[v]
                if best is None or size < best[0]:
                    best = (size, i, j, tuple(keep))
        _, i, j, keep = best
        joined = contract(live[i], live[j], keep, vres)
        live = [a for k, a in enumerate(live) if k not in (i, j)] + [joined]
    return contract(live[0], one, exposed, vres)
