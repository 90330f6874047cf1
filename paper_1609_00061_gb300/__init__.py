"""GB300 pixel array engine: Python binding of the C interface in include/pa.h.

The pixel array method (Spivak, Dobson, Kumari, Wu, arXiv 1609.00061) plots
every relation of a system as a Boolean pixel array and joins the plots by
Boolean generalized array multiplication until only the exposed variables are
left.  All of that runs in the CUDA kernels of libpa_gb300.so; this module only
marshals arguments (torch provides device memory and streams).

Functions keep the C names:
    pa_create, pa_valid_tolerance, pa_plot, pa_contract, pa_solve_network,
    pa_plan_order, pa_tree_cost, pa_array_words
and ``Engine`` bundles them for everyday use.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _native
from ._native import (PaArray, PaAxis, PaExpr, PaOptions, PaRates, PaRelation, PaStats,
                      PaSystem)

PA_OK = 0
STATUS = {0: "PA_OK", 1: "PA_ERR_INVALID_ARG", 2: "PA_ERR_UNSUPPORTED", 3: "PA_ERR_TOO_LARGE",
          4: "PA_ERR_OOM", 5: "PA_ERR_CUDA", 6: "PA_ERR_TIMEOUT"}
ORDERS = {"greedy": 0, "given": 1, "left": 2, "learned": 3, "optimal": 4}
N_FEATURES = 16


class PaError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _lib():
    return _native.load()


def _check(status, ctx=None):
    if status != PA_OK:
        msg = _lib().pa_last_error(ctx).decode() if ctx else ""
        raise PaError(status, msg)


# ------------------------------------------------------------- marshalling
def _axes(axes):
    arr = (PaAxis * max(1, len(axes)))()
    for i, (lo, hi, res) in enumerate(axes):
        arr[i].lo, arr[i].hi, arr[i].res = float(lo), float(hi), int(res)
    return arr


def _relations(rels):
    """Marshal relations; returns (array, coefficient arrays).  The expression
    programs stay referenced by the array's `_keep` attribute."""
    arr = (PaRelation * len(rels))()
    keep, extra = [], []
    for i, r in enumerate(rels):
        c = np.ascontiguousarray(r.coeffs, dtype=np.float64)
        keep.append(c)
        arr[i].arity = len(r.vars)
        for p, v in enumerate(r.vars):
            arr[i].vars[p] = int(v)
        arr[i].degree = int(r.degree)
        arr[i].coeffs = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        arr[i].kind = int(r.kind)
        arr[i].eps = float(r.eps)
        arr[i].rule = int(getattr(r, "rule", 0))
        ex = getattr(r, "expr", None)
        if ex is not None:
            ops = np.ascontiguousarray(ex[0], dtype=np.int32)
            consts = np.ascontiguousarray(ex[1], dtype=np.float64)
            pe = PaExpr()
            pe.nops = len(ops)
            pe.ops = ops.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            pe.nconsts = len(consts)
            pe.consts = consts.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            extra.append((ops, consts, pe))
            arr[i].expr = ctypes.pointer(pe)
    arr._keep = extra
    return arr, keep


def _i32(vals):
    vals = list(vals)
    a = (ctypes.c_int32 * max(1, len(vals)))(*[int(v) for v in vals])
    return a


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def pa_array_words(res) -> int:
    res = list(res)
    return int(_lib().pa_array_words(len(res), _i32(res)))


@dataclass
class BitArray:
    """A bit-packed Boolean array on the GPU (layout of include/pa.h)."""
    words: "object"       # torch.int64 CUDA tensor holding the uint64 words
    vars: tuple
    res: tuple

    @staticmethod
    def empty(vars, res, device=0):
        import torch
        n = pa_array_words(res)
        return BitArray(torch.empty(n, dtype=torch.int64, device=f"cuda:{device}"),
                        tuple(int(v) for v in vars), tuple(int(r) for r in res))

    def c(self) -> PaArray:
        a = PaArray()
        a.words = ctypes.c_void_p(self.words.data_ptr())
        a.ndim = len(self.vars)
        for i, (v, r) in enumerate(zip(self.vars, self.res)):
            a.vars[i] = v
            a.res[i] = r
        return a

    def to_numpy(self) -> np.ndarray:
        """Unpack to one uint8 per pixel (numpy shape = res)."""
        w = self.words.detach().cpu().numpy().view(np.uint64)
        if len(self.res) == 0:
            return np.array(int(w[0]) & 1, dtype=np.uint8)
        rw = (self.res[-1] + 63) // 64
        rows = w.reshape(-1, rw)
        bits = np.unpackbits(rows.view(np.uint8).reshape(rows.shape[0], rw * 8), axis=1,
                             bitorder="little")[:, :self.res[-1]]
        return bits.reshape(self.res)

    def padding_clean(self) -> bool:
        """True when every unused high bit of every row is zero."""
        if len(self.res) == 0:
            return (int(self.words[0].item()) & ~1) == 0
        r = self.res[-1]
        if r % 64 == 0:
            return True
        rw = (r + 63) // 64
        w = self.words.detach().cpu().numpy().view(np.uint64).reshape(-1, rw)[:, -1]
        mask = np.uint64(~((1 << (r % 64)) - 1) & ((1 << 64) - 1))
        return bool(np.all((w & mask) == 0))


# ------------------------------------------------------------- C entry points
def pa_create(device: int = 0, workspace_cap: int = 0):
    ctx = ctypes.c_void_p()
    _check(_lib().pa_create(ctypes.byref(ctx), device, workspace_cap))
    return ctx


def pa_valid_tolerance(rel, axes) -> float:
    r, keep = _relations([rel])
    out = ctypes.c_double()
    _check(_lib().pa_valid_tolerance(r, _axes(axes), len(axes), ctypes.byref(out)))
    return out.value


def pa_plot(ctx, rel, axes, out: BitArray, strict=False, stream=None):
    r, keep = _relations([rel])
    o = out.c()
    _check(_lib().pa_plot(ctx, r, _axes(axes), len(axes), int(bool(strict)), ctypes.byref(o),
                          _stream_ptr(stream)), ctx)
    return out


def pa_contract(ctx, A: BitArray, B: BitArray, keep, out: BitArray, stream=None):
    a, b, o = A.c(), B.c(), out.c()
    _check(_lib().pa_contract(ctx, ctypes.byref(a), ctypes.byref(b), len(keep), _i32(keep),
                              ctypes.byref(o), _stream_ptr(stream)), ctx)
    return out


def pa_contract_count(ctx, A: BitArray, B: BitArray, keep, counts, stream=None):
    """Counting-semiring cluster: `counts` is a CUDA int32 tensor of
    prod(res of keep) elements receiving the uint32 counts, row-major over keep."""
    a, b = A.c(), B.c()
    _check(_lib().pa_contract_count(ctx, ctypes.byref(a), ctypes.byref(b), len(keep), _i32(keep),
                                    ctypes.c_void_p(counts.data_ptr()), _stream_ptr(stream)), ctx)
    return counts


class _NetArgs:
    """The marshalled arguments of the last pa_solve_network call, reused while
    the same Python objects hold the same values.  Coefficients are not copied:
    the structures point at the callers' float64 arrays, so values changed in
    place are read by the next call as they are."""
    __slots__ = ("axes_ref", "axes_val", "rels_ref", "rels_val", "coeffs", "exposed_val",
                 "c_axes", "c_rels", "c_exposed")

    def matches(self, axes, rels, exposed) -> bool:
        if axes is not self.axes_ref or rels is not self.rels_ref or len(rels) != len(self.coeffs):
            return False
        if [tuple(a) for a in axes] != self.axes_val or tuple(exposed) != self.exposed_val:
            return False
        for r, (vs, deg, kind, eps, rule), c in zip(rels, self.rels_val, self.coeffs):
            if (r.coeffs is not c or not c.flags.c_contiguous or c.dtype != np.float64
                    or tuple(r.vars) != vs or r.degree != deg or r.kind != kind or r.eps != eps
                    or getattr(r, "rule", 0) != rule):
                return False
        return True


_last_net = None


def _network_args(axes, rels, exposed) -> _NetArgs:
    global _last_net
    n = _last_net
    if n is not None and n.matches(axes, rels, exposed):
        return n
    n = _NetArgs()
    n.axes_ref, n.rels_ref = axes, rels
    n.axes_val = [tuple(a) for a in axes]
    n.rels_val = [(tuple(r.vars), r.degree, r.kind, r.eps, getattr(r, "rule", 0)) for r in rels]
    n.exposed_val = tuple(exposed)
    n.c_axes = _axes(axes)
    n.c_rels, keep = _relations(rels)
    # reuse is allowed only while each relation's coefficients are its own
    # contiguous float64 array (no converted copy)
    n.coeffs = [k if k is r.coeffs else None for k, r in zip(keep, rels)]
    n.c_exposed = _i32(exposed)
    if all(c is not None for c in n.coeffs) and all(getattr(r, "expr", None) is None
                                                    for r in rels):
        _last_net = n
    else:
        n.coeffs = keep
    return n


_OPTS_CACHE = {}


def _array_c(a: BitArray) -> PaArray:
    """a.c(), kept on the object while its words, vars and res stay the same
    (the library only reads the structure)."""
    ptr = a.words.data_ptr()
    cached = a.__dict__.get("_c_cache")
    if cached is not None and cached[0] == ptr and cached[1] == (a.vars, a.res):
        return cached[2]
    c = a.c()
    a.__dict__["_c_cache"] = (ptr, (a.vars, a.res), c)
    return c


def pa_solve_network(ctx, axes, rels, exposed, out: BitArray, order="greedy", pairs=None,
                     strict=False, stream=None, model=None) -> dict:
    na = _network_args(axes, rels, exposed)
    r = na.c_rels
    pr = None
    if pairs is None and model is None:
        # options without pairs or a model are constant structures: built once
        key = (order, bool(strict))
        opts = _OPTS_CACHE.get(key)
        if opts is None:
            opts = _OPTS_CACHE[key] = _opts(order, strict)
    else:
        opts = _opts(order, strict, model)
    if pairs is not None:
        flat = [int(v) for p in pairs for v in p]
        pr = _i32(flat)
        opts.npairs = len(pairs)
        opts.pairs = ctypes.cast(pr, ctypes.POINTER(ctypes.c_int32))
    st = PaStats()
    o = _array_c(out)
    _check(_lib().pa_solve_network(ctx, len(axes), na.c_axes, len(rels), r, len(exposed),
                                   na.c_exposed, ctypes.byref(opts), ctypes.byref(o),
                                   ctypes.byref(st), _stream_ptr(stream)), ctx)
    return st.as_dict()


def pa_solve_network_static(axes, rels, exposed, out: BitArray, order="greedy", pairs=None,
                            strict=False, stream=None) -> dict:
    """pa_solve_network without any allocation by the library: the workspace is a
    fixed 16 MiB device array (see include/pa.h).  Runs on the current device."""
    r, keep = _relations(rels)
    opts = _opts(order, strict)
    pr = None
    if pairs is not None:
        pr = _i32([int(v) for p in pairs for v in p])
        opts.npairs = len(pairs)
        opts.pairs = ctypes.cast(pr, ctypes.POINTER(ctypes.c_int32))
    st = PaStats()
    o = out.c()
    status = _lib().pa_solve_network_static(len(axes), _axes(axes), len(rels), r, len(exposed),
                                            _i32(exposed), ctypes.byref(opts), ctypes.byref(o),
                                            ctypes.byref(st), _stream_ptr(stream))
    if status != PA_OK:
        raise PaError(status, f"static workspace would need {st.workspace_bytes} bytes"
                      if status == 3 else "")
    return st.as_dict()


def _struct_dtype(ctype, fields):
    """A numpy dtype laid out exactly like the ctypes Structure `ctype` for the
    listed (name, numpy type) fields (the others are left as padding)."""
    names, formats, offsets = [], [], []
    for name, fmt in fields:
        names.append(name)
        formats.append(fmt)
        offsets.append(getattr(ctype, name).offset)
    return np.dtype({"names": names, "formats": formats, "offsets": offsets,
                     "itemsize": ctypes.sizeof(ctype)})


_AXIS_DT = _struct_dtype(PaAxis, [("lo", "<f8"), ("hi", "<f8"), ("res", "<i4")])
_REL_DT = _struct_dtype(PaRelation, [("arity", "<i4"), ("vars", ("<i4", 8)), ("degree", "<i4"),
                                     ("coeffs", "<u8"), ("kind", "<i4"), ("eps", "<f8"),
                                     ("expr", "<u8"), ("rule", "<i4")])
_SYS_DT = _struct_dtype(PaSystem, [("nvars", "<i4"), ("axes", "<u8"), ("nrel", "<i4"),
                                   ("rels", "<u8"), ("nexposed", "<i4"), ("exposed", "<u8")])


def _systems(systems):
    """Marshal workloads.System objects into one array each of systems,
    axes, relations, coefficients and exposed variables (numpy buffers laid
    out as the C structures); returns (pointer to the systems, keep-alive list)."""
    n = len(systems)
    nax = np.array([len(sy.axes) for sy in systems], dtype=np.int64)
    nrl = np.array([len(sy.rels) for sy in systems], dtype=np.int64)
    nex = np.array([len(sy.exposed) for sy in systems], dtype=np.int64)
    axes = np.zeros(max(1, int(nax.sum())), dtype=_AXIS_DT)
    flat_axes = [a for sy in systems for a in sy.axes]
    if flat_axes:
        fa = np.array([(float(a[0]), float(a[1])) for a in flat_axes], dtype=np.float64)
        axes["lo"][:len(flat_axes)] = fa[:, 0]
        axes["hi"][:len(flat_axes)] = fa[:, 1]
        axes["res"][:len(flat_axes)] = [int(a[2]) for a in flat_axes]
    rels_all = [r for sy in systems for r in sy.rels]
    coeff_parts = [np.ascontiguousarray(r.coeffs, dtype=np.float64) for r in rels_all]
    lens = np.array([c.size for c in coeff_parts], dtype=np.int64)
    coeffs = np.concatenate(coeff_parts) if coeff_parts else np.zeros(1)
    coff = np.concatenate([[0], np.cumsum(lens)[:-1]]) if len(lens) else np.zeros(0, np.int64)
    rels = np.zeros(max(1, len(rels_all)), dtype=_REL_DT)
    m = len(rels_all)
    if m:
        ar = np.array([len(r.vars) for r in rels_all], dtype=np.int32)
        vv = np.zeros((m, 8), dtype=np.int32)
        for i, r in enumerate(rels_all):
            vv[i, :len(r.vars)] = r.vars
        rels["arity"][:m] = ar
        rels["vars"][:m] = vv
        rels["degree"][:m] = [int(r.degree) for r in rels_all]
        rels["coeffs"][:m] = coeffs.ctypes.data + 8 * coff.astype(np.uint64)
        rels["kind"][:m] = [int(r.kind) for r in rels_all]
        rels["eps"][:m] = [float(r.eps) for r in rels_all]
        rels["rule"][:m] = [int(getattr(r, "rule", 0)) for r in rels_all]
    keep = [axes, rels, coeffs]
    for i, r in enumerate(rels_all):
        ex = getattr(r, "expr", None)
        if ex is not None:
            ops = np.ascontiguousarray(ex[0], dtype=np.int32)
            consts = np.ascontiguousarray(ex[1], dtype=np.float64)
            pe = PaExpr()
            pe.nops = len(ops)
            pe.ops = ops.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            pe.nconsts = len(consts)
            pe.consts = consts.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            keep.extend([ops, consts, pe])
            rels["expr"][i] = ctypes.addressof(pe)
    exposed = np.array([v for sy in systems for v in sy.exposed] or [0], dtype=np.int32)
    keep.append(exposed)
    sysarr = np.zeros(n, dtype=_SYS_DT)
    ax0 = np.concatenate([[0], np.cumsum(nax)[:-1]]).astype(np.uint64)
    rl0 = np.concatenate([[0], np.cumsum(nrl)[:-1]]).astype(np.uint64)
    ex0 = np.concatenate([[0], np.cumsum(nex)[:-1]]).astype(np.uint64)
    sysarr["nvars"] = nax
    sysarr["axes"] = axes.ctypes.data + ax0 * np.uint64(_AXIS_DT.itemsize)
    sysarr["nrel"] = nrl
    sysarr["rels"] = rels.ctypes.data + rl0 * np.uint64(_REL_DT.itemsize)
    sysarr["nexposed"] = nex
    sysarr["exposed"] = exposed.ctypes.data + ex0 * np.uint64(4)
    keep.append(sysarr)
    return ctypes.cast(sysarr.ctypes.data, ctypes.POINTER(PaSystem)), keep


def _opts(order, strict, model=None, ncand=0):
    opts = PaOptions()
    opts.strict = int(bool(strict))
    opts.order = ORDERS[order] if isinstance(order, str) else int(order)
    opts.model = model.h if model is not None else None
    opts.ncand = int(ncand)
    return opts


def pa_solve_batch(ctx, systems, outs, order="greedy", strict=False, stream=None, model=None,
                   ncand=0) -> dict:
    """Solve many independent workloads.System objects in shared launches."""
    arr, keep = _systems(systems)
    oc = (PaArray * len(outs))(*[o.c() for o in outs])
    st = PaStats()
    _check(_lib().pa_solve_batch(ctx, len(systems), arr, oc,
                                 ctypes.byref(_opts(order, strict, model, ncand)),
                                 ctypes.byref(st), _stream_ptr(stream)), ctx)
    return st.as_dict()


class Batch:
    """A planned batch captured as one CUDA graph (pa_batch_create / pa_batch_run)."""

    def __init__(self, engine, systems, outs=None, order="greedy", strict=False, model=None,
                 ncand=0):
        self.engine = engine
        if outs is None:
            outs = [BitArray.empty(sy.exposed, [sy.axes[v][2] for v in sy.exposed], engine.device)
                    for sy in systems]
        self.outs = outs
        arr, keep = _systems(systems)
        oc = (PaArray * len(outs))(*[o.c() for o in outs])
        h = ctypes.c_void_p()
        _check(_lib().pa_batch_create(engine.ctx, len(systems), arr, oc,
                                      ctypes.byref(_opts(order, strict, model, ncand)),
                                      ctypes.byref(h)),
               engine.ctx)
        self.h = h

    def run(self, stream=None):
        _check(_lib().pa_batch_run(self.h, _stream_ptr(stream)), self.engine.ctx)

    def stats(self) -> dict:
        st = PaStats()
        _check(_lib().pa_batch_stats(self.h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if self.h:
            _lib().pa_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pa_plan_order(axes, rels, exposed, order="greedy"):
    """Join order (list of slot pairs), dense pixel-op count and peak bits; host only."""
    r, keep = _relations(rels)
    n = len(rels)
    pairs = (ctypes.c_int32 * max(1, 2 * (n - 1)))()
    ops = ctypes.c_double()
    peak = ctypes.c_int64()
    _check(_lib().pa_plan_order(len(axes), _axes(axes), n, r, len(exposed), _i32(exposed),
                                ORDERS[order], pairs, ctypes.byref(ops), ctypes.byref(peak)))
    return [(pairs[2 * t], pairs[2 * t + 1]) for t in range(n - 1)], ops.value, peak.value


def pa_tree_cost(link_res, packs, outer, clusters):
    """Serial and parallel cost of a cluster tree (host only).

    packs: list of link-index lists; outer: link indices of the outer pack;
    clusters: list of slot lists (slots 0..len(packs)-1 are packs, cluster t
    creates slot len(packs)+t)."""
    lr = (ctypes.c_double * max(1, len(link_res)))(*[float(v) for v in link_res])
    nports = _i32([len(p) for p in packs])
    plinks = _i32([l for p in packs for l in p])
    s, p = ctypes.c_double(), ctypes.c_double()
    _check(_lib().pa_tree_cost(len(link_res), lr, len(packs), nports, plinks, len(outer),
                               _i32(outer), len(clusters), _i32([len(c) for c in clusters]),
                               _i32([x for c in clusters for x in c]), ctypes.byref(s),
                               ctypes.byref(p)))
    return s.value, p.value


def pa_profile_enable(ctx, on=True):
    _check(_lib().pa_profile_enable(ctx, int(bool(on))), ctx)


def pa_profile_read(ctx) -> dict:
    """{kernel name: (launches, total ms)} since the last read; waits for the events."""
    cap = 64
    names = ctypes.create_string_buffer(32 * cap)
    launches = (ctypes.c_int64 * cap)()
    ms = (ctypes.c_double * cap)()
    n = ctypes.c_int32()
    _check(_lib().pa_profile_read(ctx, cap, names, launches, ms, ctypes.byref(n)), ctx)
    out = {}
    for k in range(min(n.value, cap)):
        nm = names.raw[32 * k:32 * k + 32].split(b"\0")[0].decode()
        out[nm] = (int(launches[k]), float(ms[k]))
    return out


def pa_sync(ctx, stream=None):
    _check(_lib().pa_sync(ctx, _stream_ptr(stream)), ctx)


PATHS = {"auto": 0, "rowor": 1, "mma": 2}


def pa_set_contract_path(ctx, path="auto"):
    """How matrix-form clusters are contracted: "auto", "rowor" or "mma"."""
    _check(_lib().pa_set_contract_path(ctx, PATHS[path] if isinstance(path, str) else int(path)),
           ctx)


def pa_autotune(ctx, stream=None) -> dict:
    """Measure the row-OR, tensor-core and expansion rates on this GPU; returns them."""
    r = PaRates()
    _check(_lib().pa_autotune(ctx, ctypes.byref(r), _stream_ptr(stream)), ctx)
    return r.as_dict()


def pa_wait_selftest(ctx, limit_ns=1_000_000, stream=None):
    """Enqueue a bounded device wait that runs out (the next pa_sync reports it)."""
    _check(_lib().pa_wait_selftest(ctx, int(limit_ns), _stream_ptr(stream)), ctx)


def pa_measure_peaks(ctx, stream=None) -> dict:
    """Measured LOP3, shared-memory, FP32 and FP64 throughput of this GPU."""
    from ._native import PaPeaks
    p = PaPeaks()
    _check(_lib().pa_measure_peaks(ctx, ctypes.byref(p), _stream_ptr(stream)), ctx)
    return p.as_dict()


def pa_get_rates(ctx) -> dict:
    r = PaRates()
    _check(_lib().pa_get_rates(ctx, ctypes.byref(r)), ctx)
    return r.as_dict()


def pa_set_rates(ctx, rates: dict):
    r = PaRates(**{k: float(v) for k, v in rates.items()})
    _check(_lib().pa_set_rates(ctx, ctypes.byref(r)), ctx)


# ------------------------------------------------------------------ Engine
class Engine:
    """One context on one GPU; allocates outputs as torch tensors."""

    def __init__(self, device: int = 0, workspace_cap: int = 0):
        self.device = device
        self.ctx = pa_create(device, workspace_cap)

    def set_path(self, path="auto"):
        pa_set_contract_path(self.ctx, path)

    def autotune(self, stream=None) -> dict:
        return pa_autotune(self.ctx, stream)

    def close(self):
        if self.ctx:
            _lib().pa_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plot(self, rel, axes, strict=False, stream=None) -> BitArray:
        dv = []
        for v in rel.vars:
            if v not in dv:
                dv.append(v)
        out = BitArray.empty(dv, [axes[v][2] for v in dv], self.device)
        return pa_plot(self.ctx, rel, axes, out, strict, stream)

    def contract(self, A: BitArray, B: BitArray, keep, stream=None) -> BitArray:
        res = {}
        for v, r in zip(A.vars + B.vars, A.res + B.res):
            res[v] = r
        out = BitArray.empty(keep, [res[v] for v in keep], self.device)
        return pa_contract(self.ctx, A, B, keep, out, stream)

    def contract_count(self, A: BitArray, B: BitArray, keep, stream=None):
        """Counts over the counting semiring (int32 tensor shaped by keep's resolutions)."""
        import torch
        res = {}
        for v, r in zip(A.vars + B.vars, A.res + B.res):
            res[v] = r
        shape = [res[v] for v in keep]
        n = 1
        for r in shape:
            n *= r
        out = torch.empty(n, dtype=torch.int32, device=f"cuda:{self.device}")
        pa_contract_count(self.ctx, A, B, keep, out, stream)
        return out.view(*shape)

    def solve(self, system, order="greedy", pairs=None, strict=False, stream=None, out=None,
              model=None):
        """Solve a workloads.System; returns (BitArray over system.exposed, stats)."""
        if out is None:
            out = BitArray.empty(system.exposed, [system.axes[v][2] for v in system.exposed],
                                 self.device)
        st = pa_solve_network(self.ctx, system.axes, system.rels, system.exposed, out, order,
                              pairs, strict, stream, model)
        return out, st

    def solve_batch(self, systems, order="greedy", strict=False, stream=None, outs=None,
                    model=None, ncand=0):
        """Solve a list of workloads.System; returns (list of BitArray, stats)."""
        if outs is None:
            outs = [BitArray.empty(sy.exposed, [sy.axes[v][2] for v in sy.exposed], self.device)
                    for sy in systems]
        st = pa_solve_batch(self.ctx, systems, outs, order, strict, stream, model, ncand)
        return outs, st

    def batch(self, systems, order="greedy", strict=False, outs=None, model=None,
              ncand=0) -> "Batch":
        return Batch(self, systems, outs, order, strict, model, ncand)

    def log_joins(self, system, order="greedy", pairs=None, model=None, stream=None):
        """Solve one system with one launch per join; returns (features [n,16],
        microseconds [n], result densities [n], output BitArray)."""
        out = BitArray.empty(system.exposed, [system.axes[v][2] for v in system.exposed],
                             self.device)
        arr, keep = _systems([system])
        opts = _opts(order, False, model)
        pr = None
        if pairs is not None:
            pr = _i32([int(v) for p in pairs for v in p])
            opts.npairs = len(pairs)
            opts.pairs = ctypes.cast(pr, ctypes.POINTER(ctypes.c_int32))
        mx = max(1, len(system.rels) - 1)
        feats = np.zeros((mx, N_FEATURES), dtype=np.float32)
        us = np.zeros(mx, dtype=np.float32)
        dens = np.zeros(mx, dtype=np.float32)
        nj = ctypes.c_int32()
        o = out.c()
        fp = ctypes.POINTER(ctypes.c_float)
        _check(_lib().pa_join_log(self.ctx, arr, ctypes.byref(opts), ctypes.byref(o), mx,
                                  feats.ctypes.data_as(fp), us.ctypes.data_as(fp),
                                  dens.ctypes.data_as(fp), ctypes.byref(nj), _stream_ptr(stream)),
               self.ctx)
        n = nj.value
        return feats[:n], us[:n], dens[:n], out

    def plan_learned(self, model, systems, ncand=0):
        """Orders PA_ORDER_LEARNED would pick: (list of pair lists, learned flags,
        predicted microseconds [n,2] = chosen, greedy)."""
        arr, keep = _systems(systems)
        total = sum(2 * (len(sy.rels) - 1) for sy in systems)
        pairs = (ctypes.c_int32 * max(1, total))()
        learned = (ctypes.c_int32 * len(systems))()
        pred = np.zeros(2 * len(systems), dtype=np.float32)
        _check(_lib().pa_plan_learned(self.ctx, model.h, len(systems), arr, int(ncand), pairs,
                                      learned, pred.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               self.ctx)
        out, off = [], 0
        for sy in systems:
            n = len(sy.rels) - 1
            out.append([(pairs[off + 2 * t], pairs[off + 2 * t + 1]) for t in range(n)])
            off += 2 * n
        return out, [bool(v) for v in learned], pred.reshape(-1, 2)

    def sync(self, stream=None):
        pa_sync(self.ctx, stream)


# ------------------------------------------------------------ cost model
class CostModel:
    """The learned join-cost model (FP32 MLP; forward, backward and Adam run in
    the library's own CUDA kernels).  Input: the 16 join features the library
    computes; output: log2(microseconds) / 8."""

    def __init__(self, engine, hidden=128, nlayers=3, seed=0x160900061):
        self.engine = engine
        self.hidden, self.nlayers = hidden, nlayers
        h = ctypes.c_void_p()
        _check(_lib().pa_mlp_create(engine.ctx, hidden, nlayers, seed, ctypes.byref(h)), engine.ctx)
        self.h = h

    @property
    def n_params(self) -> int:
        return int(_lib().pa_mlp_num_params(self.h))

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.n_params, dtype=np.float32)
        _check(_lib().pa_mlp_get_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        _check(_lib().pa_mlp_set_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def get_grads(self) -> np.ndarray:
        g = np.zeros(self.n_params, dtype=np.float32)
        _check(_lib().pa_mlp_get_grads(self.h, g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return g

    def forward(self, x, stream=None):
        """x: CUDA float32 tensor [n, 16] -> CUDA float32 tensor [n]."""
        import torch
        x = x.contiguous()
        y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        _check(_lib().pa_mlp_forward(self.h, ctypes.c_void_p(x.data_ptr()), x.shape[0],
                                     ctypes.c_void_p(y.data_ptr()), _stream_ptr(stream)),
               self.engine.ctx)
        return y

    def backward(self, x, t, stream=None) -> float:
        x, t = x.contiguous(), t.contiguous()
        loss = ctypes.c_float()
        _check(_lib().pa_mlp_backward(self.h, ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(t.data_ptr()), x.shape[0],
                                      ctypes.byref(loss), _stream_ptr(stream)), self.engine.ctx)
        return float(loss.value)

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        _check(_lib().pa_mlp_adam(self.h, lr, beta1, beta2, eps, _stream_ptr(stream)),
               self.engine.ctx)

    def train(self, X, T, epochs=200, batch=256, lr=2e-3, seed=0):
        """Minibatch Adam on (X [n,16], T [n]) numpy arrays; returns the loss history."""
        import torch
        dev = f"cuda:{self.engine.device}"
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
        Td = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).to(dev)
        n = Xd.shape[0]
        rng = np.random.default_rng(seed)
        hist = []
        for ep in range(epochs):
            perm = torch.from_numpy(rng.permutation(n)).to(dev)
            tot = 0.0
            for b0 in range(0, n, batch):
                idx = perm[b0:b0 + batch]
                tot += self.backward(Xd[idx], Td[idx]) * idx.numel()
                self.adam(lr)
            hist.append(tot / n)
        return hist

    def save(self, path):
        np.savez(path, params=self.get_params(), hidden=self.hidden, nlayers=self.nlayers)

    def load(self, path):
        d = np.load(path)
        assert int(d["hidden"]) == self.hidden and int(d["nlayers"]) == self.nlayers
        self.set_params(d["params"])

    def close(self):
        if self.h:
            _lib().pa_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
