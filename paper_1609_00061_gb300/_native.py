"""Build and load the engine's shared library (libpa_gb300.so) and declare its C ABI.

The library is compiled in-tree for sm_103a only.  There is no fallback: if the
library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_HERE, "libpa_gb300.so")
_ROOT = os.path.dirname(_HERE)
INCLUDE = os.path.join(_ROOT, "include")

CU_SOURCES = ["api.cu", "plot.cu", "contract.cu", "mlp.cu", "mma.cu", "expr.cu", "probe.cu"]
CPP_SOURCES = ["planner.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _sources():
    return [os.path.join(_CSRC, f) for f in CU_SOURCES + CPP_SOURCES] + \
        [os.path.join(_CSRC, f) for f in os.listdir(_CSRC) if f.endswith((".h", ".cuh"))] + \
        [os.path.join(INCLUDE, "pa.h")]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit (in parallel) and link libpa_gb300.so."""
    srcs = _sources()
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(s) for s in srcs)):
        return LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", f"-I{INCLUDE}",
              "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math"]
    jobs = []
    for f in CU_SOURCES:
        obj = os.path.join(_BUILD, f.replace(".cu", ".o"))
        jobs.append([nvcc, *ARCH, *common, "-c", os.path.join(_CSRC, f), "-o", obj])
    for f in CPP_SOURCES:
        obj = os.path.join(_BUILD, f.replace(".cpp", ".o"))
        jobs.append([nvcc, *common, "-x", "c++", "-c", os.path.join(_CSRC, f), "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    # an object is rebuilt when it is older than its source or any header
    headers = max(os.path.getmtime(s) for s in srcs if s.endswith((".h", ".cuh")))

    def stale(job):
        obj, src = job[-1], job[-3]
        return (force or not os.path.exists(obj)
                or os.path.getmtime(obj) < max(os.path.getmtime(src), headers))

    todo = [j for j in jobs if stale(j)]
    if todo:
        with ThreadPoolExecutor(max_workers=len(todo)) as pool:
            list(pool.map(run, todo))
    objs = [j[-1] for j in jobs]
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


# ----------------------------------------------------------------- C structs
MAX_DIM = 8
c_i32, c_i64, c_f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double


class PaAxis(ctypes.Structure):
    _fields_ = [("lo", c_f64), ("hi", c_f64), ("res", c_i32)]


class PaExpr(ctypes.Structure):
    _fields_ = [("nops", c_i32), ("ops", ctypes.POINTER(c_i32)), ("nconsts", c_i32),
                ("consts", ctypes.POINTER(c_f64))]


class PaRelation(ctypes.Structure):
    _fields_ = [("arity", c_i32), ("vars", c_i32 * MAX_DIM), ("degree", c_i32),
                ("coeffs", ctypes.POINTER(c_f64)), ("kind", c_i32), ("eps", c_f64),
                ("expr", ctypes.POINTER(PaExpr)), ("rule", c_i32)]


class PaArray(ctypes.Structure):
    _fields_ = [("words", ctypes.c_void_p), ("ndim", c_i32), ("vars", c_i32 * MAX_DIM),
                ("res", c_i32 * MAX_DIM)]


class PaOptions(ctypes.Structure):
    _fields_ = [("strict", c_i32), ("order", c_i32), ("npairs", c_i32),
                ("pairs", ctypes.POINTER(c_i32)), ("model", ctypes.c_void_p), ("ncand", c_i32)]


class PaStats(ctypes.Structure):
    _fields_ = [("pixels_plotted", c_f64), ("pixel_ops_dense", c_f64),
                ("words_or_executed", c_f64), ("n_plots", c_i32), ("n_joins", c_i32),
                ("n_reshapes", c_i32), ("n_launches", c_i32), ("peak_words", c_i64),
                ("workspace_bytes", c_i64), ("mma_macs", c_f64), ("n_mma", c_i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PaRates(ctypes.Structure):
    _fields_ = [("rowor_words_per_us", c_f64), ("rowor_words_per_us_dense", c_f64),
                ("mma_macs_per_us", c_f64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PaPeaks(ctypes.Structure):
    _fields_ = [("sms", c_i32), ("sm_clock_hz", c_f64), ("lop3_ops_per_s", c_f64),
                ("lop3_per_clk_sm", c_f64), ("smem_bytes_per_s", c_f64),
                ("smem_bytes_per_clk_sm", c_f64), ("fp32_flops_per_s", c_f64),
                ("fp32_flops_per_clk_sm", c_f64), ("fp64_flops_per_s", c_f64),
                ("fp64_flops_per_clk_sm", c_f64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PaSystem(ctypes.Structure):
    _fields_ = [("nvars", c_i32), ("axes", ctypes.POINTER(PaAxis)), ("nrel", c_i32),
                ("rels", ctypes.POINTER(PaRelation)), ("nexposed", c_i32),
                ("exposed", ctypes.POINTER(c_i32))]


EXPORTS = ["pa_create", "pa_destroy", "pa_last_error", "pa_sync", "pa_array_words",
           "pa_profile_enable", "pa_profile_read",
           "pa_valid_tolerance", "pa_plot", "pa_contract", "pa_contract_count",
           "pa_solve_network", "pa_solve_batch",
           "pa_batch_create", "pa_batch_run", "pa_batch_stats", "pa_batch_destroy",
           "pa_solve_network_static", "pa_plan_order", "pa_tree_cost",
           "pa_mlp_create", "pa_mlp_destroy", "pa_mlp_num_params", "pa_mlp_get_params",
           "pa_mlp_set_params", "pa_mlp_get_grads", "pa_mlp_forward", "pa_mlp_backward",
           "pa_mlp_adam", "pa_join_log", "pa_plan_learned",
           "pa_set_contract_path", "pa_autotune", "pa_get_rates", "pa_set_rates",
           "pa_measure_peaks", "pa_wait_selftest"]

_lib = None


def load(build_if_missing: bool = True):
    """Load libpa_gb300.so (building it first when allowed).  Raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise RuntimeError(f"{LIB_PATH} is missing; run __graft_entry__.build()")
        build()
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    lib.pa_create.argtypes = [P(vp), ctypes.c_int, ctypes.c_size_t]
    lib.pa_create.restype = c_i32
    lib.pa_destroy.argtypes = [vp]
    lib.pa_destroy.restype = None
    lib.pa_last_error.argtypes = [vp]
    lib.pa_last_error.restype = ctypes.c_char_p
    lib.pa_sync.argtypes = [vp, vp]
    lib.pa_sync.restype = c_i32
    lib.pa_profile_enable.argtypes = [vp, c_i32]
    lib.pa_profile_enable.restype = c_i32
    lib.pa_profile_read.argtypes = [vp, c_i32, ctypes.c_char_p, P(c_i64), P(c_f64), P(c_i32)]
    lib.pa_profile_read.restype = c_i32
    lib.pa_array_words.argtypes = [c_i32, P(c_i32)]
    lib.pa_array_words.restype = c_i64
    lib.pa_valid_tolerance.argtypes = [P(PaRelation), P(PaAxis), c_i32, P(c_f64)]
    lib.pa_valid_tolerance.restype = c_i32
    lib.pa_plot.argtypes = [vp, P(PaRelation), P(PaAxis), c_i32, c_i32, P(PaArray), vp]
    lib.pa_plot.restype = c_i32
    lib.pa_contract.argtypes = [vp, P(PaArray), P(PaArray), c_i32, P(c_i32), P(PaArray), vp]
    lib.pa_contract.restype = c_i32
    lib.pa_wait_selftest.argtypes = [vp, c_i64, vp]
    lib.pa_wait_selftest.restype = c_i32
    lib.pa_measure_peaks.argtypes = [vp, P(PaPeaks), vp]
    lib.pa_measure_peaks.restype = c_i32
    lib.pa_contract_count.argtypes = [vp, P(PaArray), P(PaArray), c_i32, P(c_i32), vp, vp]
    lib.pa_contract_count.restype = c_i32
    lib.pa_solve_network.argtypes = [vp, c_i32, P(PaAxis), c_i32, P(PaRelation), c_i32, P(c_i32),
                                     P(PaOptions), P(PaArray), P(PaStats), vp]
    lib.pa_solve_network.restype = c_i32
    lib.pa_solve_batch.argtypes = [vp, c_i32, P(PaSystem), P(PaArray), P(PaOptions), P(PaStats), vp]
    lib.pa_solve_batch.restype = c_i32
    lib.pa_batch_create.argtypes = [vp, c_i32, P(PaSystem), P(PaArray), P(PaOptions), P(vp)]
    lib.pa_batch_create.restype = c_i32
    lib.pa_batch_run.argtypes = [vp, vp]
    lib.pa_batch_run.restype = c_i32
    lib.pa_batch_stats.argtypes = [vp, P(PaStats)]
    lib.pa_batch_stats.restype = c_i32
    lib.pa_batch_destroy.argtypes = [vp]
    lib.pa_batch_destroy.restype = None
    lib.pa_solve_network_static.argtypes = [c_i32, P(PaAxis), c_i32, P(PaRelation), c_i32,
                                            P(c_i32), P(PaOptions), P(PaArray), P(PaStats), vp]
    lib.pa_solve_network_static.restype = c_i32
    fp = P(ctypes.c_float)
    lib.pa_mlp_create.argtypes = [vp, c_i32, c_i32, ctypes.c_uint64, P(vp)]
    lib.pa_mlp_create.restype = c_i32
    lib.pa_mlp_destroy.argtypes = [vp]
    lib.pa_mlp_destroy.restype = None
    lib.pa_mlp_num_params.argtypes = [vp]
    lib.pa_mlp_num_params.restype = c_i64
    for nm in ("pa_mlp_get_params", "pa_mlp_set_params", "pa_mlp_get_grads"):
        getattr(lib, nm).argtypes = [vp, fp]
        getattr(lib, nm).restype = c_i32
    lib.pa_mlp_forward.argtypes = [vp, vp, c_i32, vp, vp]
    lib.pa_mlp_forward.restype = c_i32
    lib.pa_mlp_backward.argtypes = [vp, vp, vp, c_i32, fp, vp]
    lib.pa_mlp_backward.restype = c_i32
    lib.pa_mlp_adam.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, vp]
    lib.pa_mlp_adam.restype = c_i32
    lib.pa_join_log.argtypes = [vp, P(PaSystem), P(PaOptions), P(PaArray), c_i32, fp, fp, fp,
                                P(c_i32), vp]
    lib.pa_join_log.restype = c_i32
    lib.pa_plan_learned.argtypes = [vp, vp, c_i32, P(PaSystem), c_i32, P(c_i32), P(c_i32), fp]
    lib.pa_plan_learned.restype = c_i32
    lib.pa_plan_order.argtypes = [c_i32, P(PaAxis), c_i32, P(PaRelation), c_i32, P(c_i32), c_i32,
                                  P(c_i32), P(c_f64), P(c_i64)]
    lib.pa_plan_order.restype = c_i32
    lib.pa_tree_cost.argtypes = [c_i32, P(c_f64), c_i32, P(c_i32), P(c_i32), c_i32, P(c_i32),
                                 c_i32, P(c_i32), P(c_i32), P(c_f64), P(c_f64)]
    lib.pa_tree_cost.restype = c_i32
    lib.pa_set_contract_path.argtypes = [vp, c_i32]
    lib.pa_set_contract_path.restype = c_i32
    lib.pa_autotune.argtypes = [vp, P(PaRates), vp]
    lib.pa_autotune.restype = c_i32
    lib.pa_get_rates.argtypes = [vp, P(PaRates)]
    lib.pa_get_rates.restype = c_i32
    lib.pa_set_rates.argtypes = [vp, P(PaRates)]
    lib.pa_set_rates.restype = c_i32
    _lib = lib
    return lib
