"""ctypes view of libskipper's C ABI (include/skipper.h) and its in-tree build.

Argument marshalling only: every step of the matching runs in the CUDA
kernels of ``csrc/``.  If the shared library is missing, loading fails with an
ImportError -- there is no fallback path.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import os
import shutil
import subprocess
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
CSRC = os.path.join(_PKG, "csrc")
INCLUDE = os.path.join(_ROOT, "include")
LIB_DIR = os.path.join(_PKG, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libskipper.so")
SOURCES = ["sweep.cu", "check.cu", "api.cu", "noalloc.cu", "multi.cu", "coo.cu", "server.cu", "batch.cu"]
HEADERS = ["state.cuh", "internal.h", "walk.cuh", "checkwalk.cuh"]

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a (in parallel) and link libskipper.so in-tree."""
    os.makedirs(LIB_DIR, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "skipper.h")]
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    nvcc = _nvcc()
    cuda_home = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    objs = []

    def compile_one(src):
        obj = os.path.join(LIB_DIR, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH_FLAGS, *NVCC_FLAGS, "-I", INCLUDE, "-I", CSRC, "-c",
               os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH_FLAGS, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath," + os.path.join(cuda_home, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    for o in objs:
        os.remove(o)
    return LIB_PATH


# ----------------------------------------------------------------------------
# ABI structs (layout of include/skipper.h)
# ----------------------------------------------------------------------------
class Options(ctypes.Structure):
    _fields_ = [
        ("status_bits", ctypes.c_uint32),
        ("serial", ctypes.c_uint32),
        ("grain", ctypes.c_uint32),
        ("block_threads", ctypes.c_uint32),
        ("blocks_per_sm", ctypes.c_uint32),
        ("nosync", ctypes.c_uint32),
        ("timing", ctypes.c_uint32),
        ("use_graph", ctypes.c_uint32),
        ("l2_persist", ctypes.c_uint32),
        ("stats", ctypes.c_uint32),
        ("spin_limit", ctypes.c_uint64),
        ("poison_vertex", ctypes.c_uint64),
        ("symmetric", ctypes.c_uint32),
        ("id_loads", ctypes.c_uint32),
        ("stage_windows", ctypes.c_uint32),
        ("warps_per_graph", ctypes.c_uint32),
        ("unit_order", ctypes.c_uint32),
        ("reserved32", ctypes.c_uint32),
        ("reserved", ctypes.c_uint64 * 1),
    ]


class Timing(ctypes.Structure):
    _fields_ = [
        ("init_ms", ctypes.c_float),
        ("sweep_ms", ctypes.c_float),
        ("compact_ms", ctypes.c_float),
        ("total_ms", ctypes.c_float),
        ("units", ctypes.c_uint64),
        ("reserved", ctypes.c_uint64 * 3),
    ]


class GraphDesc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64),
        ("nnz", ctypes.c_uint64),
        ("offsets", ctypes.c_void_p),
        ("nbrs", ctypes.c_void_p),
        ("mate", ctypes.c_void_p),
    ]


class Verdict(ctypes.Structure):
    _fields_ = [
        ("flags", ctypes.c_uint32),
        ("pad", ctypes.c_uint32),
        ("n_matched", ctypes.c_uint64),
        ("n_pairs", ctypes.c_uint64),
        ("n_bad_range", ctypes.c_uint64),
        ("n_asym", ctypes.c_uint64),
        ("n_nonedge", ctypes.c_uint64),
        ("n_uncovered", ctypes.c_uint64),
        ("n_pairs_bad", ctypes.c_uint64),
        ("first_bad_vertex", ctypes.c_uint64),
        ("first_uncovered", ctypes.c_uint64),
    ]
    FIELDS = ("flags", "n_matched", "n_pairs", "n_bad_range", "n_asym", "n_nonedge",
              "n_uncovered", "n_pairs_bad", "first_bad_vertex", "first_uncovered")

    def as_dict(self):
        return {k: int(getattr(self, k)) for k in self.FIELDS}


class ServerConfig(ctypes.Structure):
    _fields_ = [
        ("memory_bytes", ctypes.c_uint64),
        ("reserve_bytes", ctypes.c_uint64),
        ("max_graphs_per_tick", ctypes.c_uint64),
        ("max_bytes_per_tick", ctypes.c_uint64),
        ("in_place_max_nnz", ctypes.c_uint64),
        ("validate", ctypes.c_uint32),
        ("slots", ctypes.c_uint32),
        ("opts", Options),
        ("reserved", ctypes.c_uint64 * 4),
    ]


class ServerResult(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("in_place", ctypes.c_uint32),
        ("verdict", Verdict),
        ("submit_ns", ctypes.c_int64),
        ("done_ns", ctypes.c_int64),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("entries_read", ctypes.c_uint64),
        ("windows", ctypes.c_uint64),
        ("chunks", ctypes.c_uint64),
        ("attempts", ctypes.c_uint64),
        ("matches", ctypes.c_uint64),
        ("conflicts", ctypes.c_uint64),
        ("conflicted_entries", ctypes.c_uint64),
        ("max_conflicts", ctypes.c_uint64),
        ("hist", ctypes.c_uint64 * 10),
        ("transitions", ctypes.c_uint64 * 4),
        ("illegal_transitions", ctypes.c_uint64),
        ("id_loads", ctypes.c_uint64),
        ("id_loads_open", ctypes.c_uint64),
    ]

    def as_dict(self):
        d = {k: int(getattr(self, k)) for k, _ in self._fields_ if k not in ("hist", "transitions")}
        d["hist"] = [int(x) for x in self.hist]
        d["transitions"] = [int(x) for x in self.transitions]
        return d


# exported symbols, in header order: (name, restype, argtypes)
_P, _U32, _U64, _I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
SYMBOLS = [
    ("mm_version", ctypes.c_char_p, []),
    ("mm_last_error", ctypes.c_char_p, []),
    ("mm_default_options", _I, [ctypes.POINTER(Options)]),
    ("mm_create_csr", _I, [_U64, _U64, _P, _P, _U32, _P, ctypes.POINTER(_P)]),
    ("mm_create_coo", _I, [_U64, _U64, _P, _P, _U32, _P, ctypes.POINTER(_P)]),
    ("mm_host_device_address", _I, [_P, ctypes.POINTER(_P)]),
    ("mm_state_census", _I, [_P, ctypes.POINTER(_U64), _P]),
    ("mm_skipper", _I, [_P, ctypes.POINTER(Options), _P, _P, _U64, _P, _P]),
    ("mm_skipper_to_host", _I, [_P, ctypes.POINTER(Options), _P, _P, _U32, _P]),
    ("mm_skipper_batched", _I, [_P, _U64, _P, _P, ctypes.POINTER(Options), _P, _P, _P]),
    ("mm_validate", _I, [_P, _P, _P, _U64, ctypes.POINTER(Verdict), _P]),
    ("mm_validate_batched", _I, [_P, _U64, _P, _P, _P, ctypes.POINTER(Verdict), _P]),
    ("mm_sync", _I, [_P, _P]),
    ("mm_get_stats", _I, [_P, ctypes.POINTER(Stats), _P]),
    ("mm_get_timing", _I, [_P, ctypes.POINTER(Timing)]),
    ("mm_timing_history", _I, [_P, ctypes.POINTER(Timing), _U32, ctypes.POINTER(_U32)]),
    ("mm_autotune", _I, [_P, _P, ctypes.POINTER(Options), _P]),
    ("mm_autotune_batched", _I, [_P, _U64, _P, _P, _P, ctypes.POINTER(Options), _P]),
    ("mm_multi_create", _I, [ctypes.POINTER(_P)]),
    ("mm_skipper_multi", _I, [_P, _U64, ctypes.POINTER(GraphDesc), ctypes.POINTER(Options), _P]),
    ("mm_multi_sync", _I, [_P, _P]),
    ("mm_validate_multi", _I, [_P, _U64, ctypes.POINTER(GraphDesc), ctypes.POINTER(Verdict), _P]),
    ("mm_validate_multi_async", _I, [_P, _U64, ctypes.POINTER(GraphDesc), _P]),
    ("mm_multi_verdicts", _I, [_P, _U64, ctypes.POINTER(Verdict)]),
    ("mm_multi_destroy", _I, [_P]),
    ("mm_destroy", _I, [_P]),
    ("mm_skipper_static", _I, [_U64, _U64, _P, _P, _P, ctypes.POINTER(Options), _P]),
    ("mm_server_default_config", _I, [ctypes.POINTER(ServerConfig)]),
    ("mm_server_create", _I, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_P)]),
    ("mm_server_submit", _I, [_P, _U64, _U64, _P, _P, _P, ctypes.POINTER(_U64)]),
    ("mm_server_wait", _I, [_P, _U64, ctypes.c_double, ctypes.POINTER(ServerResult)]),
    ("mm_server_stats", _I, [_P, ctypes.POINTER(_U64), ctypes.POINTER(_U64), ctypes.POINTER(_U64)]),
    ("mm_server_destroy", _I, [_P]),
    ("mm_server_device_bytes", _I, [_U64, _U64, _U32, ctypes.POINTER(_U64)]),
    ("mm_server_plan_admission", _I, [ctypes.POINTER(_U64), _U64, _U64, _U64, _U64, ctypes.POINTER(_U64),
                                      ctypes.POINTER(_U64)]),
]

STATUS = {0: "MM_OK", 1: "MM_ERR_ARG", 2: "MM_ERR_OOM", 3: "MM_ERR_CUDA", 4: "MM_ERR_TIMEOUT",
          5: "MM_ERR_BAD_GRAPH", 6: "MM_ERR_UNSUPPORTED", 7: "MM_PENDING"}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libskipper.so (build it first with build()); raises ImportError if absent."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"libskipper.so not built at {p}: run __graft_entry__.build() "
                              f"or paper_2507_04420_gb300._native.build()")
        lib = ctypes.CDLL(p)
        for name, res, args in SYMBOLS:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib
