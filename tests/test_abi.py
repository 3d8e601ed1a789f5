"""The C ABI library loads, exports every declared symbol, and its structs have
the header's layout (CPU only; no compute call is made)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "skipper.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def native():
    import __graft_entry__
    mod = __graft_entry__._native_module()
    mod.build()
    return mod


def test_library_exports_every_declared_symbol(native):
    lib = ctypes.CDLL(native.LIB_PATH)
    names = _declared()
    assert {"mm_create_csr", "mm_skipper", "mm_skipper_batched", "mm_validate",
            "mm_destroy"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", native.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (mm_\w+)", out))
    assert set(names) <= exported
    # the binding declares the same set
    assert {s[0] for s in native.SYMBOLS} == set(names)


def test_struct_layout_matches_header(native):
    """sizeof / offsetof from a C compile of the header against the ctypes mirrors."""
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "skipper.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(mm_options), offsetof(mm_options, spin_limit),
         offsetof(mm_options, poison_vertex), sizeof(mm_verdict),
         offsetof(mm_verdict, first_uncovered), sizeof(mm_timing), offsetof(mm_timing, units));
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", offsetof(mm_options, symmetric), sizeof(mm_server_config),
         offsetof(mm_server_config, opts), offsetof(mm_server_config, reserved),
         sizeof(mm_server_result), offsetof(mm_server_result, verdict),
         offsetof(mm_server_result, done_ns), sizeof(mm_graph_desc));
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(mm_stats), offsetof(mm_stats, transitions),
         offsetof(mm_stats, illegal_transitions), offsetof(mm_stats, id_loads_open),
         offsetof(mm_options, id_loads), (size_t)MM_ID_LOADS_SELECTIVE);
  printf("%zu %zu %zu %u %zu %u\n", offsetof(mm_options, stage_windows), offsetof(mm_options, reserved),
         offsetof(mm_options, warps_per_graph), MM_BATCH_LOCAL_IDS, offsetof(mm_options, unit_order),
         MM_ORDER_DISPERSED);
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        vals = [int(x) for x in subprocess.check_output([exe]).split()]
    O, V, T = native.Options, native.Verdict, native.Timing
    C, R, G = native.ServerConfig, native.ServerResult, native.GraphDesc
    assert vals == [ctypes.sizeof(O), O.spin_limit.offset, O.poison_vertex.offset,
                    ctypes.sizeof(V), V.first_uncovered.offset, ctypes.sizeof(T), T.units.offset,
                    O.symmetric.offset, ctypes.sizeof(C), C.opts.offset, C.reserved.offset,
                    ctypes.sizeof(R), R.verdict.offset, R.done_ns.offset, ctypes.sizeof(G),
                    ctypes.sizeof(native.Stats), native.Stats.transitions.offset,
                    native.Stats.illegal_transitions.offset, native.Stats.id_loads_open.offset,
                    O.id_loads.offset, 2, O.stage_windows.offset, O.reserved.offset,
                    O.warps_per_graph.offset, 4, O.unit_order.offset, 2]


def test_default_options_and_argument_errors(native):
    lib = native.load(native.LIB_PATH)
    o = native.Options()
    assert lib.mm_default_options(ctypes.byref(o)) == 0
    assert (o.status_bits, o.grain, o.block_threads, o.spin_limit) == (8, 0, 512, 1 << 20)   # grain 0: by size
    assert lib.mm_default_options(None) == 1
    assert b"null" in lib.mm_last_error()
    # argument checks happen before any device work
    assert lib.mm_create_csr(4, 4, ctypes.c_void_p(64), ctypes.c_void_p(64), 0, None, None) == 1
    h = ctypes.c_void_p()
    assert lib.mm_create_csr(4, 4, None, ctypes.c_void_p(64), 0, None, ctypes.byref(h)) == 1
    assert lib.mm_create_csr(4, 4, ctypes.c_void_p(64), ctypes.c_void_p(68), 0, None,
                             ctypes.byref(h)) == 1   # nbrs not 16-byte aligned
    assert b"aligned" in lib.mm_last_error()
    assert lib.mm_create_csr(1 << 33, 0, ctypes.c_void_p(64), None, 0, None, ctypes.byref(h)) == 1
    # a local-id batch takes no device check and no host mapping, and its n has a ceiling too
    assert lib.mm_create_csr(4, 4, ctypes.c_void_p(64), ctypes.c_void_p(64), 4 | 1, None, ctypes.byref(h)) == 6
    assert lib.mm_create_csr(4, 4, ctypes.c_void_p(64), ctypes.c_void_p(64), 4 | 2, None, ctypes.byref(h)) == 6
    assert lib.mm_create_csr((1 << 40) + 1, 0, ctypes.c_void_p(64), None, 4, None, ctypes.byref(h)) == 1
    assert lib.mm_skipper(None, None, None, None, 0, None, None) == 1
    assert lib.mm_destroy(None) == 0
    assert lib.mm_version().startswith(b"skipper-gb300")


def test_package_refuses_host_tensors(native):
    import torch
    import paper_2507_04420_gb300 as skp
    with pytest.raises(ValueError):
        skp.Graph(torch.zeros(3, dtype=torch.int64), torch.zeros(4, dtype=torch.int32))
    with pytest.raises(TypeError):
        skp.options(no_such_field=1)


def test_missing_library_fails_loudly(native, tmp_path):
    with pytest.raises(ImportError):
        native.load(str(tmp_path / "libskipper.so"))
