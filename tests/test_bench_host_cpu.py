"""Host logic of bench.py that decides what its JSON line reports (CPU only):
the ncu traffic figure is taken from a committed profile summary only while
that summary was made on the current kernel sources, and the roofline peak
comes from the measured-peaks file when there is one."""
import json
import os

import pytest

import bench


def _tree(tmp_path, sources):
    csrc = tmp_path / "paper_2507_04420_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name, text in sources.items():
        (csrc / name).write_text(text)
    (tmp_path / "profiles").mkdir()
    return tmp_path


def test_traffic_only_while_the_source_hash_matches(tmp_path, monkeypatch):
    root = _tree(tmp_path, {"state.cuh": "a", "walk.cuh": "b", "sweep.cu": "c"})
    monkeypatch.setattr(bench, "ROOT", str(root))
    h = bench.kernel_source_hash()
    assert len(h) == 16
    prof = root / "profiles" / "sweep_u8_rmat9_ef4.md"
    prof.write_text(f"# summary\nkernel_source_sha256_16: {h}\ndram_bytes_per_launch: 1.234e9\n")
    assert bench.ncu_traffic("rmat9_ef4", 8) == pytest.approx(1.234e9)
    assert bench.ncu_traffic("rmat9_ef4", 2) is None            # no summary for that layout
    (root / "paper_2507_04420_gb300" / "csrc" / "walk.cuh").write_text("b changed")
    assert bench.kernel_source_hash() != h
    assert bench.ncu_traffic("rmat9_ef4", 8) is None            # the kernel changed since
    prof.write_text(f"kernel_source_sha256_16: {bench.kernel_source_hash()}\n")
    assert bench.ncu_traffic("rmat9_ef4", 8) is None            # no figure in the summary


def test_edge_list_traffic_uses_its_own_sources(tmp_path, monkeypatch):
    root = _tree(tmp_path, {"state.cuh": "a", "walk.cuh": "b", "sweep.cu": "c", "coo.cu": "d"})
    monkeypatch.setattr(bench, "ROOT", str(root))
    h = bench.kernel_source_hash(bench.COO_SOURCES)
    (root / "profiles" / "coo_sweep_u2_rmat9_raw.md").write_text(
        f"kernel_source_sha256_16: {h}\ndram_bytes_per_launch: 5e8\n")
    assert bench.ncu_traffic("rmat9_raw", 2, "coo_sweep", bench.COO_SOURCES) == pytest.approx(5e8)
    (root / "paper_2507_04420_gb300" / "csrc" / "sweep.cu").write_text("c changed")   # not a COO source
    assert bench.ncu_traffic("rmat9_raw", 2, "coo_sweep", bench.COO_SOURCES) == pytest.approx(5e8)
    (root / "paper_2507_04420_gb300" / "csrc" / "coo.cu").write_text("d changed")
    assert bench.ncu_traffic("rmat9_raw", 2, "coo_sweep", bench.COO_SOURCES) is None


def test_peak_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6769.4, "bf16_tflops": 1900}))
    assert bench.measured_peaks() == (6769.4, "measured")


def test_committed_profiles_parse():
    """Every committed summary bench.py reads names a source hash and a figure."""
    read = [n for n in os.listdir(os.path.join(bench.ROOT, "profiles"))
            if (n.startswith("sweep_u") and n.endswith("_ef16.md"))
            or (n.startswith("coo_sweep_u") and n.endswith("_raw.md"))]
    assert len(read) >= 3
    for name in read:
        text = open(os.path.join(bench.ROOT, "profiles", name)).read()
        assert "kernel_source_sha256_16:" in text and "dram_bytes_per_launch:" in text, name


def test_every_global_name_bench_uses_is_defined():
    """bench.py runs its GPU legs only on a GPU machine; a name it calls but no
    longer defines would surface there first, so check the module here."""
    import ast
    import builtins
    src = open(bench.__file__).read()
    tree = ast.parse(src)
    defined = set(dir(builtins)) | set(vars(bench))
    used = set()
    local = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Name):
            (used if isinstance(node.ctx, ast.Load) else local).add(node.id)
        elif isinstance(node, (ast.FunctionDef, ast.arg)):
            local.add(node.name if isinstance(node, ast.FunctionDef) else node.arg)
        elif isinstance(node, (ast.Import, ast.ImportFrom)):
            local.update((a.asname or a.name).split(".")[0] for a in node.names)
        elif isinstance(node, ast.ExceptHandler) and node.name:
            local.add(node.name)
    missing = sorted(used - defined - local)
    assert not missing, missing


def test_batch_profile_name_matches_the_committed_summary():
    class O:   # the batched autotuner's usual pick on the 4096-graph batch
        grain, blocks_per_sm, unit_order, warps_per_graph = 8192, 4, 2, 0
    name = bench.batch_profile_name(4096, O())
    assert name == "c4batch4096_g8192_b4_dispersed_w0"
    path = os.path.join(bench.ROOT, "profiles", f"sweep_u8_{name}.md")
    text = open(path).read()
    assert "kernel_source_sha256_16:" in text and "dram_bytes_per_launch:" in text
    O.unit_order = 0
    assert bench.batch_profile_name(4096, O()).endswith("_auto_w0")
