"""The ncu counters bench.py turns into roofline figures (profiles/counters.json)
belong to the code as it stands: every entry names an existing summary and
existing sources, and its code digest equals the digest of those sources now
(a kernel edited after its capture would make the bench report the roofline
as stale)."""
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_for_tests", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def entries():
    with open(os.path.join(ROOT, "profiles", "counters.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("kernel", sorted(entries()))
def test_counters_match_the_current_sources(kernel):
    bench = load_bench()
    e = entries()[kernel]
    assert os.path.exists(os.path.join(ROOT, e["summary"])), e["summary"]
    for src in e["sources"]:
        assert os.path.exists(os.path.join(ROOT, src)), src
    assert bench.source_digest(e["sources"]) == e["code_sha256"], f"{kernel}: re-capture its counters"
    assert e["warp_inst_per_unit"] > 0 and e["dram_bytes_per_unit"] > 0


def test_the_bench_reads_every_kernel_it_reports():
    bench = load_bench()
    for kernel, workload in (("build_warp_kernel", "large-200x200x120-N5000-A32"),
                             ("bellman_kernel_fused3", "large-200x200x120-N5000-A32"),
                             ("build3d_warp_kernel", "cube-64x64x16x40-N1000-A24")):
        assert bench.kernel_counters(kernel, workload) is not None, kernel
