"""The benchmark's ncu traffic table is keyed to the kernel sources it was
captured from: every entry's source hash equals the current sources', so the
bench reports the captured DRAM traffic (a kernel edited since its capture
would report null instead)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_traffic_table_matches_current_sources():
    b = _bench()
    assert b.NCU_TRAFFIC
    for wl, entries in b.NCU_TRAFFIC.items():
        for key, (traffic, h) in entries.items():
            kernel = key.split("/")[-1]
            assert kernel in b.KERNEL_SOURCES, (wl, key)
            assert traffic > 0 or kernel == "batch_persistent", (wl, key)
            assert b.kernel_sources_hash(kernel) == h, f"{wl}/{key}: captured from other sources"
            assert b.ncu_traffic(wl, key) == traffic


def test_kernel_source_lists_exist():
    b = _bench()
    csrc = os.path.join(ROOT, "paper_2108_08380_gb300", "csrc")
    for kernel, files in b.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.exists(os.path.join(csrc, f)), (kernel, f)
