"""Measurement probes (bd_probe): each kind runs, reports the operations it
performs, and bad geometry is refused before anything is launched."""
import pytest

pytestmark = pytest.mark.gpu


def test_probe_kinds_report_units(gpu_ctx):
    import torch
    import paper_2108_08380_gb300 as bd
    table = torch.zeros(1 << 16, dtype=torch.int32, device="cuda")
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    u = gpu_ctx.probe(bd.BD_PROBE_GATHER, 2, table, 1 << 11, sink=sink)
    # whole CTAs of 256 threads on every SM, 64 loads per lane per window
    assert u > 0 and u % (sms * 256 * 2 * 64) == 0
    torch.cuda.synchronize()
    assert int(sink.item()) == 0  # the table is all zeros
    table.fill_(1)
    sink.zero_()
    u = gpu_ctx.probe(bd.BD_PROBE_GATHER, 1, table, 1 << 16, sink=sink)
    torch.cuda.synchronize()
    assert int(sink.item()) == u  # every load read a one
    # L1 sector probe: every vector (1, 0, 0, 0) folds to 1; two 16-byte
    # vectors per 32-byte sector
    table.zero_()
    table[::4] = 1
    sink.zero_()
    u = gpu_ctx.probe(bd.BD_PROBE_L1_SECTORS, 3, table, sink=sink)
    torch.cuda.synchronize()
    assert u > 0 and u % (sms * 8 * 3 * 8 * 16) == 0
    assert int(sink.item()) == 2 * u
    for kind in (bd.BD_PROBE_POPC, bd.BD_PROBE_FFMA, bd.BD_PROBE_MUFU):
        u = gpu_ctx.probe(kind, 3)
        assert u > 0 and u % (sms * 256 * 3 * 64) == 0
    torch.cuda.synchronize()
    assert gpu_ctx.sync_status() == 0


def test_probe_rejects_bad_geometry(gpu_ctx):
    import torch
    import paper_2108_08380_gb300 as bd
    table = torch.zeros(1000, dtype=torch.int32, device="cuda")
    with pytest.raises(bd.BindescError):
        gpu_ctx.probe(bd.BD_PROBE_GATHER, 1, table, 512)      # table not a power of two
    t2 = torch.zeros(1 << 10, dtype=torch.int32, device="cuda")
    with pytest.raises(bd.BindescError):
        gpu_ctx.probe(bd.BD_PROBE_GATHER, 1, t2, 1 << 11)     # window larger than the table
    with pytest.raises(bd.BindescError):
        gpu_ctx.probe(bd.BD_PROBE_GATHER, 1, t2, 16)          # window under 32 words
    with pytest.raises(bd.BindescError):
        gpu_ctx.probe(bd.BD_PROBE_L1_SECTORS, 1, t2)          # table smaller than a window
    with pytest.raises(bd.BindescError):
        gpu_ctx.probe(bd.BD_PROBE_POPC, 0)                    # no repetitions
    with pytest.raises(bd.BindescError):
        gpu_ctx.probe(99, 1)                                  # unknown kind
