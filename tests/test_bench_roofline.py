"""Host logic of bench.py's roofline: the algorithmic byte counts per lattice
update, the lookup of ncu DRAM traffic (scaled by node count to a larger
lattice of the same family) and of FP64 instruction counts, both voided by a
change of the kernel source."""
import importlib.util
import json
import os
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _case(q, name, n):
    return SimpleNamespace(lattice=q, name=name, n=n)


def test_scope_byte_counts(bench):
    """Forward (2Q + 1) x 4 B, in FP64 2Q x 8 + 4 (the design field stays FP32);
    adjoint sweep 256 / 496 B, twice that in FP64."""
    for q, fwd, sweep in ((9, 76, 256), (19, 156, 496)):
        c = _case(q, "x", 1)
        assert bench.scope_bytes_per_lu(c, "forward step") == fwd == (2 * q + 1) * 4
        assert bench.scope_bytes_per_lu(c, "forward step", rs=8) == 2 * q * 8 + 4
        assert bench.scope_bytes_per_lu(c, "adjoint sweep step") == sweep
        assert bench.scope_bytes_per_lu(c, "adjoint sweep step", rs=8) == 2 * sweep


def test_traffic_lookup_scales_and_voids(bench, tmp_path, monkeypatch):
    f = tmp_path / "traffic.json"
    ent = {"kernel": "adj_step_kernel", "workload": "small", "nodes": 1000, "scales_to": ["big"],
           "bytes_per_launch": 2.0e5, "source_hash": "h1"}
    f.write_text(json.dumps({"entries": [ent]}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    monkeypatch.setattr(bench, "kernel_hash", lambda: "h1")
    assert bench.measured_traffic("adj_step_kernel", _case(19, "small", 1000)) == 2.0e5
    assert bench.measured_traffic("adj_step_kernel", _case(19, "big", 5000)) == pytest.approx(1.0e6)
    assert bench.measured_traffic("adj_step_kernel", _case(19, "other", 5000)) is None
    assert bench.unit_traffic("forward step", _case(19, "big", 5000)) is None   # no forward entries
    assert bench.measured_traffic("adj_step_kernel", _case(19, "big", 5000), "fp64") is None   # FP32 capture
    monkeypatch.setattr(bench, "kernel_hash", lambda: "h2")                        # kernel source changed
    assert bench.measured_traffic("adj_step_kernel", _case(19, "big", 5000)) is None


def test_fp64_instruction_lookup(bench, tmp_path, monkeypatch):
    f = tmp_path / "fp64_ops.json"
    ents = [{"kernel": "fwd_row_kernel", "lattice": "D2Q9", "inst_per_lu": 140.0, "source_hash": "h1"},
            {"kernel": "fwd_facerow_kernel", "lattice": "D2Q9", "inst_per_lu": 6.0, "source_hash": "h1"},
            {"kernel": "adj_step_kernel", "lattice": "D2Q9", "inst_per_lu": 260.0, "source_hash": "h1"}]
    f.write_text(json.dumps({"entries": ents}))
    monkeypatch.setattr(bench, "FP64_OPS_FILE", str(f))
    monkeypatch.setattr(bench, "kernel_hash", lambda: "h1")
    c = _case(9, "x", 10)
    assert bench.fp64_inst_per_lu("forward step", c) == 146.0      # the two forward kernels together
    assert bench.fp64_inst_per_lu("adjoint step", c) == 260.0
    assert bench.fp64_inst_per_lu("forward step", _case(19, "x", 10)) is None
    monkeypatch.setattr(bench, "kernel_hash", lambda: "h2")
    assert bench.fp64_inst_per_lu("adjoint step", c) is None


def test_committed_fp64_counts_cover_both_stencils(bench):
    """The committed counts name every step kernel for both stencils, and an
    FMA counts twice in flop_per_lu."""
    t = json.load(open(bench.FP64_OPS_FILE))
    seen = {(e["lattice"], e["kernel"]) for e in t["entries"]}
    for lat in ("D2Q9", "D3Q19"):
        for k in bench.FWD_KERNELS + bench.ADJ_KERNELS:
            assert (lat, k) in seen
    for e in t["entries"]:
        n = e["nodes"]
        assert e["inst_per_lu"] == pytest.approx((e["dadd"] + e["dmul"] + e["dfma"]) / n)
        assert e["flop_per_lu"] == pytest.approx((e["dadd"] + e["dmul"] + 2 * e["dfma"]) / n)


def test_clock_records_the_timing_rules_reject(bench):
    """Rejected: a hardware or thermal slowdown, or SM clocks far below their
    maximum with no reason (a leftover lock); kept: a power cap, full clocks,
    or no samples at all."""
    rej = bench.clocks_rejected
    assert rej({"sm_mhz": 2032.0, "sm_max_mhz": 2032.0, "reasons": ["hw_slowdown"]})
    assert rej({"sm_mhz": 1900.0, "sm_max_mhz": 2032.0, "reasons": ["sw_thermal_slowdown", "sw_power_cap"]})
    assert rej({"sm_mhz": 1200.0, "sm_max_mhz": 2032.0, "reasons": []})
    assert not rej({"sm_mhz": 1200.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"]})
    assert not rej({"sm_mhz": 1942.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"]})
    assert not rej({"sm_mhz": 2032.0, "sm_max_mhz": 2032.0, "reasons": []})
    assert not rej({"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0})
