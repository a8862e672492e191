"""Host logic of bench.py that shapes the reported numbers (no GPU): the
algorithmic bytes credited per launch, the roofline object built from profile
records, and the DRAM traffic taken from the committed ncu record, which must
be ignored once the kernel sources no longer match the capture."""

import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def rec(kind, n_in, n_out, flags=3, lb=16, ms=1.0, nops=1):
    return {"kind": kind, "n_in": n_in, "n_out": n_out, "flags": flags, "label_bytes": lb, "ms": ms,
            "nops": nops, "pass": 1}


def test_algorithmic_bytes_per_kind(bench):
    """Bytes of the method's passes: 2*B*n per fused pass, B*(n_in + n_out)
    per branching pass (B = label bytes + 16), each pass a launch carries out
    counted."""
    B = 32
    # a fused pass reads and writes the state, whatever it changes
    for flags in (3, 2, 1):
        assert bench.algorithmic_bytes(rec(1, 100, 100, flags=flags)) == 2 * B * 100
    assert bench.algorithmic_bytes(rec(1, 100, 100, flags=1, lb=8)) == 2 * 24 * 100
    # one branching gate as a gather pass: old state in, new state out
    assert bench.algorithmic_bytes(rec(6, 10, 20)) == B * (10 + 20)
    # an expansion of d gates doubles d times: sum of B*(m + 2m) for m = n, 2n, ..
    assert bench.algorithmic_bytes(rec(7, 1, 8, nops=3)) == B * (3 + 6 + 12)
    assert bench.algorithmic_bytes(rec(7, 1, 8, nops=3, flags=7)) == B * (3 + 6 + 12) + 2 * B * 8
    # an amplitude-only run of d gates: d passes over a state that keeps its labels
    assert bench.algorithmic_bytes(rec(10, 50, 50, nops=4, flags=2)) == 4 * 2 * B * 50
    assert bench.algorithmic_bytes(rec(10, 50, 50, nops=4, flags=6)) == 5 * 2 * B * 50
    assert bench.algorithmic_bytes(rec(10, 50, 0, nops=4, flags=2)) == 0     # not taken
    # a layer of 2 gates from 10 to 40 entries: 10 -> 20 -> 40
    assert abs(bench.algorithmic_bytes(rec(6, 10, 40, nops=2)) - B * (30 + 60)) < 1e-6
    # index builds read labels only
    for k in (5, 9):
        assert bench.algorithmic_bytes(rec(k, 10, 0, lb=8)) == 8 * 10


def test_moved_bytes_and_kernel_names(bench):
    assert bench.moved_bytes(rec(1, 100, 100, flags=2)) == (16 + 32) * 100
    assert bench.moved_bytes(rec(10, 50, 50, nops=4)) == (32 + 16) * 50
    assert bench.kernel_name(rec(1, 1, 1, flags=3 | 8 | 16)) == "k_bs_jit"
    assert bench.kernel_name(rec(1, 1, 1, flags=3 | 8)) == "k_fused_bs"
    assert bench.kernel_name(rec(1, 1, 1, flags=3)) == "k_fused"
    assert bench.kernel_name(rec(10, 1, 1)) == "k_amp_layer"


def test_traffic_record_is_used_only_for_matching_sources(bench, tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.json").write_text(json.dumps(
        {"k_amp_layer": {"givens64": {"source_hash": h, "dram_bytes_per_entry": 2.0}},
         "k_fused": {"adder67-w24": {"source_hash": "0" * 16, "dram_bytes_per_entry": 9.0}}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the hash is of the kernel sources under ROOT: point it back at the repository's
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.ncu_traffic("k_amp_layer", "givens64", 1000) == 2000.0
    assert bench.ncu_traffic("k_fused", "adder67-w24", 1000) is None      # stale capture
    assert bench.ncu_traffic("k_expand", "adder67", 1000) is None         # none recorded


def test_roofline_picks_the_dominant_kernel_and_scales_traffic(bench, monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: (6000.0, "measured"))
    monkeypatch.setattr(bench, "ncu_traffic",
                        lambda k, w, n: 3.0 * n if (k, w) == ("k_expand", "adder67") else None)
    recs = [rec(7, 1, 65536, ms=0.02, nops=16), rec(7, 1, 65536, ms=0.022, nops=16),
            rec(8, 65536, 65536, ms=0.001)]
    r = bench.roofline(recs, "adder67", steps=2)
    assert r["kernel"] == "k_expand"
    assert r["launches_per_step"] == 1.0
    # the roofline: what each launch moves (one entry read, 65,536 written)
    want = 32 * (1 + 65536) / (0.021e-3) / 1e9
    assert abs(r["achieved"] - round(want, 2)) < 0.01
    assert abs(r["frac"] - round(want / 6000.0, 4)) < 1e-4
    # the work rate: 16 doubling passes from one entry
    work = 32 * 3 * (2 ** 16 - 1) / (0.021e-3) / 1e9
    assert abs(r["method_passes"]["rate"] - round(work, 2)) < 0.01
    assert r["traffic"] == 3.0 * 65536      # expansions count their outputs
    assert set(r["time_share"]) == {"k_expand", "k_measure"}


def test_chain_launch_is_credited_only_when_it_ran(bench):
    """An attempted run's passes in one launch (kind 11): nothing when the
    attempt took the run (n_in 0), else each of its d passes reads and writes
    the state once."""
    assert bench.algorithmic_bytes(rec(11, 0, 50, nops=8)) == 0.0
    assert bench.moved_bytes(rec(11, 0, 50, nops=8)) == 0.0
    assert bench.algorithmic_bytes(rec(11, 40, 50, nops=8)) == 32 * (40 + 50) * 8
    assert bench.kernel_name(rec(11, 40, 50)) == "k_chain"


def test_readout_records(bench):
    """The probability readout (kind 12) reads the labels of every entry."""
    assert bench.algorithmic_bytes(rec(12, 1000, 1000, lb=16)) == 16 * 1000
    assert bench.moved_bytes(rec(12, 1000, 1000, lb=8)) == 8 * 1000
    assert bench.kernel_name(rec(12, 10, 10)) == "k_probability"
