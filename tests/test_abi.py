"""CPU-side checks of the C ABI: the library loads, exports every entry point
the header declares, rejects bad input on the host, and compiles gate streams
into passes as the batching rule says (no GPU needed)."""

import os
import re

import numpy as np
import pytest

from paper_2105_01533_gb300 import build as B
from paper_2105_01533_gb300 import sps
from paper_2105_01533_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return sps.load_library()


def header_functions():
    text = open(os.path.join(ROOT, "include", "sps.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(sps_[a-z_]+)\s*\(", text))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert "sps_create" in names and "sps_apply" in names and "sps_probability" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(sps.EXPORTS)


def test_status_strings(lib):
    for code in range(7):
        assert sps.sps_status_str(code)
    assert sps.sps_status_str(3) == "hash table probe limit reached"


def test_gate_record_layout():
    assert W.GATE_DTYPE.itemsize == 32
    text = open(os.path.join(ROOT, "include", "sps.h")).read()
    for name, code in [("SPS_OP_X", 1), ("SPS_OP_H", 10), ("SPS_OP_GIVENS", 13)]:
        assert re.search(r"%s = %d\b" % (name, code), text)
    assert W.OP_X == 1 and W.OP_H == 10 and W.OP_GIVENS == 13


def test_create_rejects_bad_arguments_on_host(lib):
    for nq, cap in [(0, 10), (128, 10), (10, 0)]:
        with pytest.raises(sps.SpsError) as e:
            sps.sps_create(nq, cap, None)
        assert e.value.status == sps.SPS_ERR_ARG


def test_create_without_gpu_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(sps.SpsError) as e:
        sps.sps_create(10, 16, None)
    assert e.value.status == sps.SPS_ERR_NO_DEVICE


def classify(op):
    return 2 if op in W.BRANCH_OPS else 1


def test_plan_splits_at_every_branching_gate(lib):
    gates = W.random_mix(3, 24, 400, keep_branch=W.CountingBound(4096), p_perm=0.5, p_diag=0.3)
    plan = sps.sps_plan(gates, 24)
    kinds = [classify(int(op)) for op in gates["op"]]
    # expected plan: runs of kind 1, cut where a run would pass 61 arbitrary-
    # phase slots (P takes 1, Rz 2); single passes of kind 2
    want = []
    slots = 0
    for i, k in enumerate(kinds):
        op = int(gates["op"][i])
        need = 1 if op == W.OP_P else (2 if op == W.OP_RZ else 0)
        if k == 2:
            want.append((2, i))
        elif not want or want[-1][0] == 2 or slots + need > 61:
            want.append((1, i))
            slots = need
        else:
            slots += need
    assert [(k, f) for k, f, _ in plan] == want
    # op count of a fused pass = number of gates in the run
    bounds = [f for _, f, _ in plan] + [len(gates)]
    for j, (k, f, nops) in enumerate(plan):
        assert nops == (bounds[j + 1] - f if k == 1 else 1)


def test_plan_respects_max_fused_ops(lib):
    lay = W.AdderLayout(32)
    add = W.cuccaro_adder(lay)
    plan = sps.sps_plan(add, lay.nqubits, max_fused_ops=50)
    assert [p[2] for p in plan] == [50, 50, 50, 43]
    assert [p[1] for p in plan] == [0, 50, 100, 150]
    plan = sps.sps_plan(add, lay.nqubits)
    assert plan == [(1, 0, len(add))]


def test_plan_rejects_bad_records(lib):
    good = W.to_array([W.H(0), W.X(3, 1)])
    cases = [
        W.to_array([W.H(0), W.X(5)]),                 # target out of range (n = 5)
        W.to_array([W.H(0), W.X(2, 2)]),              # control on the target
        W.to_array([W.H(0), W.Givens(1, 1, 0.3)]),    # p == q
        W.to_array([W.H(0), W.gate(99, 0)]),          # unknown code
        W.to_array([W.H(0), W.X(1, 70)]),             # control beyond n
    ]
    assert len(sps.sps_plan(good, 5)) == 2
    for c in cases:
        with pytest.raises(sps.SpsError) as e:
            sps.sps_plan(c, 5)
        assert e.value.status == sps.SPS_ERR_ARG and e.value.failed_gate == 1
    nan = W.to_array([W.Ry(0, float("nan"))])
    with pytest.raises(sps.SpsError):
        sps.sps_plan(nan, 2)


def test_plan_of_empty_stream(lib):
    assert sps.sps_plan(np.zeros(0, W.GATE_DTYPE), 10) == []


def test_runtime_compiler_builds_the_specialised_kernel(lib):
    """The bit-sliced pass specialised per run (SPS_OPT_BITSLICE_JIT) is
    generated and compiled for sm_103a on the host; no GPU is needed."""
    ok, msg = sps.sps_jit_selftest()
    assert ok, msg


def test_tune_cache_file_lookup(tmp_path):
    """The tuning cache is a text file, one line per size class; the last valid
    line of a class wins, lines of other classes and malformed or out-of-range
    lines are ignored (host only)."""
    p = tmp_path / "tune.txt"
    p.write_text(
        "sps-tune 1 kw=2 log2peak=24 load_factor_pct=50 bitslice_groups=8 fused_labels=0 "
        "max_fused_ops=512 ms=0.2500\n"
        "sps-tune 1 kw=1 log2peak=24 load_factor_pct=70 bitslice_groups=16 fused_labels=4 "
        "max_fused_ops=256 ms=1.0\n"
        "garbage line\n"
        "sps-tune 1 kw=2 log2peak=24 load_factor_pct=95 bitslice_groups=8 fused_labels=0 "
        "max_fused_ops=512 ms=0.1\n"          # load factor out of range: ignored
        "sps-tune 1 kw=2 log2peak=24 load_factor_pct=30 bitslice_groups=32 fused_labels=2 "
        "max_fused_ops=128 ms=0.2000\n")
    c = sps.sps_tune_cache_lookup(str(p), 2, 24)
    assert c["load_factor_pct"] == 30 and c["bitslice_groups"] == 32
    assert c["fused_labels"] == 2 and c["max_fused_ops"] == 128 and c["from_cache"] == 1
    assert abs(c["ms"] - 0.2) < 1e-6
    c1 = sps.sps_tune_cache_lookup(str(p), 1, 24)
    assert c1["load_factor_pct"] == 70 and c1["max_fused_ops"] == 256
    assert sps.sps_tune_cache_lookup(str(p), 2, 23) is None
    assert sps.sps_tune_cache_lookup(str(tmp_path / "missing.txt"), 2, 24) is None


def test_option_and_status_constants_match_the_header():
    """Every SPS_OPT_* and SPS_ERR_* value of the binding is the one the header
    declares (the enum's explicit initialisers)."""
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "sps.h")).read()
    declared = {m.group(1): int(m.group(2))
                for m in re.finditer(r"\b(SPS_(?:OPT|ERR)_[A-Z0-9_]+)\s*=\s*(\d+)", hdr)}
    assert len(declared) >= 20
    bound = {k: getattr(sps, k) for k in dir(sps) if re.match(r"SPS_(OPT|ERR)_", k)}
    for k, v in declared.items():
        assert k in bound, k
        assert bound[k] == v, (k, bound[k], v)
