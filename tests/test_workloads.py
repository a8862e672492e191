"""CPU checks of the seeded generators (shapes, mixes, determinism)."""

import math

import numpy as np

from paper_2105_01533_gb300 import workloads as W


def test_splitmix_block_matches_stream():
    rng = W.SplitMix64(12345)
    want = [rng.next_u64() for _ in range(10)]
    got = W.splitmix_block(12345, 10)
    assert [int(x) for x in got] == want


def test_batched_fast_respects_caps_and_ranges():
    cs = W.batched_workload_fast(64, first_seed=7)
    for c in cs:
        g = c.gates
        assert 20 <= c.nqubits <= 100 and 256 <= c.cap <= 65536
        assert 200 + 8 <= len(g) <= 5000 + 8
        assert np.all(g["t0"] < c.nqubits)
        nh = int(np.sum(g["op"] == W.OP_H))
        assert 2 ** nh <= c.cap
        t = g["t0"].astype(np.int64)
        tlo = np.where(t < 64, np.left_shift(np.uint64(1), (t % 64).astype(np.uint64)), 0)
        thi = np.where(t >= 64, np.left_shift(np.uint64(1), (t % 64).astype(np.uint64)), 0)
        assert np.all((g["cmask"][:, 0] & tlo.astype(np.uint64)) == 0)
        assert np.all((g["cmask"][:, 1] & thi.astype(np.uint64)) == 0)
    again = W.batched_workload_fast(4, first_seed=7)
    for a, b in zip(cs[:4], again):
        assert a.cap == b.cap and np.array_equal(a.gates, b.gates)


def test_batched_fast_mix_proportions():
    g = W.random_mix_fast(3, 60, 200_000, h_budget=0)
    ops = g["op"][8:]
    perm = np.isin(ops, [W.OP_X]).mean()
    diag = np.isin(ops, [W.OP_Z, W.OP_S, W.OP_T, W.OP_RZ]).mean()
    assert abs(perm - (0.7 + 0.1 * 7 / 9)) < 0.01
    assert abs(diag - (0.2 + 0.1 * 2 / 9)) < 0.01
    assert np.sum(ops == W.OP_H) == 0


def test_adder_layout_and_gate_count():
    wl = W.adder_workload(seed=1, width=16)
    lay = wl.layout
    assert lay.nqubits == 67 and lay.cin == 64 and lay.cout == 65
    nx = bin(wl.b_const).count("1")
    assert len(wl.gates) == 16 + nx + 2 * (6 * 32 + 1) + 32


def test_givens_layers_are_matchings():
    g = W.givens_workload(seed=4, nqubits=16, modes=3, layers=5)
    body = g[3:]
    for layer in range(5):
        gv = body[layer * 16: layer * 16 + 8]
        assert np.all(gv["op"] == W.OP_GIVENS)
        qs = np.concatenate([gv["t0"], gv["t1"]])
        assert sorted(qs.tolist()) == list(range(16))
