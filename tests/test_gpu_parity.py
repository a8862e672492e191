"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs. Labels must match bit for bit (except labels within 10x eps
of the prune threshold on one side), amplitudes to 1e-12 max abs error.

Branching passes compute every product and sum exactly as the oracle does, so
for circuits of branching gates alone the GPU result is bit-identical; fused
phase passes reorder the phase products and stay within the tolerance."""

import math

import numpy as np
import pytest

from oracle import OracleState
from paper_2105_01533_gb300 import sps
from paper_2105_01533_gb300 import workloads as W

from helpers import compare_states, plain24_gates

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2105_01533_gb300 import build as B
    B.build()
    sps.load_library()
    yield


def run_both(n, gates, eps, capacity=1 << 16, chunks=1, options=()):
    st = sps.SparseState(n, capacity)
    for opt, val in options:
        st.set_option(opt, val)
    parts = np.array_split(gates, chunks) if chunks > 1 else [gates]
    for p in parts:
        st.apply(p, eps)
    got = st.get_amplitudes()
    st.close()
    orc = OracleState(n)
    orc.apply(gates, eps=eps)
    return got, orc.get()


@pytest.mark.parametrize("n", [20, 64, 100, 127])
@pytest.mark.parametrize("op", sorted(W.OP_NAMES))
def test_each_gate_type(n, op):
    rng = W.SplitMix64(1000 * n + op)
    prep = [W.H(q) for q in rng.distinct(n, 6)] + [W.X(q) for q in rng.distinct(n, 4)]
    prep += [W.Ry(rng.below(n), rng.angle()), W.T(rng.below(n))]
    gates = list(prep)
    for nctl in range(3):
        ntarg = 2 if op == W.OP_GIVENS else 1
        qs = rng.distinct(n, ntarg + nctl)
        if op == W.OP_GIVENS:
            gates.append(W.Givens(qs[0], qs[1], rng.angle(), *qs[2:]))
        else:
            gates.append(W.gate(op, qs[0], qs[1:], rng.angle()))
    gates = W.to_array(gates)
    got, want = run_both(n, gates, eps=1e-14)
    compare_states(got, want, 1e-14)


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("n,seed", [(12, 1), (40, 2), (63, 3), (64, 4), (90, 5), (127, 6)])
def test_random_circuits_all_gates(n, seed, form):
    gates = W.random_all_gates(seed, n, 400, max_controls=3, branch_frac=0.2,
                               keep_branch=W.CountingBound(1 << 16))
    got, want = run_both(n, gates, eps=1e-14, capacity=1 << 16,
                         options=[(sps.SPS_OPT_BRANCH_FORM, form)])
    compare_states(got, want, 1e-14)


@pytest.mark.parametrize("small_cap,form", [(2048, 0), (0, 1), (0, 2)])
def test_branching_only_is_bit_identical(small_cap, form):
    n = 30
    rng = W.SplitMix64(5)
    recs = []
    for _ in range(14):
        kind = rng.below(3)
        q = rng.distinct(n, 3)
        if kind == 0:
            recs.append(W.H(q[0]))
        elif kind == 1:
            recs.append(W.Ry(q[0], rng.angle(), q[1]))
        else:
            recs.append(W.Givens(q[0], q[1], rng.angle()))
    gates = W.to_array(recs)
    # one pass per gate (no expansion passes): every product and sum as the oracle's
    got, want = run_both(n, gates, eps=0.0, options=[(sps.SPS_OPT_SMALL_RUN_CAP, small_cap),
                                                     (sps.SPS_OPT_BRANCH_FORM, form),
                                                     (sps.SPS_OPT_EXPAND, 0)])
    for a, b in zip(got, want):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("form", [0, 1])
def test_plain24_workload_full(form):
    """24 qubits, H on 8 qubits then 2000 gates (70% X/CNOT/Toffoli, 20%
    Z/S/T/CRz, 10% H kept only while the oracle reports <= 4096 nonzeros)."""
    gates = plain24_gates(seed=0)
    assert len(gates) == 2008
    got, want = run_both(24, gates, eps=1e-14, capacity=8192,
                         options=[(sps.SPS_OPT_BRANCH_FORM, form), (sps.SPS_OPT_SMALL_RUN_CAP, 0)])
    stats = compare_states(got, want, 1e-14)
    assert stats["common"] >= 256
    # same stream applied in several calls gives the same result
    got2, _ = run_both(24, gates, eps=1e-14, capacity=8192, chunks=7)
    compare_states(got2, want, 1e-14)


def test_adder_workload_full_and_closed_form():
    wl = W.adder_workload(seed=1, width=16)
    got, want = run_both(wl.layout.nqubits, wl.gates, eps=1e-14, capacity=1 << 17)
    stats = compare_states(got, want, 1e-14)
    assert stats["common"] == 1 << 16
    hi, lo, re, im = got
    n = wl.layout.nbits
    a = lo & np.uint64(0xFFFFFFFF)
    assert np.all(hi == 0) and np.all((lo >> np.uint64(n)) == np.uint64(wl.b_const))
    bsum = (a + np.uint64(wl.b_const)) & np.uint64(0xFFFFFFFF)
    reg = a | (bsum << np.uint64(n))
    phase = np.zeros(len(a))
    for q1, q2, phi in wl.cp_pairs:
        both = ((reg >> np.uint64(q1)) & np.uint64(1)) & ((reg >> np.uint64(q2)) & np.uint64(1))
        phase += phi * both.astype(float)
    amp = 2.0 ** -8 * np.exp(1j * phase)
    assert np.max(np.abs(re + 1j * im - amp)) < 1e-12


@pytest.mark.parametrize("form", [0, 1])
def test_givens_workload_few_layers(form):
    gates = W.givens_workload(seed=2, nqubits=64, modes=4, layers=3)
    got, want = run_both(64, gates, eps=1e-14, capacity=700_000,
                         options=[(sps.SPS_OPT_BRANCH_FORM, form)])
    compare_states(got, want, 1e-14)


def test_givens_workload_full_properties():
    """All 500 layers: the oracle is too slow here, so check what holds at any
    size: Hamming weight 4, nnz <= C(64,4), unit norm, and that the inverse
    circuit (which also undoes the initial X gates) returns |0...0>."""
    gates = W.givens_workload(seed=2, nqubits=64, modes=4, layers=500)
    st = sps.SparseState(64, 700_000)
    st.apply(gates, 1e-14)
    hi, lo, re, im = st.get_amplitudes(sort=False)
    assert len(lo) <= math.comb(64, 4)
    w = np.zeros(len(lo), np.int64)
    x = lo.copy()
    while np.any(x):
        w += (x & np.uint64(1)).astype(np.int64)
        x >>= np.uint64(1)
    assert np.all(w == 4) and np.all(hi == 0)
    assert abs(np.sum(re * re + im * im) - 1.0) < 1e-10
    st.apply(W.inverse(gates), 1e-14)
    hi, lo, re, im = st.get_amplitudes()
    assert lo.tolist() == [0]
    assert abs(re[0] - 1.0) < 1e-9 and abs(im[0]) < 1e-9
    st.close()


def test_probability_matches_oracle():
    gates = W.random_all_gates(8, 70, 300, max_controls=2, branch_frac=0.2,
                               keep_branch=W.CountingBound(1 << 16))
    st = sps.SparseState(70, 1 << 16)
    st.apply(gates, 1e-14)
    orc = OracleState(70)
    orc.apply(gates, eps=1e-14)
    for mask, val in [((0, 0), (0, 0)), ((1, 0), (1, 0)), ((0xF0, 1 << 3), (0x30, 1 << 3)),
                      ((~0 & 0xFFFFFFFFFFFFFFFF, 0x3F), (0, 0))]:
        p_gpu = st.probability(mask, val)
        p_orc = orc.probability(mask, val)
        assert abs(p_gpu - p_orc) < 1e-12
    p1 = st.probability((1, 0), (1, 0))
    p2 = st.probability((1, 0), (1, 0))
    assert p1 == p2
    st.close()


# ---- edge cases -------------------------------------------------------------
def test_empty_gate_list_and_identity():
    st = sps.SparseState(10, 16)
    st.apply(np.zeros(0, W.GATE_DTYPE), 0.0)
    hi, lo, re, im = st.get_amplitudes()
    assert lo.tolist() == [0] and re.tolist() == [1.0] and im.tolist() == [0.0]
    st.close()


def test_everything_pruned_then_continue():
    st = sps.SparseState(10, 64)
    st.apply(W.to_array([W.H(0), W.H(1)]), 0.0)
    st.apply(W.to_array([W.H(2)]), 1.0)        # |a| = 0.35 < 1: all pruned
    assert st.nnz() == 0
    st.apply(W.to_array([W.X(3), W.H(4), W.Ry(5, 0.3)]), 0.0)
    assert st.nnz() == 0
    st.close()


def test_ragged_sizes_span_tiles():
    """nnz not a multiple of any block size, across several grid tiles."""
    n = 40
    for k in (9, 13, 17):
        qs = list(range(k))
        gates = W.to_array([W.H(q) for q in qs] + [W.Ry(k, 0.4, 0), W.X(k + 1, 1)] +
                           [W.Givens(k + 2, 0, 0.7)] + [W.CRz(3, k + 3, 1.1)])
        got, want = run_both(n, gates, eps=0.0, capacity=1 << 19)
        compare_states(got, want, 0.0)
        assert len(got[1]) > (1 << k)


def test_capacity_overflow_leaves_last_good_state():
    st = sps.SparseState(20, 100)
    st.apply(W.to_array([W.H(q) for q in range(6)]), 0.0)       # 64 entries
    before = st.get_amplitudes()
    st.apply(W.to_array([W.X(10), W.H(7), W.Z(3)]), 0.0)        # H would make 128
    with pytest.raises(sps.SpsError) as e:
        st.sync()
    assert e.value.status == sps.SPS_ERR_CAPACITY and e.value.failed_gate == 1
    hi, lo, re, im = st.get_amplitudes()
    # the X pass ran, the H pass failed, the Z pass was skipped
    np.testing.assert_array_equal(np.sort(before[1] ^ np.uint64(1 << 10)), lo)
    np.testing.assert_allclose(re, np.full(64, 0.125), rtol=0, atol=1e-15)
    # the state is usable again
    st.apply(W.to_array([W.H(0)]), 0.0)
    assert st.nnz() == 32
    st.close()


def test_probe_limit_reports_table_full_without_hanging():
    st = sps.SparseState(30, 1 << 12)
    st.set_option(sps.SPS_OPT_SMALL_RUN_CAP, 0)      # exercise the global table
    st.set_option(sps.SPS_OPT_BRANCH_FORM, 1)        # the scatter table has the probe limit
    st.set_option(sps.SPS_OPT_EXPAND, 0)             # one table pass per gate
    st.apply(W.to_array([W.H(q) for q in range(8)]), 0.0)
    st.sync()
    st.set_option(sps.SPS_OPT_PROBE_LIMIT, 1)
    st.set_option(sps.SPS_OPT_LOAD_FACTOR_PCT, 90)
    st.apply(W.to_array([W.H(q) for q in range(8, 12)]), 0.0)
    with pytest.raises(sps.SpsError) as e:
        st.sync()
    assert e.value.status == sps.SPS_ERR_TABLE_FULL
    assert st.nnz() == 256                       # unchanged
    st.set_option(sps.SPS_OPT_PROBE_LIMIT, 0)     # back to unbounded
    st.apply(W.to_array([W.H(q) for q in range(8, 12)]), 0.0)
    assert st.nnz() == 4096
    st.close()


def test_high_load_factor_collisions():
    n = 50
    gates = W.to_array([W.H(q) for q in range(12)] + [W.Ry(q, 0.3 * q) for q in range(12, 16)])
    for form in (1, 2):
        got, want = run_both(n, gates, eps=0.0, capacity=1 << 16,
                             options=[(sps.SPS_OPT_LOAD_FACTOR_PCT, 90),
                                      (sps.SPS_OPT_SMALL_RUN_CAP, 0),
                                      (sps.SPS_OPT_BRANCH_FORM, form),
                                      (sps.SPS_OPT_EXPAND, 0)])
        compare_states(got, want, 0.0)
    compare_states(got, want, 0.0)


def test_labels_with_all_ones_low_word():
    """128-bit labels whose low 64 bits are all set go through the CAS-only
    probe path; results must still match."""
    n = 70
    gates = W.to_array([W.X(q) for q in range(64)] + [W.H(q) for q in (0, 64, 65, 3)] +
                       [W.Givens(1, 66, 0.9), W.Ry(2, 1.3, 64)] + [W.H(q) for q in (0, 64)])
    got, want = run_both(n, gates, eps=1e-14)
    compare_states(got, want, 1e-14)
    assert np.any(got[1] == np.uint64(0xFFFFFFFFFFFFFFFF))


def test_bad_gate_rejected_before_enqueue():
    st = sps.SparseState(8, 16)
    with pytest.raises(sps.SpsError) as e:
        st.apply(W.to_array([W.H(0), W.X(9)]), 0.0)
    assert e.value.status == sps.SPS_ERR_ARG and e.value.failed_gate == 1
    hi, lo, re, im = st.get_amplitudes()
    assert lo.tolist() == [0]
    st.close()


def test_set_get_roundtrip_and_rejects_out_of_range():
    rng = np.random.default_rng(3)
    for n in (30, 100):
        st = sps.SparseState(n, 1000)
        m = 777
        lo = np.unique(rng.integers(0, 2 ** 30, m * 2, dtype=np.uint64))[:m]
        hi = rng.integers(0, 2 ** (n - 64), m, dtype=np.uint64) if n > 64 else np.zeros(m, np.uint64)
        re, im = rng.normal(size=m), rng.normal(size=m)
        st.set_amplitudes(hi, lo, re, im)
        g = st.get_amplitudes()
        order = np.lexsort((lo, hi))
        for a, b in zip(g, (hi[order], lo[order], re[order], im[order])):
            np.testing.assert_array_equal(a, b)
        bad_lo = lo.copy()
        bad_lo[5] = np.uint64(1) << np.uint64(min(n, 63))
        if n <= 63:
            with pytest.raises(sps.SpsError):
                st.set_amplitudes(hi, bad_lo, re, im)
            assert st.nnz() == 1
        st.close()


def test_options_give_identical_results():
    gates = plain24_gates(seed=3, ngates=600)
    base, want = run_both(24, gates, eps=1e-14, capacity=8192)
    compare_states(base, want, 1e-14)
    for opts in ([(sps.SPS_OPT_BLOCK_THREADS, 128)], [(sps.SPS_OPT_MAX_FUSED_OPS, 3)],
                 [(sps.SPS_OPT_LOAD_FACTOR_PCT, 25)], [(sps.SPS_OPT_SMALL_RUN_CAP, 0)],
                 [(sps.SPS_OPT_SMALL_RUN_CAP, 64)], [(sps.SPS_OPT_BITSLICE_MIN_OPS, 0)]):
        got, _ = run_both(24, gates, eps=1e-14, capacity=8192, options=opts)
        compare_states(got, want, 1e-14)


def test_counters_count_launches():
    gates = W.to_array([W.X(0), W.Z(1), W.H(2), W.CX(2, 3), W.H(4)])
    st = sps.SparseState(24, 4096)
    st.set_option(sps.SPS_OPT_SMALL_RUN_CAP, 0)
    st.set_option(sps.SPS_OPT_EXPAND, 0)
    st.sync()   # the gather form allocates nothing; the scatter table comes on first use
    c0 = st.counters().kernel_launches
    st.apply(gates, 0.0)
    c = st.counters()
    assert c.fused_passes == 2 and c.branch_passes == 2
    # a branching pass: the amplitude-only attempt (index, attempt) and its
    # gather kernels (build, emit) in one cooperative launch, which returns at
    # once if the attempt took the pass
    assert c.kernel_launches - c0 == 2 * 1 + 2 * 3
    st.close()
    st = sps.SparseState(24, 4096)        # the gather kernels as separate launches
    st.set_option(sps.SPS_OPT_SMALL_RUN_CAP, 0)
    st.set_option(sps.SPS_OPT_EXPAND, 0)
    st.set_option(sps.SPS_OPT_FALLBACK_CHAIN, 0)
    st.sync()
    c0 = st.counters().kernel_launches
    st.apply(gates, 0.0)
    assert st.counters().kernel_launches - c0 == 2 * 1 + 2 * 4
    st.close()
    st = sps.SparseState(24, 4096)
    st.set_option(sps.SPS_OPT_SMALL_RUN_CAP, 0)
    st.set_option(sps.SPS_OPT_EXPAND, 0)
    st.set_option(sps.SPS_OPT_AMP_ONLY, 0)
    st.sync()
    c0 = st.counters().kernel_launches
    st.apply(gates, 0.0)
    assert st.counters().kernel_launches - c0 == 2 * 1 + 2 * 2
    st.close()
    st = sps.SparseState(24, 4096)        # all five passes fit one small-state run
    st.set_option(sps.SPS_OPT_EXPAND, 0)
    c0 = st.counters().kernel_launches
    st.apply(gates, 0.0)
    c = st.counters()
    assert c.fused_passes == 2 and c.branch_passes == 2
    assert c.kernel_launches - c0 == 1
    st.close()
    # H(2) and H(4) flip qubits still 0 in every label: one expansion launch each
    st = sps.SparseState(24, 4096)
    c0 = st.counters().kernel_launches
    st.apply(gates, 0.0)
    c = st.counters()
    assert c.fused_passes == 2 and c.branch_passes == 2
    assert c.kernel_launches - c0 == 4
    st.close()


@pytest.mark.parametrize("small_cap", [0, 16, 2048])
def test_small_run_boundaries(small_cap):
    """Runs that end exactly at the cap, errors inside a run, and a run that
    starts from a state loaded with set_amplitudes."""
    n = 50
    gates = W.to_array([W.H(q) for q in range(12)] + [W.T(3), W.CX(1, 40)] +
                       [W.Givens(2, 41, 0.8), W.Ry(42, 1.1, 5)])
    got, want = run_both(n, gates, eps=1e-14, capacity=1 << 15,
                         options=[(sps.SPS_OPT_SMALL_RUN_CAP, small_cap)])
    compare_states(got, want, 1e-14)
    st = sps.SparseState(n, 300)
    st.set_option(sps.SPS_OPT_SMALL_RUN_CAP, small_cap)
    st.set_amplitudes(None, np.arange(100, dtype=np.uint64) * 2, np.full(100, 0.1), np.zeros(100))
    st.apply(W.to_array([W.H(0), W.X(9), W.H(20), W.Z(1)]), 0.0)   # 100 -> 200 -> 200 -> 400
    with pytest.raises(sps.SpsError) as e:
        st.sync()
    assert e.value.status == sps.SPS_ERR_CAPACITY and e.value.failed_gate == 2
    assert st.nnz() == 200
    st.close()


# ---- bit-sliced fused passes ------------------------------------------------------
def perm_diag_run(seed, n, ngates, max_controls=5, p_arbitrary=0.15):
    """A long phase/permutation run drawing X, Y, Z, S, Sdg, T, Tdg, P, Rz with
    0..max_controls controls."""
    rng = W.SplitMix64(seed)
    codes = [W.OP_X, W.OP_Y, W.OP_Z, W.OP_S, W.OP_SDG, W.OP_T, W.OP_TDG]
    recs = []
    for _ in range(ngates):
        if rng.uniform() < p_arbitrary:
            op = (W.OP_P, W.OP_RZ)[rng.below(2)]
        else:
            op = codes[rng.below(len(codes))]
        qs = rng.distinct(n, 1 + rng.below(max_controls + 1))
        recs.append(W.gate(op, qs[0], qs[1:], rng.angle()))
    return W.to_array(recs)


@pytest.mark.parametrize("n", [9, 24, 40, 64, 100, 127])
@pytest.mark.parametrize("min_ops,jit", [(1, 0), (0, 0), (1, 2)])
def test_bitslice_and_direct_long_runs(n, min_ops, jit):
    """Long phase/permutation runs in the direct form, the general bit-sliced
    kernel and the bit-sliced kernel compiled for the run (jit 2)."""
    rng = W.SplitMix64(n)
    k = min(n, 12)
    prep = W.to_array([W.H(q) for q in rng.distinct(n, k)] + [W.Ry(rng.below(n), 0.77)])
    gates = np.concatenate([prep, perm_diag_run(100 + n, n, 300)])
    got, want = run_both(n, gates, eps=1e-14, capacity=1 << 14,
                         options=[(sps.SPS_OPT_BITSLICE_MIN_OPS, min_ops),
                                  (sps.SPS_OPT_BITSLICE_MIN_NNZ, 0), (sps.SPS_OPT_SMALL_RUN_CAP, 0),
                                  (sps.SPS_OPT_BITSLICE_JIT, jit)])
    compare_states(got, want, 1e-14)


@pytest.mark.parametrize("jit", [0, 2])
def test_bitslice_many_phase_slots_and_split(jit):
    """More arbitrary phases than one pass holds: 70 Rz (140 fire slots) plus
    40 P; the compiler splits the run, each part uses two aux words and up to
    four phase tables."""
    n = 30
    rng = W.SplitMix64(77)
    prep = [W.H(q) for q in range(10)]
    run = [W.Rz(rng.below(n), rng.angle(), *([rng.below(10)] if rng.below(2) else []))
           for _ in range(70)]
    run += [W.CP(rng.below(10), 10 + rng.below(20), rng.angle()) for _ in range(40)]
    run = [g for g in run if g[5][0] & (1 << g[2]) == 0]   # control never on the target
    gates = W.to_array(prep + run + [W.X(q, (q + 1) % 10) for q in range(10)])
    plan = sps.sps_plan(gates, n)
    assert sum(1 for k, _, _ in plan if k == 1) >= 2
    got, want = run_both(n, gates, eps=1e-14, options=[(sps.SPS_OPT_BITSLICE_MIN_OPS, 1),
                                                       (sps.SPS_OPT_BITSLICE_MIN_NNZ, 0), (sps.SPS_OPT_SMALL_RUN_CAP, 0),
                                                       (sps.SPS_OPT_BITSLICE_JIT, jit)])
    compare_states(got, want, 1e-14)


@pytest.mark.parametrize("nnz_log2,groups,jit", [(5, 0, 0), (10, 0, 0), (15, 0, 0), (17, 0, 0),
                                                 (15, 2, 0), (17, 8, 0), (17, 32, 0), (5, 0, 2),
                                                 (12, 0, 2), (17, 0, 2)])
def test_bitslice_sizes(nnz_log2, groups, jit):
    """Tiles of 1..32 groups and a ragged tail: 2^k entries plus a few (the
    compiled form always takes tiles of 32 groups)."""
    n = 70
    prep = [W.H(q) for q in range(nnz_log2)] + [W.Ry(40, 0.3, 0)] + [W.H(41, 1)]
    gates = np.concatenate([W.to_array(prep), perm_diag_run(9, n, 200, max_controls=3)])
    got, want = run_both(n, gates, eps=1e-14, capacity=1 << 19,
                         options=[(sps.SPS_OPT_BITSLICE_MIN_OPS, 1),
                                  (sps.SPS_OPT_BITSLICE_MIN_NNZ, 0), (sps.SPS_OPT_SMALL_RUN_CAP, 0),
                                  (sps.SPS_OPT_BITSLICE_GROUPS, groups),
                                  (sps.SPS_OPT_BITSLICE_JIT, jit)])
    compare_states(got, want, 1e-14)
    assert len(got[1]) > (1 << nnz_log2)


def test_gather_epoch_wraps():
    """66,000 gather passes (H.H pairs) push the 16-bit table epoch through a
    wrap; the state must come back unchanged."""
    n = 20
    st = sps.SparseState(n, 1 << 12)
    st.set_option(sps.SPS_OPT_SMALL_RUN_CAP, 0)
    st.set_option(sps.SPS_OPT_BRANCH_FORM, 2)
    prep = W.to_array([W.H(q) for q in range(6)] + [W.Ry(7, 0.4), W.T(7)])
    st.apply(prep, 0.0)
    before = st.get_amplitudes()
    pair = W.to_array([W.H(9), W.H(9)])
    st.apply(np.tile(pair, 33_000), 1e-14)
    after = st.get_amplitudes()
    compare_states(after, before, 1e-14, atol=1e-11)
    st.close()


def test_probability_async_matches():
    import torch
    st = sps.SparseState(40, 1 << 12)
    out = torch.full((3,), float("nan"), dtype=torch.float64, pin_memory=True)
    st.apply(W.to_array([W.H(q) for q in range(6)] + [W.Ry(7, 0.3, 0), W.T(2)]), 1e-14)
    st.probability_async((0b101, 0), (0b001, 0), out.data_ptr())
    st.apply(W.to_array([W.H(0), W.CX(1, 9)]), 1e-14)
    st.probability_async((1 << 9, 0), (1 << 9, 0), out.data_ptr() + 8)
    dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    st.probability_async((0, 0), (0, 0), dev.data_ptr())          # into device memory
    st.sync()
    torch.cuda.synchronize()
    orc = OracleState(40)
    orc.apply(W.to_array([W.H(q) for q in range(6)] + [W.Ry(7, 0.3, 0), W.T(2)]), eps=1e-14)
    assert abs(out[0].item() - orc.probability((0b101, 0), (0b001, 0))) < 1e-12
    assert abs(out[1].item() - st.probability((1 << 9, 0), (1 << 9, 0))) < 1e-15
    assert abs(dev.item() - 1.0) < 1e-12
    st.close()


def test_repeated_applies_reuse_the_plan():
    """The same gate list applied again (same start, options, threshold) runs
    the cached plan and image; anything that differs compiles afresh. Results
    must not depend on which happened."""
    n = 50
    a = W.to_array([W.H(q) for q in range(5)] + [W.CX(0, 20), W.T(20), W.Ry(21, 0.4, 1)] +
                   [W.CCX(1, 2, 22), W.P(22, 0.9), W.H(3)])
    b = W.to_array([W.H(30), W.X(31, 30), W.Rz(31, 0.3), W.Givens(30, 32, 0.5)])
    orc_a = OracleState(n)
    orc_a.apply(a, eps=1e-14)
    want_a = orc_a.get()
    orc_ab = orc_a.clone()
    orc_ab.apply(b, eps=1e-14)
    want_ab = orc_ab.get()
    for small in (0, 2048):
        st = sps.SparseState(n, 1 << 12)
        st.set_option(sps.SPS_OPT_SMALL_RUN_CAP, small)
        for rep in range(3):
            st.reset()
            st.apply(a, 1e-14)
            compare_states(st.get_amplitudes(), want_a, 1e-14)
            st.apply(b, 1e-14)                 # another plan in between
            compare_states(st.get_amplitudes(), want_ab, 1e-14)
        st.reset()
        st.apply(a, 1e-3)                      # another threshold: compiled afresh
        orc = OracleState(n)
        orc.apply(a, eps=1e-3)
        compare_states(st.get_amplitudes(), orc.get(), 1e-3)
        st.close()


def test_cached_plan_reports_failures():
    """A capacity failure inside a reused plan names the same gate."""
    for small in (0, 2048):
        st = sps.SparseState(30, 40)
        st.set_option(sps.SPS_OPT_SMALL_RUN_CAP, small)
        st.set_option(sps.SPS_OPT_EXPAND, 0)
        g = W.to_array([W.H(q) for q in range(5)] + [W.X(9), W.H(10)])   # 32 -> 64 > 40
        for _ in range(2):
            st.reset()
            st.apply(g, 0.0)
            with pytest.raises(sps.SpsError) as e:
                st.sync()
            assert e.value.status == sps.SPS_ERR_CAPACITY and e.value.failed_gate == 6
            assert st.nnz() == 32
        st.close()


def test_commuting_queues_on_the_device():
    """SPS_OPT_COMMUTE: the rewritten stream runs on the device; the state equals
    the oracle's gate-by-gate result, with fewer branching passes, and a
    failure names the caller's gate."""
    n = 24
    rng = W.SplitMix64(9)
    recs = []
    for _ in range(300):
        q = rng.distinct(10, 2)          # at most 2^10 labels
        k = rng.below(6)
        recs.append([W.H(q[0]), W.X(q[0]), W.Ry(q[0], rng.angle()), W.CX(q[1], q[0]),
                     W.Z(q[0]), W.T(q[0])][k])
    gates = W.to_array(recs)
    orc = OracleState(n)
    orc.apply(gates, eps=1e-14)
    want = orc.get()
    passes = []
    for commute in (0, 1):
        st = sps.SparseState(n, 1 << 16)
        st.set_option(sps.SPS_OPT_COMMUTE, commute)
        st.apply(gates, 1e-14)
        compare_states(st.get_amplitudes(), want, 1e-14)
        passes.append(st.counters().branch_passes)
        st.close()
    assert passes[1] < passes[0]
    st = sps.SparseState(20, 40)
    st.set_option(sps.SPS_OPT_COMMUTE, 1)
    st.set_option(sps.SPS_OPT_EXPAND, 0)
    g = W.to_array([W.H(q) for q in range(5)] + [W.X(9), W.T(7), W.H(10), W.T(10)])
    # T(10) flushes H(10) early; the queued H(0..4) run at the end, H(4) makes 64 > 40
    st.apply(g, 0.0)
    with pytest.raises(sps.SpsError) as e:
        st.sync()
    assert e.value.status == sps.SPS_ERR_CAPACITY and e.value.failed_gate == 4
    st.close()


@pytest.mark.parametrize("coop", [2, 4, 8])
@pytest.mark.parametrize("n,load", [(30, 50), (70, 90)])
def test_scatter_cooperative_probing(coop, n, load):
    """Scatter form with W lanes probing one insert together: bit-identical
    to single-lane probing (each slot receives at most two contributions, and
    0 + x and x + y are exact in either order) at a normal and a high table
    load (long probe runs), and equal to the oracle."""
    rng = W.SplitMix64(40 + n)
    recs = [W.H(q) for q in range(9)]
    branching = 0
    for _ in range(40):
        kind = rng.below(4) if branching < 5 else 3   # at most 2^14 nonzeros
        branching += kind < 3
        q = rng.distinct(n, 3)
        if kind == 0:
            recs.append(W.H(q[0]))
        elif kind == 1:
            recs.append(W.Ry(q[0], rng.angle(), q[1]))
        elif kind == 2:
            recs.append(W.Givens(q[0], q[1], rng.angle()))
        else:
            recs.append(W.CX(q[0], q[1]))
    gates = W.to_array(recs)
    base = [(sps.SPS_OPT_BRANCH_FORM, 1), (sps.SPS_OPT_SMALL_RUN_CAP, 0),
            (sps.SPS_OPT_EXPAND, 0), (sps.SPS_OPT_LOAD_FACTOR_PCT, load)]
    one, want = run_both(n, gates, eps=1e-14, capacity=1 << 15, options=base)
    got, _ = run_both(n, gates, eps=1e-14, capacity=1 << 15,
                      options=base + [(sps.SPS_OPT_COOP_WIDTH, coop)])
    for a, b in zip(got, one):
        np.testing.assert_array_equal(a, b)
    compare_states(got, want, 1e-14)


def test_scatter_cooperative_probe_limit():
    """With a probe limit of one slot and 8 lanes per insert, only the first
    slot is probed: 4,096 labels hashed into 8,192 slots collide, so the pass
    fails with SPS_ERR_TABLE_FULL as the single-lane form does."""
    gates = W.to_array([W.H(q) for q in range(12)])
    for coop in (1, 8):
        st = sps.SparseState(20, 1 << 13)
        for o, v in [(sps.SPS_OPT_BRANCH_FORM, 1), (sps.SPS_OPT_SMALL_RUN_CAP, 0),
                     (sps.SPS_OPT_EXPAND, 0), (sps.SPS_OPT_LOAD_FACTOR_PCT, 90),
                     (sps.SPS_OPT_PROBE_LIMIT, 1), (sps.SPS_OPT_COOP_WIDTH, coop)]:
            st.set_option(o, v)
        st.apply(gates, 0.0)
        with pytest.raises(sps.SpsError) as e:
            st.sync()
        assert e.value.status == sps.SPS_ERR_TABLE_FULL
        st.close()


@pytest.mark.parametrize("n_entries", [1, 255, 256, 257, 4095, 70001, 200001])
@pytest.mark.parametrize("nq", [40, 90])
def test_probability_ragged_sizes(n_entries, nq):
    """The readout over states whose size is not a multiple of a warp's 256
    entries (full spans and the ragged tail), 64- and 128-bit labels: equal to
    the sum of |a|^2 over the matching labels of the state itself."""
    rng = np.random.default_rng(n_entries + nq)
    lo = rng.choice(1 << 38, size=n_entries, replace=False).astype(np.uint64)
    hi = (rng.integers(0, 1 << 20, size=n_entries).astype(np.uint64) if nq > 64
          else np.zeros(n_entries, np.uint64))
    re = rng.normal(size=n_entries)
    im = rng.normal(size=n_entries)
    st = sps.SparseState(nq, max(n_entries, 16))
    st.set_amplitudes(hi if nq > 64 else None, lo, re, im)
    mag = re * re + im * im
    for mask, val in [((0, 0), (0, 0)), ((0b1011, 0), (0b0010, 0)),
                      ((1 << 37, 1 if nq > 64 else 0), (0, 1 if nq > 64 else 0))]:
        sel = ((lo & np.uint64(mask[0])) == np.uint64(val[0])) & \
              ((hi & np.uint64(mask[1])) == np.uint64(val[1]))
        want = float(np.sum(mag[sel]))
        got = st.probability(mask, val)
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (mask, got, want)
    st.close()
