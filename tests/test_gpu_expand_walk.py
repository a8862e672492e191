"""GPU parity of expansion passes that carry the phase/permutation run after
them (SPS_OPT_EXPAND_WALK): the expansion kernel walks the run's op stream on
its outputs before it stores them. Against the same apply with two passes the
result must be identical bit for bit (same labels, same amplitudes, same update
count); against the oracle it agrees to the usual tolerance (an expansion rounds
its table products differently from one pass per gate)."""

import numpy as np
import pytest

from oracle import OracleState
from paper_2105_01533_gb300 import sps
from paper_2105_01533_gb300 import workloads as W

from helpers import compare_states

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


def run(n, parts, eps, cap, walk, init=None):
    st = sps.SparseState(n, cap)
    st.set_option(sps.SPS_OPT_EXPAND_WALK, walk)
    # two passes: the second in the direct form, which the walk uses (the
    # bit-sliced form takes its phase products in another order)
    st.set_option(sps.SPS_OPT_BITSLICE_MIN_OPS, 0)
    if init is not None:
        st.set_amplitudes(*init)
    for gates in parts:
        st.apply(W.to_array(gates), eps)
    got = st.get_amplitudes()
    c = st.counters()
    upd = st.updates()
    st.close()
    return got, c, upd


def oracle(n, parts, eps, init=None):
    orc = OracleState(n)
    if init is not None:
        orc.set(*init)
    for gates in parts:
        orc.apply(W.to_array(gates), eps=eps)
    return orc.get()


def identical(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def phase_perm_run(rng, n, length):
    """X/CNOT/Toffoli, Z/S/T, controlled phases and Rz (arbitrary angles) on
    random qubits: a run that permutes labels and sets arbitrary phases."""
    recs = []
    for _ in range(length):
        q = rng.distinct(n, 3)
        k = rng.below(8)
        if k == 0:
            recs.append(W.X(q[0]))
        elif k == 1:
            recs.append(W.CX(q[0], q[1]))
        elif k == 2:
            recs.append(W.CCX(q[0], q[1], q[2]))
        elif k == 3:
            recs.append(W.Z(q[0]))
        elif k == 4:
            recs.append(W.S(q[0]))
        elif k == 5:
            recs.append(W.T(q[0]))
        elif k == 6:
            recs.append(W.P(q[0], rng.angle(), q[1]))
        else:
            recs.append(W.Rz(q[0], rng.angle()))
    return recs


# d: expanded qubits; 16, 17 and 18 from one entry give 2, 4 and 8 outputs per lane
@pytest.mark.parametrize("n,d,seed", [(30, 3, 1), (30, 9, 2), (64, 12, 3), (100, 16, 4),
                                      (127, 17, 5), (70, 18, 6)])
def test_walked_expansion_identical_to_two_passes(n, d, seed):
    rng = W.SplitMix64(seed)
    qs = rng.distinct(n, d)
    parts = [[W.X(q) for q in rng.distinct(n, 3)],
             [W.H(q) for q in qs] + phase_perm_run(rng, n, 150)]
    got, c, upd = run(n, parts, 1e-14, 1 << d, 1)
    two, c2, upd2 = run(n, parts, 1e-14, 1 << d, 0)
    identical(got, two)
    assert upd == upd2
    if (1 << d) > 2048:      # smaller states run the fused gates in a one-block run
        assert c.kernel_launches < c2.kernel_launches
    if d <= 16:
        compare_states(got, oracle(n, parts, 1e-14), 1e-14)


def test_walk_from_uploaded_entries_and_pruning():
    """Several input entries (expanded on qubits the masks show constant),
    Ry angles that give images below eps, an arbitrary-phase run after."""
    n = 90
    rng = np.random.default_rng(7)
    m = 300
    free = [0, 1, 2, 3, 4, 5, 6, 7, 8, 80]
    codes = rng.choice(1 << len(free), size=m, replace=False)
    labels = [(1 << 40) | sum(((int(c) >> b) & 1) << q for b, q in enumerate(free)) for c in codes]
    lo = np.array([v & (2**64 - 1) for v in labels], np.uint64)
    hi = np.array([v >> 64 for v in labels], np.uint64)
    init = (hi, lo, rng.normal(size=m), rng.normal(size=m))
    srng = W.SplitMix64(11)
    for eps in (0.0, 1e-14, 1e-7):
        parts = [[W.H(20), W.Ry(21, 1e-9), W.H(85), W.Ry(22, 3e-5), W.Rx(23, 0.4, 40)]
                 + phase_perm_run(srng, n, 60)]
        got, _, upd = run(n, parts, eps, 1 << 14, 1, init=init)
        two, _, upd2 = run(n, parts, eps, 1 << 14, 0, init=init)
        identical(got, two)
        assert upd == upd2
        compare_states(got, oracle(n, parts, eps, init=init), eps)


def test_walk_with_every_gate_folded_on_the_host():
    """A run whose gates all resolve on known qubits leaves no device ops: the
    expansion still counts their updates."""
    n = 40
    parts = [[W.H(q) for q in range(10)] + [W.X(30), W.CX(30, 31), W.Z(32)]]
    got, _, upd = run(n, parts, 0.0, 1 << 10, 1)
    two, _, upd2 = run(n, parts, 0.0, 1 << 10, 0)
    identical(got, two)
    assert upd == upd2 == (1 << 10) - 1 + 3 * (1 << 10)


def test_capacity_failure_in_walked_expansion():
    st = sps.SparseState(30, 1000)
    st.apply(W.to_array([W.H(q) for q in range(5)]), 0.0)          # 32 entries
    before = st.get_amplitudes()
    st.apply(W.to_array([W.X(20), W.H(10), W.H(11), W.H(12), W.H(13), W.H(14), W.CX(10, 3),
                         W.T(11)]), 0.0)                             # 32 * 32 > 1000
    with pytest.raises(sps.SpsError) as e:
        st.sync()
    assert e.value.status == sps.SPS_ERR_CAPACITY and e.value.failed_gate == 1
    hi, lo, re, im = st.get_amplitudes()
    np.testing.assert_array_equal(np.sort(before[1] ^ np.uint64(1 << 20)), lo)
    st.close()


def test_option_values():
    st = sps.SparseState(10, 64)
    for v in (-1, 2):
        with pytest.raises(sps.SpsError):
            st.set_option(sps.SPS_OPT_EXPAND_WALK, v)
    st.close()


@pytest.mark.parametrize("kw_bits", [60, 120])
def test_fused_labels_per_thread_identical(kw_bits):
    """Direct fused passes with 1, 2, 4 and 8 labels per thread: the same ops
    on every label, so the same state bit for bit; a ragged count (not a
    multiple of any slice) and the oracle beside them."""
    n = kw_bits
    rng = np.random.default_rng(kw_bits)
    m = 70_001
    codes = rng.choice(1 << 24, size=m, replace=False)
    free = list(range(0, n, max(1, n // 24)))[:24]
    labels = [sum(((int(c) >> b) & 1) << q for b, q in enumerate(free)) for c in codes]
    lo = np.array([v & (2**64 - 1) for v in labels], np.uint64)
    hi = np.array([v >> 64 for v in labels], np.uint64)
    init = (hi, lo, rng.normal(size=m), rng.normal(size=m))
    parts = [phase_perm_run(W.SplitMix64(kw_bits), n, 200)]
    want = oracle(n, parts, 1e-14, init=init)
    first = None
    for lanes in (1, 2, 4, 8, 0):
        st = sps.SparseState(n, 1 << 17)
        st.set_option(sps.SPS_OPT_FUSED_LABELS, lanes)
        st.set_option(sps.SPS_OPT_BITSLICE_MIN_OPS, 0)        # the direct form only
        st.set_amplitudes(*init)
        st.apply(W.to_array(parts[0]), 1e-14)
        got = st.get_amplitudes()
        st.close()
        if first is None:
            first = got
            compare_states(got, want, 1e-14)
        else:
            identical(got, first)
