"""GPU parity of expansion passes (SPS_OPT_EXPAND): runs of branching gates
that act on every entry and flip only qubits known to be constant are applied
as one pass whose amplitudes are a times a product of matrix entries from
per-8-gate tables. Compared with the oracle (one pass per gate) to the usual
tolerance, and with the library's own one-pass-per-gate form."""

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


def run(n, parts, eps, cap, expand=1, form=0, small_cap=2048, init=None):
    st = sps.SparseState(n, cap)
    st.set_option(sps.SPS_OPT_EXPAND, expand)
    st.set_option(sps.SPS_OPT_BRANCH_FORM, form)
    st.set_option(sps.SPS_OPT_SMALL_RUN_CAP, small_cap)
    if init is not None:
        st.set_amplitudes(*init)
    for gates in parts:
        st.apply(W.to_array(gates), eps)
    got = st.get_amplitudes()
    c = st.counters()
    st.close()
    return got, c


def oracle(n, parts, eps, init=None):
    orc = OracleState(n)
    if init is not None:
        orc.set(*init)
    for gates in parts:
        orc.apply(W.to_array(gates), eps=eps)
    return orc.get()


@pytest.mark.parametrize("n", [30, 100])
@pytest.mark.parametrize("k", [1, 7, 8, 9, 16, 17])
def test_hadamard_layers(n, k):
    qs = [(7 * i + 3) % n for i in range(k)]
    parts = [[W.H(q) for q in qs]]
    got, c = run(n, parts, 1e-14, 1 << k)
    compare_states(got, oracle(n, parts, 1e-14), 1e-14)
    assert c.branch_passes == 1 and len(got[1]) == 1 << k


@pytest.mark.parametrize("k", [24, 25])
def test_widest_expansions_closed_form(k):
    """24 gates fill one pass (three 8-gate tables); 25 take two passes. The
    result is every label over the k qubits with amplitude 2^(-k/2)."""
    n = 30
    qs = list(range(3, 3 + k))
    got, c = run(n, [[W.H(q) for q in qs]], 0.0, 1 << k)
    assert c.branch_passes == (k + 23) // 24
    hi, lo, re, im = got
    want = np.arange(1 << k, dtype=np.uint64) << np.uint64(3)
    np.testing.assert_array_equal(lo, want)      # sorted by label
    np.testing.assert_allclose(re, np.full(1 << k, 2.0 ** (-k / 2)), rtol=1e-13, atol=0)
    assert not im.any() and not hi.any()


@pytest.mark.parametrize("n", [40, 90])
def test_mixed_gates_and_eligibility(n):
    """Eligible: H/Rx/Ry on known qubits with known-1 controls, Givens on known
    qubits holding different values. Not eligible: unknown controls, a flipped
    qubit already varying, Givens on equal known qubits (acts nowhere)."""
    parts = [[W.X(n - 1), W.X(2)],
             [W.H(0), W.Rx(1, 0.7), W.Ry(3, 1.9, n - 1), W.Givens(2, 4, 0.6),
              W.Ry(5, 0.8, 0),            # control 0 varies: a pass of its own
              W.H(6), W.H(0),             # H(0) again: qubit 0 varies
              W.Givens(7, 8, 0.3),        # both 0: acts nowhere
              W.Rx(9, 2.2, n - 1, 2)],
             [W.T(0), W.CX(0, 10), W.H(10), W.H(11)]]
    for form in (0, 1):
        got, _ = run(n, parts, 1e-14, 1 << 12, form=form)
        compare_states(got, oracle(n, parts, 1e-14), 1e-14)
        off, _ = run(n, parts, 1e-14, 1 << 12, expand=0, form=form)
        compare_states(got, off, 1e-14)


def test_zero_entries_and_pruning():
    """Ry(0) has zero off-diagonal entries: those images are exact zeros and
    dropped. Small angles give images below eps, pruned on the final amplitude."""
    n = 20
    parts = [[W.Ry(0, 0.0), W.H(1), W.Ry(2, 1e-9), W.Ry(3, 3e-7), W.Rx(4, 1e-8), W.H(5)]]
    for eps in (0.0, 1e-14, 1e-9, 1e-6):
        got, _ = run(n, parts, eps, 1 << 8)
        compare_states(got, oracle(n, parts, eps), eps)


def test_knowledge_from_uploaded_labels():
    """Labels uploaded with set_amplitudes: the device masks tell which qubits
    are constant; expansion passes on those, merging passes on the rest."""
    n = 70
    rng = np.random.default_rng(5)
    m = 500
    free = [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 65]
    codes = rng.choice(1 << len(free), size=m, replace=False)
    labels = [(1 << 30) | (1 << 66) | sum(((int(c) >> b) & 1) << q for b, q in enumerate(free))
              for c in codes]
    lo = np.array([v & (2**64 - 1) for v in labels], np.uint64)
    hi = np.array([v >> 64 for v in labels], np.uint64)
    init = (hi, lo, rng.normal(size=m), rng.normal(size=m))
    parts = [[W.H(30), W.H(66), W.H(40), W.Givens(41, 30, 0.4)],   # 30 now varies
             [W.H(0), W.H(65), W.H(50), W.H(30)]]
    got, c = run(n, parts, 1e-14, 1 << 16, init=init)
    compare_states(got, oracle(n, parts, 1e-14, init=init), 1e-14)


def test_capacity_failure_in_expansion():
    st = sps.SparseState(30, 1000)
    st.apply(W.to_array([W.H(q) for q in range(5)]), 0.0)          # 32 entries
    before = st.get_amplitudes()
    st.apply(W.to_array([W.X(20), W.H(10), W.H(11), W.H(12), W.H(13), W.H(14), W.Z(3)]), 0.0)
    with pytest.raises(sps.SpsError) as e:                          # 32 * 32 > 1000
        st.sync()
    assert e.value.status == sps.SPS_ERR_CAPACITY and e.value.failed_gate == 1
    hi, lo, re, im = st.get_amplitudes()
    np.testing.assert_array_equal(np.sort(before[1] ^ np.uint64(1 << 20)), lo)
    # nothing is assumed after the failure; the state is usable
    parts = [[W.H(20), W.H(0), W.H(25)]]
    st.apply(W.to_array(parts[0]), 0.0)
    orc = OracleState(30)
    orc.apply(W.to_array([W.H(q) for q in range(5)] + [W.X(20)] + parts[0]), eps=0.0)
    compare_states(st.get_amplitudes(), orc.get(), 0.0)
    st.close()


def test_update_counter_and_reset():
    st = sps.SparseState(40, 1 << 12)
    st.apply(W.to_array([W.H(q) for q in range(10)]), 0.0)
    assert st.updates() == (1 << 10) - 1
    st.reset()                       # |0...0> again: every qubit known
    c0 = st.counters().kernel_launches
    st.apply(W.to_array([W.H(q) for q in range(10, 20)]), 0.0)
    assert st.counters().kernel_launches - c0 == 1
    assert st.nnz() == 1 << 10
    st.close()
