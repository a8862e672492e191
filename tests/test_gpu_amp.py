"""GPU parity of amplitude-only branching passes (SPS_OPT_AMP_ONLY): where a
branching pass (one gate or a layer) meets only complete groups and prunes
nothing, the labels stay in place and only amplitudes are written. The result
must equal the out-of-place passes bit for bit (labels, amplitudes, update
count), and the oracle to the usual tolerance. Profile records show which
passes the form took (kind 10, n_out > 0)."""

import numpy as np
import pytest

from oracle import OracleState
from paper_2105_01533_gb300 import sps
from paper_2105_01533_gb300 import workloads as W

from helpers import compare_states

pytestmark = pytest.mark.gpu

AMP_KIND = 10


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2105_01533_gb300 import build as B
    B.build()
    sps.load_library()
    yield


def run(n, parts, eps, cap, amp, opts=(), init=None, between=None):
    """Applies each gate list in turn; `between(st, k)` may act on the state
    after part k. Returns the state, the update count and the number of
    passes the amplitude-only form took."""
    st = sps.SparseState(n, cap)
    st.set_option(sps.SPS_OPT_AMP_ONLY, amp)
    st.set_option(sps.SPS_OPT_PROFILE, 1)
    for o, v in opts:
        st.set_option(o, v)
    if init is not None:
        st.set_amplitudes(*init)
    took = 0
    for k, gates in enumerate(parts):
        st.apply(W.to_array(gates), eps)
        if between is not None:
            between(st, k)
        took += sum(1 for r in st.profile_read() if r["kind"] == AMP_KIND and r["n_out"] > 0)
    got = st.get_amplitudes()
    upd = st.updates()
    st.close()
    return got, upd, took


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


def givens_parts(n, modes, layers, seed, per_part=4):
    """The Givens workload (X on the first modes, then layers of n/2 Givens
    and n/2 CZ) cut into applies of per_part layers each."""
    g = W.givens_workload(seed=seed, nqubits=n, modes=modes, layers=layers)
    step = n * per_part
    return [g[:modes]] + [g[i:i + step] for i in range(modes, len(g), step)]


@pytest.mark.parametrize("n,modes,layers,lay", [(16, 3, 30, 4), (40, 2, 24, 4), (64, 3, 12, 1),
                                                (100, 2, 10, 4), (24, 5, 12, 4), (20, 6, 12, 4),
                                                (18, 6, 12, 1)])
def test_givens_layers_take_the_amplitude_form(n, modes, layers, lay):
    """Particle-number-conserving circuits: once every label of the sector is
    present, Givens layers and single Givens gates keep the label set. With 5
    or 6 occupied modes a label activates up to 5 or 6 Givens of a layer:
    groups of 32 and 64 members."""
    parts = givens_parts(n, modes, layers, seed=n + modes)
    opts = [(sps.SPS_OPT_LAYER_GATES, lay)]
    got, upd, took = run(n, parts, 1e-14, 1 << 18, 1, opts)
    ref, upd0, took0 = run(n, parts, 1e-14, 1 << 18, 0, opts)
    identical(got, ref)
    assert upd == upd0
    assert took > 0 and took0 == 0
    compare_states(got, oracle(n, parts, 1e-14), 1e-14)


@pytest.mark.parametrize("seed", range(3))
def test_mixed_circuits_fall_back_exactly(seed):
    """H, Rx, Ry and Givens with controls, CNOTs and phases between: some
    passes keep the label set, others create or prune labels (fallback), and
    permutations in between make the index stale."""
    n = 30
    rng = W.SplitMix64(500 + seed)
    parts = [[W.H(q) for q in range(8)]]
    for k in range(12):
        recs = []
        for _ in range(6):
            q = rng.distinct(12, 3)
            c = rng.below(6)
            if c == 0:
                recs.append(W.H(q[0]))
            elif c == 1:
                recs.append(W.Rx(q[0], rng.angle(), *([q[2]] if rng.below(2) else [])))
            elif c == 2:
                recs.append(W.Ry(q[0], rng.angle()))
            elif c == 3:
                recs.append(W.Givens(q[0], q[1], rng.angle()))
            elif c == 4:
                recs.append(W.CX(q[0], q[1]))
            else:
                recs.append(W.P(q[0], rng.angle(), q[1]))
        parts.append(recs)
    for eps in (0.0, 1e-14, 1e-4):
        opts = [(sps.SPS_OPT_SMALL_RUN_CAP, 0)]
        got, upd, took = run(n, parts, eps, 1 << 14, 1, opts)
        ref, upd0, _ = run(n, parts, eps, 1 << 14, 0, opts)
        identical(got, ref)
        assert upd == upd0
        compare_states(got, oracle(n, parts, eps), eps)


def test_closed_state_repeated_hadamards():
    """All 2^10 labels over ten qubits: gates on them keep the label set
    (amplitude form) unless they collapse a qubit to one value (an H on |+>:
    exact zeros, fallback); an H on an eleventh qubit doubles the state (an
    expansion), after which the index is rebuilt."""
    n = 24
    parts = [[W.H(q) for q in range(10)] + [W.T(3), W.CX(0, 1)],
             [W.H(2), W.H(5), W.Ry(7, 0.3)],
             [W.H(12)],
             [W.H(3), W.Rx(12, 0.8), W.Givens(1, 12, 0.5)],
             [W.Z(4), W.H(4)]]
    opts = [(sps.SPS_OPT_SMALL_RUN_CAP, 0), (sps.SPS_OPT_LAYER_GATES, 1)]
    got, upd, took = run(n, parts, 1e-14, 1 << 12, 1, opts)
    ref, upd0, _ = run(n, parts, 1e-14, 1 << 12, 0, opts)
    identical(got, ref)
    assert upd == upd0
    assert took >= 1      # (runs that collapse a qubit fall back, then skip one attempt)
    compare_states(got, oracle(n, parts, 1e-14), 1e-14)


def test_index_survives_phase_passes_and_not_measurement():
    """Phase-only fused passes keep the index; a measurement moves labels, so
    the next attempt rebuilds it. Results against the out-of-place passes."""
    n = 20
    parts = [[W.H(q) for q in range(8)],
             [W.H(1), W.Z(2), W.T(3), W.H(4)],
             [W.Ry(5, 0.9), W.S(0), W.Rz(6, 0.4)],
             [W.H(0), W.H(6)]]

    def between(st, k):
        if k == 1:
            st.measure(7, 0.3)

    opts = [(sps.SPS_OPT_SMALL_RUN_CAP, 0), (sps.SPS_OPT_LAYER_GATES, 1)]
    got, upd, took = run(n, parts, 1e-14, 1 << 10, 1, opts, between=between)
    ref, upd0, _ = run(n, parts, 1e-14, 1 << 10, 0, opts, between=between)
    identical(got, ref)
    assert upd == upd0
    assert took >= 2


def test_uploaded_state_and_option_values():
    n = 70
    rng = np.random.default_rng(3)
    m = 1 << 9
    labels = [(1 << 66) | sum(((c >> b) & 1) << (2 * b) for b in range(9)) for c in range(m)]
    lo = np.array([v & (2**64 - 1) for v in labels], np.uint64)
    hi = np.array([v >> 64 for v in labels], np.uint64)
    init = (hi, lo, rng.normal(size=m), rng.normal(size=m))
    parts = [[W.H(0), W.H(2), W.Givens(4, 6, 0.7), W.Ry(8, 1.1, 66)], [W.H(1)]]
    opts = [(sps.SPS_OPT_SMALL_RUN_CAP, 0)]
    got, upd, took = run(n, parts, 1e-14, 1 << 11, 1, opts, init=init)
    ref, upd0, _ = run(n, parts, 1e-14, 1 << 11, 0, opts, init=init)
    identical(got, ref)
    assert upd == upd0 and took >= 1
    compare_states(got, oracle(n, parts, 1e-14, init=init), 1e-14)
    st = sps.SparseState(10, 64)
    for v in (-1, 2):
        with pytest.raises(sps.SpsError):
            st.set_option(sps.SPS_OPT_AMP_ONLY, v)
    st.close()


@pytest.mark.parametrize("phases", ["cz", "cz+t"])
def test_sign_runs_taken_by_parity(phases):
    """With the bit-sliced form chosen for every phase run (thresholds at
    their minimum), a run of Z and controlled-Z gates after an amplitude-only
    run is applied by it as a parity of conditions; a run with a T gate is not
    (it stays a bit-sliced pass of its own). Both equal the passes without the
    amplitude-only form bit for bit."""
    n, modes = 20, 3
    g = W.givens_workload(seed=9, nqubits=n, modes=modes, layers=16)
    parts = [g[:modes]]
    rng = W.SplitMix64(77)
    for i in range(modes, len(g), n):
        layer = [tuple(r) for r in g[i:i + n]]
        if phases == "cz+t":
            layer.append(W.T(rng.below(n)))
        layer += [W.Z(rng.below(n))]
        parts.append(layer)
    opts = [(sps.SPS_OPT_BITSLICE_MIN_NNZ, 1), (sps.SPS_OPT_BITSLICE_MIN_OPS, 1),
            (sps.SPS_OPT_SMALL_RUN_CAP, 0)]
    got, upd, took = run(n, parts, 1e-14, 1 << 12, 1, opts)
    ref, upd0, _ = run(n, parts, 1e-14, 1 << 12, 0, opts)
    identical(got, ref)
    assert upd == upd0 and took > 0
    compare_states(got, oracle(n, parts, 1e-14), 1e-14)


CHAIN_KIND = 11


def run_counted(n, parts, eps, cap, opts):
    """As run(), also returning the kernel launches and the chain records
    (kind 11) seen."""
    st = sps.SparseState(n, cap)
    st.set_option(sps.SPS_OPT_PROFILE, 1)
    for o, v in opts:
        st.set_option(o, v)
    c0 = st.counters().kernel_launches
    chains = []
    for gates in parts:
        st.apply(W.to_array(gates), eps)
        chains += [r for r in st.profile_read() if r["kind"] == CHAIN_KIND]
    launches = st.counters().kernel_launches - c0
    got = st.get_amplitudes()
    upd = st.updates()
    st.close()
    return got, upd, launches, chains


@pytest.mark.parametrize("n,modes,layers,lay", [(16, 3, 24, 4), (24, 2, 16, 1), (40, 3, 8, 4)])
def test_fallback_chain_equals_separate_launches(n, modes, layers, lay):
    """The passes an attempt stands in for, as one cooperative launch: while
    the sector fills (attempts fail) the launch runs the layer or gather passes
    and the phase run; once it is full the launch returns at once. The state
    and update count equal the separate launches' bit for bit, and the oracle's."""
    parts = givens_parts(n, modes, layers, seed=3 * n + modes, per_part=2)
    base = [(sps.SPS_OPT_LAYER_GATES, lay), (sps.SPS_OPT_SMALL_RUN_CAP, 0),
            (sps.SPS_OPT_AMP_ONLY, 1)]
    got, upd, nl, chains = run_counted(n, parts, 1e-14, 1 << 16, base)
    ref, upd0, nl0, chains0 = run_counted(n, parts, 1e-14, 1 << 16,
                                          base + [(sps.SPS_OPT_FALLBACK_CHAIN, 0)])
    identical(got, ref)
    assert upd == upd0
    assert not chains0 and len(chains) > 0
    assert any(r["n_in"] > 0 for r in chains), "no chain ran its passes"
    assert any(r["n_in"] == 0 for r in chains), "no attempt took a run"
    assert nl < nl0
    compare_states(got, oracle(n, parts, 1e-14), 1e-14)


def test_givens_layer_is_three_launches():
    """Steady state of the Givens workload (every label of the sector present):
    each layer of n/2 Givens and n/2 CZ is the index check, the attempt and the
    chain, whatever the layer size of the fallback passes."""
    n, modes = 32, 3
    g = W.givens_workload(seed=5, nqubits=n, modes=modes, layers=40)
    prep, rest = g[:modes + 20 * n], g[modes + 20 * n:]
    st = sps.SparseState(n, 1 << 14)
    st.set_option(sps.SPS_OPT_SMALL_RUN_CAP, 0)
    st.apply(prep, 1e-14)
    st.sync()
    c0 = st.counters().kernel_launches
    st.apply(rest, 1e-14)
    st.sync()
    per_layer = (st.counters().kernel_launches - c0) / 20
    assert per_layer <= 3.0, per_layer
    orc = OracleState(n)
    orc.apply(g, eps=1e-14)
    compare_states(st.get_amplitudes(), orc.get(), 1e-14)
    st.close()


def test_mixed_circuits_chain_on_and_off():
    """Runs with gather-form single gates, layers and failed attempts that
    create and prune labels: chain on and off agree bit for bit."""
    n = 30
    rng = W.SplitMix64(901)
    parts = [[W.H(q) for q in range(8)]]
    for k in range(10):
        recs = []
        for _ in range(8):
            q = rng.distinct(14, 3)
            c = rng.below(4)
            if c == 0:
                recs.append(W.H(q[0]))
            elif c == 1:
                recs.append(W.Ry(q[0], rng.angle()))
            elif c == 2:
                recs.append(W.Givens(q[0], q[1], rng.angle()))
            else:
                recs.append(W.CZ(q[0], q[1]))
        parts.append(recs)
    for eps in (0.0, 1e-3):
        base = [(sps.SPS_OPT_SMALL_RUN_CAP, 0), (sps.SPS_OPT_AMP_ONLY, 1)]
        got, upd, _, chains = run_counted(n, parts, eps, 1 << 14, base)
        ref, upd0, _, _ = run_counted(n, parts, eps, 1 << 14,
                                      base + [(sps.SPS_OPT_FALLBACK_CHAIN, 0)])
        identical(got, ref)
        assert upd == upd0 and chains
        compare_states(got, oracle(n, parts, eps), eps)


def test_grid_barrier_wait_is_bounded():
    """The cooperative fallback launch's grid barrier: with every block
    arriving, three barriers pass and nothing is recorded; with one block
    missing its first arrival (a wait that nothing completes) the others give
    up after their poll limit, the launch ends and SPS_ERR_TIMEOUT is recorded
    for the host to read; the device stays usable."""
    assert sps.sps_barrier_selftest(99, 1 << 14) == sps.SPS_OK
    assert sps.sps_barrier_selftest(3, 1 << 14) == sps.SPS_ERR_TIMEOUT
    assert sps.sps_barrier_selftest(0, 1 << 14) == sps.SPS_ERR_TIMEOUT
    assert sps.sps_barrier_selftest(99, 1 << 14) == sps.SPS_OK
    st = sps.SparseState(20, 1 << 10)   # the context still serves new work
    st.apply(W.to_array([W.H(q) for q in range(6)]), 0.0)
    assert st.nnz() == 64
    st.close()
