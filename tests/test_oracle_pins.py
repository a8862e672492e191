"""Pins for the CPU oracle against facts that do not come from the oracle.

Each test names what fixes the expected value:
  * the Kronecker-product construction of Sec. 2.1 (kron_ref.full_unitary),
  * a second dense simulator on an n-axis tensor (kron_ref.tensor_run),
  * integer addition (the adder), closed forms, invariants
    (norm, Hamming weight), and the identities H.H = 1 and C^-1 C = 1.
A plausible mistake in the oracle (a dropped term, a wrong sign, a swapped
matrix index, a wrong qubit order) fails at least one of them.
"""

import math

import numpy as np
import pytest

from oracle import OracleState, classical_eval, dense_run, sector_run
from paper_2105_01533_gb300 import workloads as W

import kron_ref


def sparse_vector(st: OracleState, n: int) -> np.ndarray:
    hi, lo, re, im = st.get()
    assert np.all(hi == 0)
    v = np.zeros(1 << n, dtype=complex)
    v[lo.astype(np.int64)] = re + 1j * im
    return v


def run_oracle(n, gates, eps=0.0, mode=0):
    st = OracleState(n)
    st.apply(gates, eps=eps, mode=mode)
    return st


# ---- single gates against the Kronecker construction ---------------------------
@pytest.mark.parametrize("op", sorted(W.OP_NAMES))
def test_each_gate_matches_kron_definition(op):
    """Every gate code with 0, 1 and 2 controls, on a random 4-qubit state
    prepared by a fixed prefix, equals the Kronecker-product matrix."""
    n = 4
    prep = W.to_array([W.H(0), W.H(1), W.Ry(2, 0.7), W.T(0), W.Rx(3, 1.9), W.CX(3, 1),
                       W.S(2), W.Ry(1, 2.3, 0)])
    rng = W.SplitMix64(op)
    for nctl in range(3):
        ntarg = 2 if op == W.OP_GIVENS else 1
        qs = rng.distinct(n, ntarg + nctl)
        theta = rng.angle()
        if op == W.OP_GIVENS:
            g = W.Givens(qs[0], qs[1], theta, *qs[2:])
        else:
            g = W.gate(op, qs[0], qs[1:], theta)
        gates = np.concatenate([prep, W.to_array([g])])
        want = kron_ref.kron_run(n, gates)
        for mode in (0, 1):
            got = sparse_vector(run_oracle(n, gates, mode=mode), n)
            np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
        dense = dense_run(n, gates)
        np.testing.assert_allclose(dense, want, rtol=0, atol=1e-13)


def test_random_circuits_match_kron_definition():
    n = 5
    for seed in range(6):
        gates = W.random_all_gates(seed, n, 40, max_controls=2, branch_frac=0.4)
        want = kron_ref.kron_run(n, gates)
        got = sparse_vector(run_oracle(n, gates), n)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
        np.testing.assert_allclose(dense_run(n, gates), want, rtol=0, atol=1e-12)


def test_tensor_simulator_agrees_with_kron():
    """Pins the second numpy reference itself against the first."""
    n = 5
    gates = W.random_all_gates(11, n, 30, max_controls=2)
    np.testing.assert_allclose(kron_ref.tensor_run(n, gates), kron_ref.kron_run(n, gates),
                               rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_larger_circuits_match_tensor_simulator(seed):
    n = 12
    gates = W.random_all_gates(100 + seed, n, 150, max_controls=3, branch_frac=0.25)
    want = kron_ref.tensor_run(n, gates)
    got = sparse_vector(run_oracle(n, gates), n)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


# ---- textbook closed forms ------------------------------------------------------
def test_basis_facts():
    r = math.sqrt(0.5)
    st = run_oracle(1, W.to_array([W.H(0)]))
    np.testing.assert_array_equal(sparse_vector(st, 1), [r, r])
    th = 1.234
    st = run_oracle(1, W.to_array([W.Ry(0, th)]))
    np.testing.assert_allclose(sparse_vector(st, 1), [math.cos(th / 2), math.sin(th / 2)],
                               atol=1e-16)
    st = run_oracle(1, W.to_array([W.Rx(0, th)]))
    np.testing.assert_allclose(sparse_vector(st, 1),
                               [math.cos(th / 2), -1j * math.sin(th / 2)], atol=1e-16)
    st = run_oracle(1, W.to_array([W.X(0), W.Y(0)]))       # Y|1> = -i|0>
    np.testing.assert_array_equal(sparse_vector(st, 1), [-1j, 0])
    st = run_oracle(1, W.to_array([W.Y(0)]))               # Y|0> = i|1>
    np.testing.assert_array_equal(sparse_vector(st, 1), [0, 1j])
    # qubit order: X on qubit 3 of 5 gives label 8
    st = run_oracle(5, W.to_array([W.X(3)]))
    hi, lo, re, im = st.get()
    assert lo.tolist() == [8] and re.tolist() == [1.0]
    # Rz = e^{-i theta/2} P(theta) on |1>
    st = run_oracle(1, W.to_array([W.X(0), W.Rz(0, th)]))
    np.testing.assert_allclose(sparse_vector(st, 1), [0, np.exp(0.5j * th)], atol=1e-16)
    # Givens on |p=1, q=0> = e1 -> -sin|e0> + cos|e1>
    st = run_oracle(2, W.to_array([W.X(0), W.Givens(0, 1, th)]))
    np.testing.assert_allclose(sparse_vector(st, 2), [0, math.cos(th), -math.sin(th), 0],
                               atol=1e-16)


def test_uniform_superposition_closed_form():
    n, k = 20, 10
    qs = list(range(0, 20, 2))
    st = run_oracle(n, W.to_array([W.H(q) for q in qs]))
    hi, lo, re, im = st.get()
    assert len(lo) == 1 << k
    assert np.all(np.abs(re - 2.0 ** (-k / 2)) < 1e-15) and np.all(im == 0)
    spread = np.zeros(1 << k, np.uint64)
    for j, q in enumerate(qs):
        spread |= ((np.arange(1 << k, dtype=np.uint64) >> np.uint64(j)) & np.uint64(1)) << np.uint64(q)
    np.testing.assert_array_equal(np.sort(lo), np.sort(spread))


# ---- identities -----------------------------------------------------------------
def test_hh_is_identity_on_keys():
    gates = W.random_mix(5, 24, 300, keep_branch=W.CountingBound(4096))
    st = run_oracle(24, gates, eps=1e-14)
    hi0, lo0, re0, im0 = st.get()
    for q in (0, 5, 23):
        st2 = st.clone()
        st2.apply(W.to_array([W.H(q), W.H(q)]), eps=0.0)
        hi, lo, re, im = st2.get()
        np.testing.assert_array_equal(lo, lo0)
        np.testing.assert_allclose(re + 1j * im, re0 + 1j * im0, rtol=0, atol=1e-15)


def test_circuit_then_inverse_returns_start():
    for seed in range(4):
        n = 30 + 20 * seed
        gates = W.random_all_gates(seed, n, 120, max_controls=2, branch_frac=0.15)
        st = run_oracle(n, np.concatenate([gates, W.inverse(gates)]), eps=1e-14)
        hi, lo, re, im = st.get()
        assert hi.tolist() == [0] and lo.tolist() == [0]
        assert abs(re[0] - 1.0) < 1e-12 and abs(im[0]) < 1e-12


def test_norm_preserved():
    gates = W.random_mix(3, 24, 2000, keep_branch=W.CountingBound(4096))
    st = run_oracle(24, gates, eps=0.0)
    hi, lo, re, im = st.get()
    assert abs(np.sum(re * re + im * im) - 1.0) < 1e-12


def test_scatter_and_gather_modes_bit_identical():
    """The scatter form and the insert-once rule of Sec. 3.1 give the same
    floating-point result, bit for bit."""
    for seed in range(5):
        gates = W.random_all_gates(seed + 40, 18, 200, max_controls=2, branch_frac=0.35)
        a = run_oracle(18, gates, eps=1e-14, mode=0).get()
        b = run_oracle(18, gates, eps=1e-14, mode=1).get()
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


def test_dense_checker_on_24_qubit_mix():
    gates = W.random_mix(0, 20, 600, keep_branch=W.CountingBound(4096))
    st = run_oracle(20, gates, eps=0.0)
    dense = dense_run(20, gates)
    np.testing.assert_allclose(sparse_vector(st, 20), dense, rtol=0, atol=1e-12)


def test_prune_threshold_is_strict():
    """Entries with re^2+im^2 < eps^2 go, entries at exactly eps^2 stay, exact
    zeros always go (after a branching gate only)."""
    st = OracleState(3)
    st.set([0, 0, 0], [0, 2, 4], [0.5, 0.25, 0.125], [0.0, 0.0, 0.0])
    # Ry(pi) maps |x,0> -> |x,1> with cos(pi/2) ~ 6e-17 left on |x,0>
    st.apply(W.to_array([W.Ry(0, math.pi)]), eps=1e-15)
    hi, lo, re, im = st.get()
    assert lo.tolist() == [1, 3, 5]
    st = OracleState(2)
    st.set([0], [0], [3e-8], [4e-8])          # |a| = 5e-8, |a|^2 = 2.5e-15
    st.apply(W.to_array([W.X(1)]), eps=1.0)   # permutations never prune
    assert st.nnz() == 1
    st.apply(W.to_array([W.H(0), W.H(0)]), eps=5e-8 * math.sqrt(0.5) * math.sqrt(0.5) * 2)
    assert st.nnz() in (0, 1)


def test_prune_keeps_an_entry_at_exactly_eps_squared():
    """The strict reading: an entry with re^2 + im^2 == eps^2 exactly stays,
    one an ulp below goes. eps = 2^-20 makes eps^2 = 2^-40 exact, and Ry(0)
    copies each amplitude unchanged (cos 0 = 1) while its partner gets an
    exact zero (sin 0 = 0), which always goes."""
    eps = 2.0 ** -20
    below = np.nextafter(eps, 0.0)
    assert below * below < eps * eps
    st = OracleState(4)
    st.set([0, 0, 0, 0], [0, 2, 4, 8], [eps, below, 0.0, -eps], [0.0, 0.0, eps, 0.0])
    st.apply(W.to_array([W.Ry(0, 0.0)]), eps=eps)
    hi, lo, re, im = st.get()
    assert lo.tolist() == [0, 4, 8]
    assert re.tolist() == [eps, 0.0, -eps] and im.tolist() == [0.0, eps, 0.0]
    # the insert-once mode prunes the same way
    st = OracleState(4)
    st.set([0, 0], [0, 2], [eps, below], [0.0, 0.0])
    st.apply(W.to_array([W.Ry(0, 0.0)]), eps=eps, mode=1)
    assert st.get()[1].tolist() == [0]


# ---- reversible arithmetic ------------------------------------------------------
def test_adder_is_integer_addition():
    lay = W.AdderLayout(32)
    add = W.cuccaro_adder(lay)
    rng = np.random.default_rng(7)
    a = rng.integers(0, 2 ** 32, 500, dtype=np.uint64)
    b = rng.integers(0, 2 ** 32, 500, dtype=np.uint64)
    a[:3] = [0, 2 ** 32 - 1, 2 ** 31]
    b[:3] = [0, 1, 2 ** 31]
    key = a | (b << np.uint64(32))
    hi0 = np.zeros_like(key)
    hi, lo = classical_eval(lay.nqubits, add, hi0, key)
    s = [(int(x) + int(y)) for x, y in zip(a, b)]
    want_lo = np.array([int(x) | ((v & 0xFFFFFFFF) << 32) for x, v in zip(a, s)], np.uint64)
    want_hi = np.array([(v >> 32) << 1 for v in s], np.uint64)  # cout is qubit 65
    np.testing.assert_array_equal(lo, want_lo)
    np.testing.assert_array_equal(hi, want_hi)


def test_sparse_oracle_on_permutations_equals_classical_eval():
    lay = W.AdderLayout(32)
    add = W.cuccaro_adder(lay)
    prep = W.to_array([W.H(q) for q in lay.a[:6]] + [W.X(lay.b[i]) for i in (0, 3, 31)])
    st = run_oracle(lay.nqubits, np.concatenate([prep, add]))
    hi, lo, re, im = st.get()
    pre = run_oracle(lay.nqubits, prep).get()
    chi, clo = classical_eval(lay.nqubits, add, pre[0], pre[1])
    order = np.lexsort((clo, chi))
    np.testing.assert_array_equal(hi, chi[order])
    np.testing.assert_array_equal(lo, clo[order])
    np.testing.assert_array_equal(re, pre[2][order])
    np.testing.assert_array_equal(im, pre[3][order])


def adder_closed_form(wl: W.AdderWorkload):
    """Final state of the adder workload from integer addition alone:
    keys (a, b) for a < 2^width, amplitude 2^(-width/2) * prod_j e^{i phi_j}
    over CP pairs whose two bits are set in the registers after the adder
    (a in a, (a + b) mod 2^n in b)."""
    n, w = wl.layout.nbits, wl.width
    avals = np.arange(1 << w, dtype=np.uint64)
    bsum = (avals + np.uint64(wl.b_const)) & np.uint64((1 << n) - 1)
    reg = avals | (bsum << np.uint64(n))          # label of qubits 0..2n-1 after the adder
    phase = np.zeros(len(avals))
    for q1, q2, phi in wl.cp_pairs:
        both = ((reg >> np.uint64(q1)) & np.uint64(1)) & ((reg >> np.uint64(q2)) & np.uint64(1))
        phase += phi * both.astype(float)
    keys = avals | (np.uint64(wl.b_const) << np.uint64(n))
    amp = 2.0 ** (-w / 2) * np.exp(1j * phase)
    return keys, amp


def test_adder_workload_closed_form():
    wl = W.adder_workload(seed=1, width=10)
    st = run_oracle(wl.layout.nqubits, wl.gates, eps=1e-14)
    hi, lo, re, im = st.get()
    keys, amp = adder_closed_form(wl)
    order = np.argsort(keys)
    assert np.all(hi == 0)
    np.testing.assert_array_equal(lo, keys[order])
    np.testing.assert_allclose(re + 1j * im, amp[order], rtol=0, atol=1e-12)


# ---- number-conserving workload -------------------------------------------------
def test_givens_conserves_weight_and_matches_tensor_sim():
    n, k = 12, 3
    gates = W.givens_workload(seed=9, nqubits=n, modes=k, layers=6)
    st = run_oracle(n, gates, eps=0.0)
    hi, lo, re, im = st.get()
    weights = [bin(int(x)).count("1") for x in lo]
    assert set(weights) == {k}
    assert len(lo) <= math.comb(n, k)
    want = kron_ref.tensor_run(n, gates)
    np.testing.assert_allclose(sparse_vector(st, n), want, rtol=0, atol=1e-12)


def test_givens_workload_inverse_returns_start():
    gates = W.givens_workload(seed=3, nqubits=64, modes=4, layers=3)
    st = run_oracle(64, np.concatenate([gates, W.inverse(gates)]), eps=1e-14)
    hi, lo, re, im = st.get()
    assert lo.tolist() == [0] and hi.tolist() == [0]
    assert abs(re[0] - 1) < 1e-12 and abs(im[0]) < 1e-12


def test_probability_matches_dense():
    n = 10
    gates = W.random_all_gates(77, n, 80)
    st = run_oracle(n, gates)
    psi = kron_ref.kron_run(n, gates)
    p = np.abs(psi) ** 2
    idx = np.arange(1 << n)
    for mask, val in [(0, 0), (1, 1), (0b1010, 0b1000), (0x3FF, 5)]:
        want = p[(idx & mask) == val].sum()
        got = st.probability([mask, 0], [val, 0])
        assert abs(got - want) < 1e-12


def test_bad_records_are_rejected():
    st = OracleState(4)
    bad = W.to_array([W.H(0), W.X(4)])
    with pytest.raises(ValueError, match="index 1"):
        st.apply(bad)
    with pytest.raises(ValueError):
        st.apply(W.to_array([W.X(1, 1)]))          # control on its own target
    with pytest.raises(ValueError):
        st.apply(W.to_array([W.Givens(2, 2, 0.1)]))


# ---- measurement with collapse ----------------------------------------------------
def test_measure_bell_pair_closed_form():
    """(|00> + |11>)/sqrt2: each outcome has probability 1/2 and leaves the
    matching basis state with amplitude 1 (Sec. 2.1 projection)."""
    for r, outcome, label in ((0.3, 1, 3), (0.7, 0, 0)):
        st = run_oracle(4, W.to_array([W.H(0), W.CX(0, 1)]))
        got = st.measure(0, r)
        assert got[0] == outcome and abs(got[1] - 0.5) < 1e-15
        hi, lo, re, im = st.get()
        assert lo.tolist() == [label] and abs(re[0] - 1.0) < 1e-15 and im[0] == 0.0
        # the partner qubit is now determined: measuring it is certain
        assert st.measure(1, 0.999)[0] == outcome


def test_measure_matches_numpy_projection():
    """Marginals and post-measurement states against a numpy statevector from the
    tensor simulator: P(q = 1) = sum over indices with bit q set of |v|^2, and
    the kept part of v divided by its norm."""
    n = 7
    gates = W.to_array([W.H(q) for q in range(4)] + [W.Ry(4, 0.8, 1), W.Rx(5, 1.3, 2),
                       W.CX(0, 6), W.T(3), W.P(5, 0.4, 0), W.Givens(2, 6, 0.5), W.H(1)])
    v = kron_ref.tensor_run(n, gates)
    idx = np.arange(1 << n)
    for q in range(n):
        p1 = float(np.sum(np.abs(v[((idx >> q) & 1) == 1]) ** 2))
        for r in (0.05, 0.37, 0.61, 0.95):
            if abs(r - p1) < 1e-9:     # a draw on the edge: either outcome is right
                continue
            st = run_oracle(n, gates)
            outcome, p = st.measure(q, r)
            assert outcome == (1 if r < p1 else 0)
            assert abs(p - (p1 if outcome else 1 - p1)) < 1e-12
            w = np.where(((idx >> q) & 1) == outcome, v, 0)
            w = w / np.linalg.norm(w)
            np.testing.assert_allclose(sparse_vector(st, n), w, atol=1e-12)


def test_measure_constant_qubit_and_unnormalised_state():
    """A qubit that is 0 in every label: outcome 0 with probability 1, amplitudes
    unchanged. An input of norm 2: probabilities are relative, the result has
    norm 1."""
    st = run_oracle(10, W.to_array([W.H(0), W.H(1)]))
    before = st.get()
    assert st.measure(7, 0.999999) == (0, 1.0)
    after = st.get()
    for a, b in zip(after[:2], before[:2]):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_allclose(after[2], before[2], rtol=1e-15)   # divided by sqrt(1 + ulp)
    st = OracleState(10)
    st.set(np.zeros(4, np.uint64), np.array([0, 1, 2, 3], np.uint64),
           np.array([1.0, 1.0, 1.0, 1.0]), np.zeros(4))            # norm^2 = 4
    outcome, p = st.measure(1, 0.6)                                 # P(bit 1 = 1) = 1/2
    assert outcome == 0 and p == 0.5
    hi, lo, re, im = st.get()
    assert sorted(lo.tolist()) == [0, 1]
    np.testing.assert_allclose(re, [1 / math.sqrt(2)] * 2, rtol=1e-15)


def test_measure_rejects_bad_arguments():
    st = OracleState(5)
    for q, r in ((5, 0.5), (0, 1.0), (0, -0.1), (0, float("nan"))):
        with pytest.raises(ValueError):
            st.measure(q, r)


# ---- Pauli exponentials ---------------------------------------------------------------
def test_pauli_exp_matches_kron_definition():
    """exp(-i theta/2 P) for random Pauli strings (X, Y and Z factors) with 0 or 1
    control, on a random 5-qubit state: against scipy's matrix exponential of the
    Kronecker product of the factors."""
    n = 5
    rng = W.SplitMix64(2024)
    prep = W.to_array([W.H(0), W.Ry(1, 0.7), W.H(2), W.Rx(3, 1.9, 0), W.T(2), W.H(4),
                       W.P(4, 0.3, 1)])
    for trial in range(24):
        x = rng.below(1 << n)
        z = rng.below(1 << n)
        if (x | z) == 0:
            z = 1
        free = [q for q in range(n) if not ((x | z) >> q) & 1]
        c = (1 << free[rng.below(len(free))]) if free and trial % 2 else 0
        theta = rng.angle()
        want = kron_ref.pauli_exp_unitary(n, x, z, c, theta) @ kron_ref.kron_run(n, prep)
        st = run_oracle(n, prep)
        st.pauli_exp((x, 0), (z, 0), (c, 0), theta)
        np.testing.assert_allclose(sparse_vector(st, n), want, atol=1e-12)


def test_single_factor_exponentials_are_rotations():
    """exp(-i t/2 X_q), exp(-i t/2 Y_q), exp(-i t/2 Z_q) equal Rx, Ry, Rz on q."""
    n = 4
    prep = W.to_array([W.H(0), W.Ry(1, 0.4), W.H(3), W.T(3)])
    for (x, z), gate in (((1 << 2, 0), W.Rx), ((1 << 2, 1 << 2), W.Ry), ((0, 1 << 2), W.Rz)):
        a = run_oracle(n, prep)
        a.pauli_exp((x, 0), (z, 0), (0, 0), 0.9)
        b = run_oracle(n, W.to_array(list(prep) + [gate(2, 0.9)]))
        np.testing.assert_allclose(sparse_vector(a, n), sparse_vector(b, n), atol=1e-15)


def test_pauli_exp_rejects_bad_strings():
    st = OracleState(6)
    for x, z, c in (((0, 0), (0, 0), (0, 0)), ((1 << 6, 0), (0, 0), (0, 0)),
                    ((1, 0), (0, 0), (1, 0)), ((0, 0), (1 << 2, 0), (1 << 2, 0))):
        with pytest.raises(ValueError):
            st.pauli_exp(x, z, c, 0.5)


# ---- weight-sector dense checker ---------------------------------------------
def test_sector_labels_are_the_weight_k_set():
    labels, amp = sector_run(16, 0b1111, W.to_array([]))
    assert len(labels) == math.comb(16, 4)
    assert np.all(np.diff(labels.astype(np.int64)) > 0)
    assert {bin(int(x)).count("1") for x in labels} == {4}
    assert np.count_nonzero(amp) == 1 and amp[labels == 0b1111][0] == 1.0


def test_sector_sim_matches_tensor_simulator():
    """A number-conserving circuit on 10 qubits, 3 modes: the sector vector
    embedded in 2^10 equals the n-axis tensor simulator (Sec. 2.2), and the
    tensor state is exactly zero outside the sector."""
    n, k = 10, 3
    gates = W.givens_workload(seed=4, nqubits=n, modes=k, layers=8)
    gates = np.concatenate([gates, W.to_array([W.Rz(2, 0.7, 5), W.T(4), W.P(1, 1.3, 0)])])
    labels, amp = sector_run(n, (1 << k) - 1, gates[k:])
    want = kron_ref.tensor_run(n, gates)
    np.testing.assert_allclose(amp, want[labels.astype(np.int64)], rtol=0, atol=1e-12)
    outside = np.ones(1 << n, bool)
    outside[labels.astype(np.int64)] = False
    assert np.max(np.abs(want[outside])) < 1e-15
    assert abs(np.sum(np.abs(amp) ** 2) - 1.0) < 1e-12


def test_sector_sim_bit_identical_to_sparse_oracle():
    """Without pruning the sparse oracle and the sector vector form every
    amplitude with the same products and sums."""
    n, k = 24, 3
    gates = W.givens_workload(seed=5, nqubits=n, modes=k, layers=10)
    labels, amp = sector_run(n, (1 << k) - 1, gates[k:])
    hi, lo, re, im = run_oracle(n, gates, eps=0.0).get()
    nz = amp != 0
    np.testing.assert_array_equal(lo, labels[nz])
    np.testing.assert_array_equal(re, amp[nz].real)
    np.testing.assert_array_equal(im, amp[nz].imag)


def test_sector_sim_rejects_weight_changing_gates():
    with pytest.raises(ValueError):
        sector_run(8, 0b11, W.to_array([W.H(0)]))
    with pytest.raises(ValueError):
        sector_run(8, 0b11, W.to_array([W.X(3)]))
