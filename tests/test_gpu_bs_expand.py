"""GPU parity of an expansion from |0...0> fused with the bit-sliced run after
it (one launch compiled for the run: the expansion's outputs are generated in
bit-sliced form, walked, and written once). The form is taken when sps_apply
starts with a reset still pending, the first pass is an expansion of one-qubit
gates and the second a bit-sliced run. Results are checked against the CPU
oracle and against the same gates applied without a pending reset (the
expansion and the run as two passes); the profile must show the fused launch
(kind 7 with the compiled flag)."""

import numpy as np
import pytest

from oracle import OracleState
from paper_2105_01533_gb300 import sps
from paper_2105_01533_gb300 import workloads as W

from helpers import compare_states

pytestmark = pytest.mark.gpu

EPS = 1e-14
FORCE = [(sps.SPS_OPT_BITSLICE_MIN_OPS, 1), (sps.SPS_OPT_BITSLICE_MIN_NNZ, 0),
         (sps.SPS_OPT_SMALL_RUN_CAP, 0), (sps.SPS_OPT_BITSLICE_JIT, 2)]


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2105_01533_gb300 import build as B
    B.build()
    sps.load_library()
    yield


def run(n, gates, cap, opts, reset_first):
    st = sps.SparseState(n, cap)
    for o, v in opts:
        st.set_option(o, v)
    st.set_option(sps.SPS_OPT_PROFILE, 1)
    if reset_first:
        st.reset()
    st.apply(gates, EPS)
    recs = st.profile_read()
    got = st.get_amplitudes()
    upd = st.updates()
    st.close()
    fused = [r for r in recs if r["kind"] == 7 and r["flags"] & 16]
    return got, upd, fused


def run_gates(seed, n, d, nrun, kinds, nphase=6):
    """d one-qubit branching gates on distinct qubits (from |0...0>; kinds cycle
    through the list), then a phase/permutation run of nrun gates with up to 3
    controls, nphase of them arbitrary phases (each Rx or Ry of the head and
    each arbitrary phase takes phase-table bits; one table holds 22)."""
    rng = W.SplitMix64(seed)
    qs = rng.distinct(n, d)
    head = []
    for j, q in enumerate(qs):
        k = kinds[j % len(kinds)]
        if k == "h":
            head.append(W.H(q))
        elif k == "ry":
            head.append(W.Ry(q, 0.3 + 2.0 * rng.uniform()))
        else:
            head.append(W.Rx(q, 0.3 + 2.0 * rng.uniform()))
    codes = [W.OP_X, W.OP_Z, W.OP_S, W.OP_T, W.OP_TDG, W.OP_Y, W.OP_X, W.OP_X]
    body = []
    for i in range(nrun):
        op = W.OP_P if i % max(1, nrun // max(1, nphase)) == 7 else codes[rng.below(len(codes))]
        q = rng.distinct(n, 1 + rng.below(4))
        body.append(W.gate(op, q[0], q[1:], rng.angle()))
    return W.to_array(head + body)


@pytest.mark.parametrize("n,d,kinds,seed", [
    (20, 10, ["h"], 1), (40, 12, ["h", "h", "ry"], 2), (67, 11, ["rx", "h", "h", "h", "ry"], 3),
    (100, 9, ["ry", "h", "h"], 4), (127, 13, ["h"], 5), (33, 5, ["h"], 6)])
def test_fused_expansion_matches_oracle_and_two_passes(n, d, kinds, seed):
    gates = run_gates(seed, n, d, 150, kinds)
    got, upd, fused = run(n, gates, 1 << (d + 1), FORCE, True)
    assert len(fused) == 1 and fused[0]["n_out"] == 1 << d
    ref, upd0, fused0 = run(n, gates, 1 << (d + 1), FORCE, False)
    assert not fused0
    assert upd == upd0
    compare_states(got, ref, EPS)
    orc = OracleState(n)
    orc.apply(gates, eps=EPS)
    compare_states(got, orc.get(), EPS)


def test_fused_expansion_pure_permutation_run():
    """A run without phases: every output takes the common factor."""
    n = 30
    gates = W.to_array([W.H(q) for q in range(12)] +
                       [W.X(20 + (i % 9), i % 12, (i + 3) % 12) for i in range(40)])
    got, upd, fused = run(n, gates, 1 << 13, FORCE, True)
    assert len(fused) == 1
    orc = OracleState(n)
    orc.apply(gates, eps=EPS)
    compare_states(got, orc.get(), EPS)


def test_fused_expansion_not_taken_when_outputs_could_prune():
    """An Ry whose sine is below eps would prune outputs: the two passes run."""
    n = 24
    gates = W.to_array([W.H(q) for q in range(10)] + [W.Ry(11, 1e-15)] +
                       [W.T(q, (q + 1) % 10) for q in range(10)])
    got, upd, fused = run(n, gates, 1 << 13, FORCE, True)
    assert not fused
    orc = OracleState(n)
    orc.apply(gates, eps=EPS)
    compare_states(got, orc.get(), EPS)


def test_adder67_w24_after_reset_closed_form():
    """The benchmark's step shape (reset, then the whole adder workload): the 24
    Hadamards and the adder run in one launch, checked against integer
    addition and the controlled-phase closed form."""
    from test_gpu_large import adder_closed_form
    wl = W.adder_workload(seed=1, width=24)
    st = sps.SparseState(wl.layout.nqubits, 1 << 25)
    st.set_option(sps.SPS_OPT_PROFILE, 1)
    st.reset()
    st.apply(wl.gates, EPS)
    recs = st.profile_read()
    hi, lo, re, im = st.get_amplitudes()
    st.close()
    assert [r for r in recs if r["kind"] == 7 and r["flags"] & 16]
    keys, cre, cim = adder_closed_form(wl)
    order = np.argsort(keys)
    assert np.all(hi == 0)
    np.testing.assert_array_equal(lo, keys[order])
    err = max(float(np.max(np.abs(re - cre[order]))), float(np.max(np.abs(im - cim[order]))))
    assert err <= 1e-12, err
