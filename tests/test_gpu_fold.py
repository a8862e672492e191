"""GPU parity of fused runs compiled with known qubits resolved (SPS_OPT_FOLD):
gates with a control known 0 dropped, known controls removed, flips of known
qubits collected into one flip, adjacent flips with one condition merged.
Each case is compared with the oracle and with the same circuit compiled one
op per gate, in the direct and bit-sliced fused forms and in one-block runs."""

import pytest

from oracle import OracleState
from paper_2105_01533_gb300 import sps
from paper_2105_01533_gb300 import workloads as W

from helpers import compare_states

pytestmark = pytest.mark.gpu

FORMS = {
    "direct": [(sps.SPS_OPT_SMALL_RUN_CAP, 0), (sps.SPS_OPT_BITSLICE_MIN_OPS, 0)],
    "bitsliced": [(sps.SPS_OPT_SMALL_RUN_CAP, 0), (sps.SPS_OPT_BITSLICE_MIN_OPS, 4),
                  (sps.SPS_OPT_BITSLICE_MIN_NNZ, 0)],
    "one-block": [(sps.SPS_OPT_SMALL_RUN_CAP, 2048)],
}


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2105_01533_gb300 import build as B
    B.build()
    sps.load_library()
    yield


def run(n, parts, eps, cap, fold, opts):
    st = sps.SparseState(n, cap)
    st.set_option(sps.SPS_OPT_FOLD, fold)
    for o, v in opts:
        st.set_option(o, v)
    for g in parts:
        st.apply(W.to_array(g), eps)
    got = st.get_amplitudes()
    upd = st.updates()
    st.close()
    return got, upd


def oracle(n, parts, eps):
    orc = OracleState(n)
    for g in parts:
        orc.apply(W.to_array(g), eps=eps)
    return orc.get()


def mixed_run(rng, n, qubits, count):
    """Phase/permutation gates over `qubits` with 0..3 controls."""
    gates = []
    for _ in range(count):
        q = [qubits[i] for i in rng.distinct(len(qubits), 4)]
        nc = rng.below(4)
        kind = rng.below(10)
        if kind < 5:
            gates.append(W.X(q[0], *q[1:1 + nc]))
        elif kind == 5:
            gates.append(W.Y(q[0], *q[1:1 + min(nc, 1)]))
        elif kind == 6:
            gates.append(W.T(q[0], *q[1:1 + nc]))
        elif kind == 7:
            gates.append(W.P(q[0], rng.angle(), *q[1:1 + nc]))
        elif kind == 8:
            gates.append(W.Rz(q[0], rng.angle(), *q[1:1 + min(nc, 1)]))
        else:
            gates.append(W.Z(q[0], *q[1:1 + nc]))
    return gates


@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("n,seed", [(24, 1), (64, 2), (70, 3), (127, 4)])
def test_random_runs_with_known_qubits(form, n, seed):
    rng = W.SplitMix64(seed)
    qubits = rng.distinct(n, 20)
    parts = [[W.X(q) for q in qubits[10:14]] + [W.H(q) for q in qubits[:8]],
             mixed_run(rng, n, qubits, 300),
             [W.H(qubits[15]), W.H(qubits[0])],
             mixed_run(rng, n, qubits, 300)]
    want = oracle(n, parts, 1e-14)
    got, upd = run(n, parts, 1e-14, 1 << 12, 1, FORMS[form])
    compare_states(got, want, 1e-14)
    off, upd_off = run(n, parts, 1e-14, 1 << 12, 0, FORMS[form])
    compare_states(got, off, 1e-14)
    assert upd == upd_off          # updates count gates, however many ops remain


def test_adder_constants_fold():
    """The adder over a superposed register and a classical constant: most
    carries and the constant's bits are known, so the run folds."""
    wl = W.adder_workload(seed=3, width=8)
    parts = [wl.gates]
    n = wl.layout.nqubits
    for form in sorted(FORMS):
        got, _ = run(n, parts, 1e-14, 1 << 10, 1, FORMS[form])
        compare_states(got, oracle(n, parts, 1e-14), 1e-14)


def test_runs_that_fold_to_one_flip_or_nothing():
    """Flips of known qubits only: the run becomes one flip of the changed
    qubits, or no op at all when they cancel; labels change as they must and
    the update count still counts every gate."""
    n = 40
    one = [W.X(5), W.X(6, 5), W.X(7, 9), W.Z(8), W.T(8), W.X(5), W.CX(6, 12)]
    none = [W.X(21), W.X(21), W.Z(22), W.X(23, 24), W.CCX(25, 26, 27)]
    parts = [[W.H(0), W.H(1)], one, none]
    for form in sorted(FORMS):
        got, upd = run(n, parts, 0.0, 64, 1, FORMS[form])
        compare_states(got, oracle(n, parts, 0.0), 0.0)
        assert upd == 1 + 2 + 4 * len(one) + 4 * len(none)


def test_merged_flips_and_cancellation():
    """Adjacent flips with one condition merge (and cancel when they repeat);
    merged flips expand to one bit-sliced op per target."""
    n = 30
    parts = [[W.H(q) for q in range(6)],
             [W.CX(0, 10), W.CX(0, 11), W.CX(0, 12), W.CX(0, 12), W.CCX(1, 2, 13),
              W.CCX(1, 2, 14), W.CX(13, 15), W.X(16), W.X(16), W.X(17), W.CX(3, 20), W.T(20)]]
    for form in sorted(FORMS):
        got, _ = run(n, parts, 0.0, 256, 1, FORMS[form])
        compare_states(got, oracle(n, parts, 0.0), 0.0)
