"""GPU parity of Pauli exponentials (sps_pauli_exp) against the oracle: strings
with X, Y and Z factors (one branching pass on the pairs j, j ^ x, in both
branching forms), strings of Z factors only (a fused run), with and without
controls, on 64- and 128-bit labels, mixed with ordinary gates."""

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


def words(bits):
    v = sum(1 << b for b in bits)
    return (v & (2**64 - 1), v >> 64)


def random_string(rng, qubits, kinds):
    """X/Y/Z factors on the given qubits; kinds: which factors to draw from."""
    x, z = [], []
    for q in qubits:
        f = kinds[rng.below(len(kinds))]
        if f in "XY":
            x.append(q)
        if f in "ZY":
            z.append(q)
    return words(x), words(z)


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("n,seed", [(20, 1), (64, 2), (100, 3), (127, 4)])
def test_pauli_strings_match_oracle(form, n, seed):
    rng = W.SplitMix64(seed)
    qs = rng.distinct(n, 16)
    prep = W.to_array([W.H(q) for q in qs[:7]] + [W.Ry(qs[7], rng.angle(), qs[0]),
                      W.T(qs[1]), W.CX(qs[2], qs[8])])
    st = sps.SparseState(n, 1 << 15)
    st.set_option(sps.SPS_OPT_BRANCH_FORM, form)
    st.apply(prep, 1e-14)
    orc = OracleState(n)
    orc.apply(prep, eps=1e-14)
    for k in range(8):
        m = 1 + rng.below(5)
        support = [qs[(k + 2 * i) % 16] for i in range(m)]
        kinds = "XYZ" if k % 3 else "Z"
        x, z = random_string(rng, support, kinds)
        if x == (0, 0) and z == (0, 0):
            z = words(support[:1])
        free = [q for q in qs if q not in support]
        ctl = words([free[rng.below(len(free))]]) if k % 2 else (0, 0)
        theta = rng.angle()
        st.pauli_exp(x, z, ctl, theta, 1e-14)
        orc.pauli_exp(x, z, ctl, theta, eps=1e-14)
        compare_states(st.get_amplitudes(), orc.get(), 1e-14)
        g = W.to_array([W.H(qs[(3 * k) % 16]), W.CX(qs[(3 * k + 1) % 16], qs[(3 * k + 5) % 16])])
        st.apply(g, 1e-14)
        orc.apply(g, eps=1e-14)
    compare_states(st.get_amplitudes(), orc.get(), 1e-14)
    st.close()


def test_pauli_exp_on_fresh_and_uploaded_states():
    """From |0...0> (the flipped qubits constant: no entry meets a partner) and
    from uploaded labels; the result must not depend on what is known."""
    n = 70
    st = sps.SparseState(n, 1 << 12)
    orc = OracleState(n)
    for x, z, c, t in ((words([3, 66]), words([66, 10]), (0, 0), 0.7),
                       (words([3, 5]), words([5]), words([10]), 1.3),
                       (words([66]), words([]), words([3]), 2.1)):
        st.pauli_exp(x, z, c, t, 1e-14)
        orc.pauli_exp(x, z, c, t, eps=1e-14)
        compare_states(st.get_amplitudes(), orc.get(), 1e-14)
    st.close()


def test_pauli_exp_rejects_bad_strings():
    st = sps.SparseState(10, 64)
    for x, z, c, t in (((0, 0), (0, 0), (0, 0), 0.5), ((1 << 10, 0), (0, 0), (0, 0), 0.5),
                       ((1, 0), (0, 0), (1, 0), 0.5), ((1, 0), (0, 0), (0, 0), float("inf"))):
        with pytest.raises(sps.SpsError) as e:
            st.pauli_exp(x, z, c, t)
        assert e.value.status == sps.SPS_ERR_ARG
    st.close()
