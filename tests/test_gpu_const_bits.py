"""GPU parity for the constant-bit shortcut of branching passes.

The device keeps the OR and the AND of every stored label; a branching gate
whose flip bits agree in the two masks cannot pair any entry, so its pass
skips the partner index and the lookups. These tests drive the masks through
every kernel that writes labels (set, reset, fused direct and bit-sliced,
scatter and gather branching, the one-block small runs, a failed pass) and
then apply gates whose answer depends on the masks being exact: a stale mask
that called a varying bit constant would leave pairs unmerged, one that
called a constant bit varying only costs time."""

import numpy as np
import pytest

from oracle import OracleState
from paper_2105_01533_gb300 import sps
from paper_2105_01533_gb300 import workloads as W

from helpers import compare_states

pytestmark = pytest.mark.gpu

FORMS = [(2048, 0), (0, 0), (0, 1)]   # (small-run cap, branch form)


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2105_01533_gb300 import build as B
    B.build()
    sps.load_library()
    yield


def open_state(n, cap, small_cap, form, extra=()):
    st = sps.SparseState(n, cap)
    st.set_option(sps.SPS_OPT_SMALL_RUN_CAP, small_cap)
    st.set_option(sps.SPS_OPT_BRANCH_FORM, form)
    for opt, val in extra:
        st.set_option(opt, val)
    return st


def seeded_state(n, m, free, ones, seed):
    """m distinct labels random over the qubits in `free`; the qubits in
    `ones` are 1 in every label, every other qubit 0."""
    rng = np.random.default_rng(seed)
    base = sum(1 << q for q in ones)
    codes = rng.choice(1 << len(free), size=m, replace=False)
    labels = sorted(base | sum(((int(c) >> b) & 1) << q for b, q in enumerate(free))
                    for c in codes)
    lo = np.array([v & (2**64 - 1) for v in labels], np.uint64)
    hi = np.array([v >> 64 for v in labels], np.uint64)
    re, im = rng.normal(size=m), rng.normal(size=m)
    return hi, lo, re, im


def both_from(n, arrays, parts, eps, cap, small_cap, form, extra=()):
    st = open_state(n, cap, small_cap, form, extra)
    st.set_amplitudes(*arrays)
    orc = OracleState(n)
    orc.set(*arrays)
    for gates in parts:
        g = W.to_array(gates)
        st.apply(g, eps)
        orc.apply(g, eps=eps)
    got = st.get_amplitudes()
    st.close()
    return got, orc.get()


@pytest.mark.parametrize("small_cap,form", FORMS)
@pytest.mark.parametrize("n", [40, 100])
def test_branch_on_constant_and_varying_bits(n, small_cap, form):
    free = [0, 1, 2, 4, 5, 6, 8, 10, 11, 12, 13]
    arrays = seeded_state(n, 1500, free, [3, n - 2], seed=n)
    parts = [
        [W.H(3)],                      # constant 1: pure doubling
        [W.H(0)],                      # varying: most entries pair
        [W.H(n - 1), W.Ry(7, 0.4)],    # constant 0, twice
        [W.Givens(20, 3, 0.9)],        # bit 20 constant, bit 3 varying
        [W.H(3)],
        [W.CX(0, n - 2), W.H(n - 2)],  # a permutation makes a constant bit vary
        [W.Givens(n - 1, 7, 0.3, 1)],
        [W.Givens(30, 31, 0.7)],       # both constant 0: inactive everywhere
    ]
    got, want = both_from(n, arrays, parts, 1e-14, 1 << 16, small_cap, form)
    compare_states(got, want, 1e-14)


@pytest.mark.parametrize("small_cap,form", FORMS)
def test_masks_follow_fused_passes(small_cap, form):
    """Long permutation runs (bit-sliced and direct) move constant bits around;
    each branching gate after them must see the moved masks."""
    n = 64
    rng = W.SplitMix64(11)
    region = list(range(0, 64, 4))           # labels stay within these 16 qubits
    arrays = seeded_state(n, 3000, [region[i] for i in (0, 2, 3, 4, 5, 7, 8, 10, 11, 12, 13, 15)],
                          [region[1], region[9]], seed=4)
    parts = []
    for _ in range(6):
        perm = []
        for _ in range(40):
            q = [region[i] for i in rng.distinct(16, 3)]
            kind = rng.below(3)
            if kind == 0:
                perm.append(W.X(q[0]))
            elif kind == 1:
                perm.append(W.CX(q[0], q[1]))
            else:
                perm.append(W.CCX(q[0], q[1], q[2]))
        perm.append(W.T(region[rng.below(16)]))
        parts.append(perm)
        parts.append([W.H(region[rng.below(16)]), W.Ry(region[rng.below(16)], rng.angle())])
    for extra in ([], [(sps.SPS_OPT_BITSLICE_MIN_NNZ, 0), (sps.SPS_OPT_BITSLICE_MIN_OPS, 8)]):
        got, want = both_from(n, arrays, parts, 1e-14, 1 << 17, small_cap, form, extra)
        compare_states(got, want, 1e-14)


def test_form_switch_and_reset_keep_masks_exact():
    n = 50
    st = open_state(n, 1 << 15, 0, 1)
    orc = OracleState(n)
    seq = [
        (1, [W.H(0), W.H(1), W.CX(1, 30)]),
        (0, [W.H(30), W.H(31)]),                # gather after scatter
        (1, [W.H(31), W.X(40), W.H(40)]),       # scatter after gather
        (0, [W.H(40), W.Givens(0, 45, 1.1)]),
    ]
    for form, gates in seq:
        st.set_option(sps.SPS_OPT_BRANCH_FORM, form)
        g = W.to_array(gates)
        st.apply(g, 1e-14)
        orc.apply(g, eps=1e-14)
    compare_states(st.get_amplitudes(), orc.get(), 1e-14)
    st.reset()
    orc = OracleState(n)
    g = W.to_array([W.H(4), W.H(4), W.H(5)])
    st.apply(g, 1e-14)
    orc.apply(g, eps=1e-14)
    compare_states(st.get_amplitudes(), orc.get(), 1e-14)
    st.close()


@pytest.mark.parametrize("small_cap,form", FORMS)
def test_masks_after_capacity_failure(small_cap, form):
    n = 30
    st = open_state(n, 64, small_cap, form)
    orc = OracleState(n)
    good = W.to_array([W.H(q) for q in range(6)] + [W.CX(0, 10)])
    st.apply(good, 0.0)
    orc.apply(good, eps=0.0)
    st.apply(W.to_array([W.H(20)]), 0.0)   # 128 entries > 64
    with pytest.raises(sps.SpsError) as e:
        st.sync()
    assert e.value.status == sps.SPS_ERR_CAPACITY
    # the failed pass left the state (and so its masks) as they were
    more = W.to_array([W.CX(0, 10), W.H(0)])
    st.apply(more, 0.0)
    orc.apply(more, eps=0.0)
    compare_states(st.get_amplitudes(), orc.get(), 0.0)
    st.close()


@pytest.mark.parametrize("form", [0, 1])
def test_fresh_qubit_doubling_closed_form(form):
    """H on 20 fresh qubits of |0>: every pass is a pure doubling; the result
    is all 2^20 labels with amplitude 2^-10."""
    n, k = 100, 20
    qs = [3 * i + 1 for i in range(k)]
    st = open_state(n, 1 << k, 0, form)
    st.apply(W.to_array([W.H(q) for q in qs]), 1e-14)
    hi, lo, re, im = st.get_amplitudes()
    st.close()
    assert len(lo) == 1 << k
    idx = np.arange(1 << k, dtype=np.uint64)
    want = np.zeros(1 << k, dtype=np.uint64)
    for b, q in enumerate(qs):
        want |= ((idx >> np.uint64(b)) & np.uint64(1)) << np.uint64(q)
    assert not hi.any()
    np.testing.assert_array_equal(np.sort(lo), np.sort(want))
    np.testing.assert_allclose(re, np.full(1 << k, 2.0 ** -10), rtol=1e-13, atol=0)
    assert not im.any()
