"""GPU parity of measurement with collapse (sps_measure) against the oracle:
outcome, its probability and the collapsed state, on 64- and 128-bit labels,
followed by further gates (the measured qubit is then constant, which the
branching passes detect) and by further measurements."""

import math

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


def prepared(n, seed, cap=1 << 14):
    rng = W.SplitMix64(seed)
    qs = rng.distinct(n, 12)
    gates = [W.H(q) for q in qs[:8]] + [W.Ry(qs[8], rng.angle(), qs[0]), W.CX(qs[1], qs[9]),
             W.T(qs[2]), W.P(qs[3], rng.angle(), qs[4]), W.Givens(qs[5], qs[10], rng.angle()),
             W.Rx(qs[11], rng.angle(), qs[6])]
    g = W.to_array(gates)
    st = sps.SparseState(n, cap)
    st.apply(g, 1e-14)
    orc = OracleState(n)
    orc.apply(g, eps=1e-14)
    return st, orc, qs


@pytest.mark.parametrize("n,seed", [(20, 1), (64, 2), (100, 3), (127, 4)])
def test_measure_matches_oracle(n, seed):
    rng = np.random.default_rng(seed)
    st, orc, qs = prepared(n, seed)
    for step in range(6):
        q = qs[step] if step % 2 == 0 else int(rng.integers(n))
        p1 = orc.probability((1 << q if q < 64 else 0, 1 << (q - 64) if q >= 64 else 0),
                             (1 << q if q < 64 else 0, 1 << (q - 64) if q >= 64 else 0))
        total = orc.probability((0, 0), (0, 0))
        r = float(rng.random())
        if abs(r * total - p1) < 1e-9:          # a draw on the edge: either outcome is right
            r = (r + 0.25) % 1.0
        want = orc.measure(q, r)
        got = st.measure(q, r)
        assert got[0] == want[0] and abs(got[1] - want[1]) < 1e-12
        compare_states(st.get_amplitudes(), orc.get(), 1e-14)
        c = next(x for x in qs[step + 1:] + qs if x != q)
        g = W.to_array([W.H(q), W.CX(c, q), W.Ry(qs[(step + 3) % 12], 0.7)])
        st.apply(g, 1e-14)                      # the measured qubit is constant now
        orc.apply(g, eps=1e-14)
        compare_states(st.get_amplitudes(), orc.get(), 1e-14)
    st.close()


def test_bell_pair_and_async_outputs():
    import torch
    st = sps.SparseState(10, 64)
    st.apply(W.to_array([W.H(0), W.CX(0, 1)]), 0.0)
    pinned = torch.full((2,), float("nan"), dtype=torch.float64, pin_memory=True)
    dev = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    st.measure_async(0, 0.3, pinned.data_ptr())        # r < 1/2: outcome 1
    st.measure_async(1, 0.999, dev.data_ptr())         # certain now
    st.sync()
    torch.cuda.synchronize()
    assert pinned[0].item() == 1.0 and abs(pinned[1].item() - 0.5) < 1e-15
    assert dev[0].item() == 1.0 and abs(dev[1].item() - 1.0) < 1e-15
    hi, lo, re, im = st.get_amplitudes()
    assert lo.tolist() == [3] and abs(re[0] - 1.0) < 1e-15
    st.close()


@pytest.mark.parametrize("small_cap,form", [(2048, 0), (0, 0), (0, 1)])
def test_measure_between_passes_of_every_form(small_cap, form):
    n = 40
    st = sps.SparseState(n, 1 << 13)
    st.set_option(sps.SPS_OPT_SMALL_RUN_CAP, small_cap)
    st.set_option(sps.SPS_OPT_BRANCH_FORM, form)
    orc = OracleState(n)
    seq = [([W.H(q) for q in range(6)], (2, 0.2)),
           ([W.CX(0, 20), W.H(20), W.Givens(1, 21, 0.4)], (20, 0.8)),
           ([W.H(2), W.H(20), W.Ry(3, 1.1, 20)], (3, 0.45)),
           ([W.X(30), W.H(30)], (30, 0.1))]
    for gates, (q, r) in seq:
        g = W.to_array(gates)
        st.apply(g, 1e-14)
        orc.apply(g, eps=1e-14)
        want = orc.measure(q, r)
        got = st.measure(q, r)
        assert got[0] == want[0] and abs(got[1] - want[1]) < 1e-12
        compare_states(st.get_amplitudes(), orc.get(), 1e-14)
    st.close()


def test_measure_edge_cases_and_counts():
    st = sps.SparseState(30, 256)
    st.apply(W.to_array([W.H(0), W.H(1), W.H(2)]), 0.0)      # 8 entries
    u0 = st.updates()
    assert st.measure(9, 0.99) == (0, 1.0)                    # a constant qubit
    assert st.updates() == u0 + 8 and st.nnz() == 8
    hi, lo, re, im = st.get_amplitudes()
    np.testing.assert_allclose(re, np.full(8, 1 / math.sqrt(8)), rtol=1e-15)
    for q, r in ((30, 0.5), (0, 1.0), (0, -0.5), (0, float("nan"))):
        with pytest.raises(sps.SpsError) as e:
            st.measure(q, r)
        assert e.value.status == sps.SPS_ERR_ARG
    st.apply(W.to_array([W.H(3)]), 1.0)                       # |a| = 0.25 < 1: all pruned
    assert st.nnz() == 0
    assert st.measure(0, 0.5) == (0, 0.0)                     # empty stays empty
    assert st.nnz() == 0
    st.close()
