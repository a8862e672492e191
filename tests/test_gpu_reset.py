"""sps_reset is enqueued lazily: an apply that starts with an expansion pass
builds its outputs from |0...0> itself, and every other use of the state
enqueues the reset first. The state, the update count, the status and the
failure behaviour must be those of an eager reset."""

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


def oracle(n, gates, eps=1e-14):
    orc = OracleState(n)
    orc.apply(W.to_array(gates), eps=eps)
    return orc.get()


def test_reset_then_expansion_is_one_launch_and_counts_from_zero():
    n = 40
    st = sps.SparseState(n, 1 << 14)
    g0 = [W.H(q) for q in range(6)] + [W.CX(0, 20), W.T(1)]
    st.apply(W.to_array(g0), 1e-14)
    st.sync()
    gates = [W.H(q) for q in range(3, 15)] + [W.CX(3, 30), W.P(4, 0.7, 5), W.X(31)]
    for _ in range(3):
        st.reset()
        c0 = st.counters().kernel_launches
        st.apply(W.to_array(gates), 1e-14)
        launches = st.counters().kernel_launches - c0
        compare_states(st.get_amplitudes(), oracle(n, gates), 1e-14)
        assert st.updates() == (1 << 12) - 1 + 3 * (1 << 12)
        assert launches == 1
    st.close()


def test_reset_then_other_uses_see_the_reset_state():
    n = 30
    st = sps.SparseState(n, 1 << 10)
    st.apply(W.to_array([W.H(0), W.H(1), W.X(7)]), 0.0)
    st.sync()
    st.reset()
    assert st.nnz() == 1
    hi, lo, re, im = st.get_amplitudes()
    assert lo.tolist() == [0] and re.tolist() == [1.0] and im.tolist() == [0.0]
    st.apply(W.to_array([W.H(0)]), 0.0)
    st.reset()
    assert st.probability((1, 0), (0, 0)) == 1.0
    st.apply(W.to_array([W.H(2)]), 0.0)
    st.reset()
    assert st.measure(3, 0.5) == (0, 1.0)
    st.reset()
    st.reset()
    st.apply(W.to_array([W.X(4), W.H(5)]), 0.0)       # starts with a fused pass
    compare_states(st.get_amplitudes(), oracle(n, [W.X(4), W.H(5)], 0.0), 0.0)
    assert st.updates() == 1 + 1
    st.close()


def test_reset_clears_a_failure_and_a_failing_expansion_leaves_the_reset_state():
    n = 30
    st = sps.SparseState(n, 100)
    st.apply(W.to_array([W.H(q) for q in range(5)]), 0.0)        # 32 entries
    st.apply(W.to_array([W.H(q) for q in range(10, 13)]), 0.0)   # 256 > 100: fails
    st.reset()                                                   # (no sync in between)
    st.apply(W.to_array([W.H(q) for q in range(6)]), 0.0)        # 64 entries
    compare_states(st.get_amplitudes(), oracle(n, [W.H(q) for q in range(6)], 0.0), 0.0)
    st.reset()
    st.apply(W.to_array([W.H(q) for q in range(8)] + [W.T(0)]), 0.0)   # 256 > 100
    with pytest.raises(sps.SpsError) as e:
        st.sync()
    assert e.value.status == sps.SPS_ERR_CAPACITY and e.value.failed_gate == 0
    hi, lo, re, im = st.get_amplitudes()
    assert lo.tolist() == [0] and re.tolist() == [1.0] and im.tolist() == [0.0]
    st.apply(W.to_array([W.H(1), W.CX(1, 2)]), 0.0)             # usable afterwards
    compare_states(st.get_amplitudes(), oracle(n, [W.H(1), W.CX(1, 2)], 0.0), 0.0)
    st.close()
