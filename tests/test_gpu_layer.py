"""GPU parity of layer passes (SPS_OPT_LAYER_GATES): up to 4 consecutive
branching gates on disjoint qubits in one gather pass. The group writer runs
the gates in order with the per-gate arithmetic and pruning, so the result
equals the oracle's gate-by-gate result bit for bit, and so does the update
count of one pass per gate."""

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


def run(n, gates, eps, cap, layer, opts=(), init=None):
    st = sps.SparseState(n, cap)
    st.set_option(sps.SPS_OPT_SMALL_RUN_CAP, 0)      # whole-GPU passes
    st.set_option(sps.SPS_OPT_LAYER_GATES, layer)
    for o, v in opts:
        st.set_option(o, v)
    if init is not None:
        st.set_amplitudes(*init)
    st.apply(gates, eps)
    got = st.get_amplitudes()
    c = st.counters()
    upd = st.updates()
    st.close()
    return got, c, upd


def oracle(n, gates, eps, init=None):
    orc = OracleState(n)
    if init is not None:
        orc.set(*init)
    orc.apply(gates, eps=eps, mode=1)
    return orc.get()


def same(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("n", [32, 64, 90])
def test_givens_layers_bit_identical(n):
    g = W.givens_workload(seed=5, nqubits=n, modes=3, layers=6) if n == 64 else None
    if g is None:
        rng = W.SplitMix64(n)
        recs = [W.X(q) for q in range(3)]
        for _ in range(6):
            perm = rng.distinct(n, n - n % 2)
            recs += [W.Givens(perm[2 * i], perm[2 * i + 1], rng.angle()) for i in range(len(perm) // 2)]
            recs += [W.CZ(*rng.distinct(n, 2)) for _ in range(8)]
        g = W.to_array(recs)
    want = oracle(n, g, 1e-14)
    got, c, upd = run(n, g, 1e-14, 1 << 17, 4)
    same(got, want)
    got1, c1, upd1 = run(n, g, 1e-14, 1 << 17, 1)
    same(got1, want)
    assert upd == upd1                       # the same nonzeros before every gate
    assert c.branch_passes < c1.branch_passes


@pytest.mark.parametrize("seed", range(4))
def test_random_branching_layers(seed):
    """H, Rx, Ry and Givens with controls; runs of disjoint gates form layers,
    overlapping ones end them; fresh qubits (no partners) mix with occupied ones."""
    n = 40
    rng = W.SplitMix64(100 + seed)
    recs = [W.H(q) for q in rng.distinct(12, 6)]
    for _ in range(60):
        q = [x for x in rng.distinct(16, 3)]
        k = rng.below(5)
        if k == 0:
            recs.append(W.H(q[0]))
        elif k == 1:
            recs.append(W.Rx(q[0], rng.angle(), *([q[2]] if rng.below(3) == 0 else [])))
        elif k == 2:
            recs.append(W.Ry(q[0], rng.angle()))
        elif k == 3:
            recs.append(W.Givens(q[0], q[1], rng.angle(), *([q[2]] if rng.below(3) == 0 else [])))
        else:
            recs.append(W.CX(q[0], q[1]))
    g = W.to_array(recs)
    for eps in (0.0, 1e-14, 1e-3):
        want = oracle(n, g, eps)
        for opts in ([], [(sps.SPS_OPT_EXPAND, 0)]):
            got, _, upd = run(n, g, eps, 1 << 16, 4, opts)
            got1, _, upd1 = run(n, g, eps, 1 << 16, 1, opts)
            same(got, got1)                     # layers = one pass per gate, bit for bit
            assert upd == upd1
            if opts:
                same(got, want)                 # and gate by gate = the oracle
            else:                               # expansion passes round their products
                compare_states(got, want, eps)


def test_layer_capacity_failure_names_its_first_gate():
    n = 30
    st = sps.SparseState(n, 100)
    st.set_option(sps.SPS_OPT_SMALL_RUN_CAP, 0)
    st.set_option(sps.SPS_OPT_EXPAND, 0)
    st.apply(W.to_array([W.H(q) for q in range(5)]), 0.0)            # 32 entries
    before = st.get_amplitudes()
    st.apply(W.to_array([W.X(20), W.H(10), W.H(11), W.H(12), W.Z(3)]), 0.0)   # 256 > 100
    with pytest.raises(sps.SpsError) as e:
        st.sync()
    assert e.value.status == sps.SPS_ERR_CAPACITY and e.value.failed_gate == 1
    hi, lo, re, im = st.get_amplitudes()
    np.testing.assert_array_equal(np.sort(before[1] ^ np.uint64(1 << 20)), lo)
    st.close()
