"""GPU tests of the plain path's autotuner (sps_tune): the chosen options
leave the results as the oracle gives them (bit for bit against the default
options where only shape options changed), the choice is recorded per size
class in the cache file and taken from there the next time without timing."""

import numpy as np
import pytest

from oracle import OracleState
from paper_2105_01533_gb300 import sps
from paper_2105_01533_gb300 import workloads as W

from helpers import compare_states

pytestmark = pytest.mark.gpu

EPS = 1e-14


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2105_01533_gb300 import build as B
    B.build()
    sps.load_library()
    yield


def run_default(nq, cap, gates):
    st = sps.SparseState(nq, cap)
    st.apply(gates, EPS)
    r = st.get_amplitudes()
    st.close()
    return r


@pytest.mark.parametrize("case", ["adder", "givens"])
def test_tuned_options_keep_results_and_cache(case, tmp_path):
    if case == "adder":
        wl = W.adder_workload(seed=4, nbits=32, width=14, n_cp=8)
        nq, cap, gates = wl.layout.nqubits, 1 << 14, wl.gates
    else:
        nq, cap = 24, 2048
        gates = W.givens_workload(seed=6, nqubits=nq, modes=3, layers=12)
    cache = str(tmp_path / "tune.txt")
    st = sps.SparseState(nq, cap)
    c = st.tune(gates, EPS, repeats=1, cache=cache)
    assert c["from_cache"] == 0 and c["ms"] > 0
    assert c["kw"] == (1 if nq <= 63 else 2)
    assert 2 ** c["log2peak"] >= min(cap, 2)
    st.apply(gates, EPS)            # the state was left reset, with the choice set
    got = st.get_amplitudes()
    st.close()
    o = OracleState(nq)
    o.apply(gates, eps=EPS)
    compare_states(got, o.get(), EPS)
    if c["max_fused_ops"] == 512:   # only shape options changed: the same bits
        ref = run_default(nq, cap, gates)
        for x, y in zip(got, ref):
            np.testing.assert_array_equal(x, y)
    lines = [l for l in open(cache).read().splitlines() if l.startswith("sps-tune")]
    assert len(lines) == 1
    # the next state of the class takes the recorded choice without timing
    st2 = sps.SparseState(nq, cap)
    c2 = st2.tune(gates, EPS, repeats=1, cache=cache)
    assert c2["from_cache"] == 1
    for k in ("load_factor_pct", "bitslice_groups", "fused_labels", "max_fused_ops", "log2peak"):
        assert c2[k] == c[k]
    st2.apply(gates, EPS)
    compare_states(st2.get_amplitudes(), got, EPS)
    st2.close()
    assert len([l for l in open(cache).read().splitlines() if l.startswith("sps-tune")]) == 1
