"""GPU tests of the batched executor: every circuit of a batch against the CPU
oracle and against the plain path (alone vs in the batch), resumption with a
bounded number of passes per launch, failure isolation, configurations and
the autotuner."""

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


def small_batch(count=24, seed0=500):
    """Circuits of the batched mix at reduced depth so the oracle stays fast;
    caps 2^8..2^13 straddle the shared-memory cap, qubits 20..100."""
    return W.batched_workload_fast(count, first_seed=seed0, depth=(150, 400), log2_cap=(8, 13))


def oracle_result(c):
    o = OracleState(c.nqubits)
    o.apply(c.gates, eps=EPS)
    return o.get()


def plain_result(c):
    st = sps.SparseState(c.nqubits, c.cap)
    st.apply(c.gates, EPS)
    r = st.get_amplitudes()
    st.close()
    return r


@pytest.mark.parametrize("cfg", [None, (512, 2, 1024), (1024, 1, 2048), (256, 2, 0)])
def test_batch_matches_oracle_and_plain(cfg):
    circs = small_batch()
    b = sps.Batch()
    for c in circs:
        b.add(c.nqubits, c.cap, c.gates, EPS)
    if cfg:
        b.set_config(*cfg)
    b.run()
    assert b.sync() == 0
    for i, c in enumerate(circs):
        st = b.status(i)
        assert st["status"] == 0 and st["finished"]
        got = b.get_amplitudes(i)
        compare_states(got, oracle_result(c), EPS)
        compare_states(got, plain_result(c), EPS)
    b.close()


def test_batch_resume_with_bounded_passes():
    circs = small_batch(12, seed0=900)
    b = sps.Batch()
    for c in circs:
        b.add(c.nqubits, c.cap, c.gates, EPS)
    rounds = 0
    while True:
        b.run(max_passes=2)
        rounds += 1
        if b.sync() == 0:
            break
        assert rounds < 10000
    assert rounds > 2
    for i, c in enumerate(circs):
        compare_states(b.get_amplitudes(i), oracle_result(c), EPS)
    # reset and run again in one launch: same results
    b.reset()
    b.run()
    b.sync()
    for i, c in enumerate(circs):
        compare_states(b.get_amplitudes(i), oracle_result(c), EPS)
    b.close()


def test_batch_failure_is_isolated():
    good = small_batch(6, seed0=1300)
    b = sps.Batch()
    for c in good[:3]:
        b.add(c.nqubits, c.cap, c.gates, EPS)
    bad = W.to_array([W.H(q) for q in range(10)] + [W.X(3)])   # 1024 entries, cap 100
    ib = b.add(40, 100, bad, EPS)
    for c in good[3:]:
        b.add(c.nqubits, c.cap, c.gates, EPS)
    b.run()
    b.sync()
    st = b.status(ib)
    assert st["status"] == sps.SPS_ERR_CAPACITY and st["failed_gate"] == 6 and st["nnz"] == 64
    for k, c in enumerate(good):
        i = k if k < 3 else k + 1
        assert b.status(i)["status"] == 0
        compare_states(b.get_amplitudes(i), oracle_result(c), EPS)
    with pytest.raises(sps.SpsError):
        b.add(10, 16, W.to_array([W.X(12)]))
    b.close()


def test_batch_rejects_bad_records():
    b = sps.Batch()
    with pytest.raises(sps.SpsError) as e:
        b.add(10, 64, W.to_array([W.H(0), W.X(3, 3)]))
    assert e.value.failed_gate == 1
    b.close()


def test_batch_tune_keeps_results():
    circs = small_batch(16, seed0=2000)
    b = sps.Batch()
    for c in circs:
        b.add(c.nqubits, c.cap, c.gates, EPS)
    best = b.tune(repeats=1)
    assert best["threads"] in (256, 512, 1024) and best["ms"] > 0
    b.run()
    b.sync()
    for i, c in enumerate(circs):
        compare_states(b.get_amplitudes(i), oracle_result(c), EPS)
    b.close()


def identical(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_graph_step_equals_reset_and_run():
    """One step captured as a CUDA graph (reset, then the persistent launch),
    replayed several times, with a bounded pass count and after a change of
    launch configuration: each replay gives what sps_batch_reset +
    sps_batch_run give, bit for bit, and one launch per step is counted."""
    circs = small_batch(20, seed0=2600)
    ref = sps.Batch()
    for c in circs:
        ref.add(c.nqubits, c.cap, c.gates, EPS)
    ref.run()
    ref.sync()
    want = [ref.get_amplitudes(i) for i in range(len(circs))]
    ref.close()
    b = sps.Batch()
    for c in circs:
        b.add(c.nqubits, c.cap, c.gates, EPS)
    for cfg in (None, (256, 2, 0)):
        if cfg:
            b.set_config(*cfg)
        for _ in range(3):
            l0 = b.launches()
            b.run_graph()
            assert b.sync() == 0
            assert b.launches() == l0 + 1
            for i in range(len(circs)):
                identical(b.get_amplitudes(i), want[i])
    # a bounded step: every circuit reset and advanced by two passes, as reset + run(2)
    b.run_graph(max_passes=2)
    b.sync()
    two = [b.get_amplitudes(i) for i in range(len(circs))]
    b.reset()
    b.run(max_passes=2)
    b.sync()
    for i in range(len(circs)):
        identical(b.get_amplitudes(i), two[i])
    b.close()
