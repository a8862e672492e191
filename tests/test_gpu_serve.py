"""GPU tests of the serving loop: results in a mixed, continuously batched
stream equal the same circuits applied alone; admission follows arrival order
under the memory budget; a failing request does not disturb the others; the
per-tick pass limit does not change results; update counters."""

import math

import numpy as np
import pytest

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


def request_mix():
    """(nqubits, capacity, gates): random mixes, adders (small and large) and
    Givens circuits."""
    reqs = []
    for c in W.batched_workload_fast(10, first_seed=3000, depth=(100, 300), log2_cap=(8, 12)):
        reqs.append((c.nqubits, c.cap, c.gates))
    for w in (6, 10, 17):
        wl = W.adder_workload(seed=w, nbits=32, width=w, n_cp=8)
        reqs.append((wl.layout.nqubits, 1 << w, wl.gates))
    for n, k in ((24, 3), (40, 2)):
        reqs.append((n, math.comb(n, k), W.givens_workload(seed=n, nqubits=n, modes=k, layers=4)))
    return reqs


def alone(nq, cap, gates):
    st = sps.SparseState(nq, cap)
    st.apply(gates, EPS)
    r = st.get_amplitudes()
    st.close()
    return r


@pytest.mark.parametrize("passes_per_tick", [2, 0])
def test_served_mix_equals_alone(passes_per_tick):
    reqs = request_mix()
    srv = sps.Server(mem_budget_bytes=8 << 30, max_active=64, passes_per_tick=passes_per_tick)
    ids = []
    # arrivals interleaved with ticks: three requests before each tick
    pending = list(range(len(reqs)))
    while pending or any(srv.poll(i)["state"] != 2 for i in ids):
        for _ in range(3):
            if pending:
                k = pending.pop(0)
                ids.append(srv.submit(*reqs[k][:2], reqs[k][2], EPS))
        srv.tick()
    assert any(srv.poll(i)["large"] for i in ids)
    for i, (nq, cap, gates) in zip(ids, reqs):
        info = srv.poll(i)
        assert info["state"] == 2 and info["status"] == 0 and info["updates"] > 0
        compare_states(srv.result(i), alone(nq, cap, gates), EPS)
    srv.close()


def test_completed_lists_each_request_once():
    """sps_server_completed reports the requests that finished in the last tick:
    over the whole run every request appears exactly once, after it is done."""
    reqs = [(20 + 3 * k, 256, W.to_array([W.H(q) for q in range(k % 5 + 1)] + [W.X(19)]))
            for k in range(12)]
    srv = sps.Server(mem_budget_bytes=1 << 26, max_active=16, passes_per_tick=2)
    ids = [srv.submit(nq, cap, g, EPS) for nq, cap, g in reqs]
    seen = []
    for _ in range(10000):
        srv.tick()
        done_now = srv.completed()
        for i in done_now:
            assert srv.poll(i)["state"] == 2
        seen += done_now
        if all(srv.poll(i)["state"] == 2 for i in ids):
            break
    assert sorted(seen) == sorted(ids)
    srv.close()


def test_admission_follows_budget_and_order():
    reqs = request_mix()[:10]          # small random mixes
    need = max(64 * cap for _, cap, _ in reqs) + 64 * 1024
    budget = 2 * need + 1
    srv = sps.Server(mem_budget_bytes=budget, max_active=64, passes_per_tick=1)
    ids = [srv.submit(nq, cap, g, EPS) for nq, cap, g in reqs]
    saw_pending = False
    ticks = 0
    while any(srv.poll(i)["state"] != 2 for i in ids):
        active, pending, done = srv.tick()
        assert 0 < srv.stats()["bytes_in_use"] <= budget or active == 0
        saw_pending = saw_pending or pending > 0
        ticks += 1
        assert ticks < 100000
    assert saw_pending
    admits = [srv.poll(i)["admit_tick"] for i in ids]
    assert admits == sorted(admits)            # first come, first admitted
    for i, (nq, cap, g) in zip(ids, reqs):
        compare_states(srv.result(i), alone(nq, cap, g), EPS)
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()


def test_failing_request_is_isolated():
    reqs = request_mix()[:4]
    srv = sps.Server(mem_budget_bytes=1 << 30, max_active=16, passes_per_tick=3)
    bad = W.to_array([W.H(q) for q in range(9)] + [W.Z(2)])
    ids = [srv.submit(nq, cap, g, EPS) for nq, cap, g in reqs[:2]]
    ib = srv.submit(30, 100, bad, EPS)
    ids += [srv.submit(nq, cap, g, EPS) for nq, cap, g in reqs[2:]]
    while any(srv.poll(i)["state"] != 2 for i in ids + [ib]):
        srv.tick()
    info = srv.poll(ib)
    assert info["status"] == sps.SPS_ERR_CAPACITY and info["failed_gate"] == 6
    assert info["nnz"] == 64
    for i, (nq, cap, g) in zip(ids, reqs):
        assert srv.poll(i)["status"] == 0
        compare_states(srv.result(i), alone(nq, cap, g), EPS)
    wide = W.to_array([W.H(q) for q in range(30)])   # projected peak 2^30: capped at 10^9
    with pytest.raises(sps.SpsError):
        srv.submit(30, 10 ** 9, wide, EPS)   # can never fit the budget
    srv.submit(30, 10 ** 9, bad, EPS)        # charged for its peak, 2^9: fits
    srv.close()


def test_state_update_counter():
    st = sps.SparseState(20, 64)
    st.apply(W.to_array([W.H(0), W.H(1), W.H(2), W.X(3), W.Z(4)]), 0.0)
    assert st.updates() == 1 + 2 + 4 + 8 + 8
    st.reset()
    assert st.updates() == 0
    st.set_option(sps.SPS_OPT_SMALL_RUN_CAP, 0)
    st.apply(W.to_array([W.H(0), W.H(1), W.H(2), W.X(3), W.Z(4)]), 0.0)
    assert st.updates() == 23
    st.close()


def test_admission_charges_the_projected_peak():
    """A request declared with capacity 2^26 whose circuit can reach only 2^8
    (or 2^20) nonzeros is charged and sized for that peak: it fits a 256 MiB
    budget that the declared capacity (6 GB at 96 B per entry) would not, the
    small one takes the batched route, and both equal sps_apply alone. A
    2^22-nonzero adder runs beside small requests in the same ticks."""
    small = W.to_array([W.H(q) for q in range(8)] + [W.CX(0, 9), W.T(3), W.Ry(9, 0.4)])
    ad20 = W.adder_workload(seed=20, nbits=32, width=20, n_cp=4)
    srv = sps.Server(mem_budget_bytes=256 << 20, max_active=16, passes_per_tick=0)
    a = srv.submit(40, 1 << 26, small, EPS)
    b = srv.submit(ad20.layout.nqubits, 1 << 26, ad20.gates, EPS)
    while any(srv.poll(i)["state"] != 2 for i in (a, b)):
        srv.tick()
        assert srv.stats()["bytes_in_use"] <= 256 << 20
    ia, ib = srv.poll(a), srv.poll(b)
    assert ia["status"] == 0 and ib["status"] == 0
    assert ia["large"] == 0 and ib["large"] == 1
    compare_states(srv.result(a), alone(40, 1 << 26, small), EPS)
    compare_states(srv.result(b), alone(ad20.layout.nqubits, 1 << 20, ad20.gates), EPS)
    srv.close()
    # a large request among small ones, served in the same ticks
    reqs = request_mix()[:8]
    ad22 = W.adder_workload(seed=22, nbits=32, width=22, n_cp=4)
    srv = sps.Server(mem_budget_bytes=8 << 30, max_active=64, passes_per_tick=4)
    big = srv.submit(ad22.layout.nqubits, 1 << 22, ad22.gates, EPS)
    ids = [srv.submit(nq, cap, g, EPS) for nq, cap, g in reqs]
    overlap = False
    while any(srv.poll(i)["state"] != 2 for i in ids + [big]):
        srv.tick()
        if srv.poll(big)["state"] == 1 and any(srv.poll(i)["state"] == 1 for i in ids):
            overlap = True   # small requests advanced in the ticks the large one did
    assert overlap and srv.poll(big)["large"] == 1
    compare_states(srv.result(big), alone(ad22.layout.nqubits, 1 << 22, ad22.gates), EPS)
    for i, (nq, cap, g) in zip(ids, reqs):
        compare_states(srv.result(i), alone(nq, cap, g), EPS)
    srv.close()
