"""Gate commuting queues (sps_commute, host only): the rewritten stream must
compute the same state as the caller's, which the CPU oracle checks gate by
gate on both streams, and the identities of the queue rules must show in the
output (cancelled and merged gates, gates turned into their conjugates)."""

import numpy as np
import pytest

from oracle import OracleState
from paper_2105_01533_gb300 import sps
from paper_2105_01533_gb300 import workloads as W

from helpers import compare_states


def ops(g):
    return [(int(r["op"]), int(r["t0"]), int(r["cmask"][0]), round(float(r["theta"]), 12))
            for r in g]


def test_queue_identities():
    n = 6
    c = lambda *gs: ops(sps.sps_commute(W.to_array(list(gs)), n))   # noqa: E731
    assert c(W.H(0), W.H(0)) == []                                   # H H = 1
    assert c(W.H(0), W.X(0), W.H(0)) == [(W.OP_Z, 0, 0, 0.0)]       # H X H = Z
    assert c(W.H(0), W.Z(0), W.H(0)) == [(W.OP_X, 0, 0, 0.0)]       # H Z H = X
    assert c(W.H(0), W.Ry(0, 0.3), W.H(0)) == [(W.OP_RY, 0, 0, -0.3)]
    assert c(W.Rx(1, 0.2), W.Rx(1, 0.5)) == [(W.OP_RX, 1, 0, 0.7)]
    assert c(W.Ry(2, 0.4), W.X(2)) == [(W.OP_X, 2, 0, 0.0), (W.OP_RY, 2, 0, -0.4)]
    assert c(W.Rx(2, 0.4), W.Z(2)) == [(W.OP_Z, 2, 0, 0.0), (W.OP_RX, 2, 0, -0.4)]
    assert c(W.Rx(3, 0.4), W.CX(1, 3)) == [(W.OP_X, 3, 2, 0.0), (W.OP_RX, 3, 0, 0.4)]
    # C-X through H on its target becomes C-Z; the H pair cancels
    assert c(W.H(0), W.CX(1, 0), W.H(0)) == [(W.OP_Z, 0, 2, 0.0)]
    # a T on a qubit with a queued H forces the H out first
    assert c(W.H(0), W.T(0)) == [(W.OP_H, 0, 0, 0.0), (W.OP_T, 0, 0, 0.0)]
    # a control with a queued H forces it out; the phase/permutation queue goes first
    assert c(W.X(4), W.H(1), W.CX(1, 2)) == [(W.OP_X, 4, 0, 0.0), (W.OP_H, 1, 0, 0.0),
                                            (W.OP_X, 2, 2, 0.0)]


def random_mix(seed, n, count):
    rng = W.SplitMix64(seed)
    g = []
    for _ in range(count):
        q = rng.distinct(n, 3)
        k = rng.below(12)
        if k < 3:
            g.append(W.H(q[0]))
        elif k == 3:
            g.append(W.Rx(q[0], rng.angle()))
        elif k == 4:
            g.append(W.Ry(q[0], rng.angle()))
        elif k == 5:
            g.append(W.X(q[0]))
        elif k == 6:
            g.append(W.CX(q[1], q[0]))
        elif k == 7:
            g.append(W.Z(q[0], *([q[1]] if rng.below(2) else [])))
        elif k == 8:
            g.append(W.T(q[0]))
        elif k == 9:
            g.append(W.CP(q[1], q[0], rng.angle()))
        elif k == 10:
            g.append(W.Givens(q[0], q[1], rng.angle()))
        else:
            g.append(W.Ry(q[0], rng.angle(), q[2]))
    return W.to_array(g)


@pytest.mark.parametrize("seed", range(6))
def test_rewritten_stream_computes_the_same_state(seed):
    n = 10
    g = random_mix(seed, n, 120)
    r = sps.sps_commute(g, n)
    a = OracleState(n)
    a.apply(g)
    b = OracleState(n)
    b.apply(r)
    compare_states(b.get(), a.get(), 0.0)
    branch = lambda x: int(np.isin(x["op"], [W.OP_H, W.OP_RX, W.OP_RY, W.OP_GIVENS]).sum())  # noqa: E731
    assert branch(r) <= branch(g) and len(r) <= len(g)


def test_bad_record_is_reported():
    g = W.to_array([W.H(0), W.X(9)])
    with pytest.raises(sps.SpsError) as e:
        sps.sps_commute(g, 5)
    assert e.value.status == sps.SPS_ERR_ARG and e.value.failed_gate == 1


def test_fig1_walkthrough():
    """Sec. 3.3, Fig. 1, replayed on 8 qubits. Starting queues (black in the
    figure): phase/permutation queue CNOT(0->3), Z(2), CZ(1,4); H queued on
    qubits 1..4; Rx(0.75) on qubit 4; Ry(0.6) on qubit 1; Rx(-pi/4) on qubit 6.
    Steps: (a) H on qubit 0 only sets its H queue; (b) H on qubit 1 flips the
    queued Ry angle (H Ry(t) = Ry(-t) H) and cancels the queued H (H H = 1);
    (c) X on qubit 2 adds Z(2) to the phase/permutation queue (X H = H Z);
    (d) CCNOT(3,4 -> 5) cannot pass the queued Rx on qubit 4 nor the H gates:
    the whole phase/permutation queue is executed, then H on 3 and 4, then
    Rx(0.75), and the CCNOT waits in the emptied queue; (e) the Rx(-pi/4) on
    qubit 6 is never executed by these steps. Each prefix is rewritten by
    sps_commute (which emits whatever is still queued at the end: the
    phase/permutation queue, then per qubit H, Rx, Ry) and must compute the
    same state as the original stream."""
    n = 8
    start = [W.CX(0, 3), W.Z(2), W.CZ(1, 4), W.H(1), W.H(2), W.H(3), W.H(4),
             W.Rx(4, 0.75), W.Ry(1, 0.6), W.Rx(6, -np.pi / 4)]
    steps = [W.H(0), W.H(1), W.X(2), W.X(5, 3, 4)]
    CX = (W.OP_X, 3, 1 << 0, 0.0)
    Z2 = (W.OP_Z, 2, 0, 0.0)
    CZ = (W.OP_Z, 4, 1 << 1, 0.0)
    H = lambda q: (W.OP_H, q, 0, 0.0)                         # noqa: E731
    RX4 = (W.OP_RX, 4, 0, 0.75)
    RX6 = (W.OP_RX, 6, 0, round(-np.pi / 4, 12))
    want = {
        "start": [CX, Z2, CZ, H(1), (W.OP_RY, 1, 0, 0.6), H(2), H(3), H(4), RX4, RX6],
        "a": [CX, Z2, CZ, H(0), H(1), (W.OP_RY, 1, 0, 0.6), H(2), H(3), H(4), RX4, RX6],
        "b": [CX, Z2, CZ, H(0), (W.OP_RY, 1, 0, -0.6), H(2), H(3), H(4), RX4, RX6],
        "c": [CX, Z2, CZ, Z2, H(0), (W.OP_RY, 1, 0, -0.6), H(2), H(3), H(4), RX4, RX6],
        "d": [CX, Z2, CZ, Z2, H(3), H(4), RX4, (W.OP_X, 5, (1 << 3) | (1 << 4), 0.0),
              H(0), (W.OP_RY, 1, 0, -0.6), H(2), RX6],
    }
    for k, name in enumerate(["start", "a", "b", "c", "d"]):
        g = W.to_array(start + steps[:k])
        r = sps.sps_commute(g, n)
        assert ops(r) == want[name], name
        a = OracleState(n)
        a.apply(g)
        b = OracleState(n)
        b.apply(r)
        compare_states(b.get(), a.get(), 0.0)
    # (d): what ran before the CCNOT is exactly the caption's flush, and (e)
    # the Rx(-pi/4) on qubit 6 only comes out at the very end
    d = want["d"]
    assert d.index((W.OP_X, 5, (1 << 3) | (1 << 4), 0.0)) == 7
    assert d[-1] == RX6
