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
