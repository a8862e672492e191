"""GPU parity of a registered readout summed by the compiled expansion launch
(sps_set_readout): the probability of a condition on the output labels,
formed as the launch stores the outputs, then answered without a readout
launch. Checked against the CPU oracle, against the readout kernel on the
same state, and for staleness: any call that changes the state afterwards
makes the next readout launch the kernel again."""

import numpy as np
import pytest

from oracle import OracleState
from paper_2105_01533_gb300 import sps
from paper_2105_01533_gb300 import workloads as W

from test_gpu_bs_expand import FORCE, run_gates

pytestmark = pytest.mark.gpu

EPS = 1e-14
M64 = (1 << 64) - 1


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2105_01533_gb300 import build as B
    B.build()
    sps.load_library()
    yield


def conditions(n, gates, seed):
    """Conditions on bits the circuit drives (the expansion's and the run's
    qubits), on bits it never touches (0 in every label), a wanted bit outside
    the mask, a wanted untouched bit, the empty mask and, above 64 qubits,
    high-word bits."""
    rng = W.SplitMix64(seed)
    touched = sorted({int(g["t0"]) for g in gates})
    untouched = [q for q in range(n) if q not in touched]

    def cond(qs, want):
        m, v = [0, 0], [0, 0]
        for q, b in zip(qs, want):
            m[q >> 6] |= 1 << (q & 63)
            if b:
                v[q >> 6] |= 1 << (q & 63)
        return m, v

    out = []
    for k in (1, 2, 3, 5):
        qs = [touched[i] for i in rng.distinct(len(touched), min(k, len(touched)))]
        out.append(cond(qs, [rng.below(2) for _ in qs]))
    if untouched:
        q = untouched[rng.below(len(untouched))]
        out.append(cond([touched[0], q], [1, 0]))   # an untouched bit wanted 0
        out.append(cond([touched[0], q], [0, 1]))   # wanted 1: nothing matches
    m, v = cond([touched[1]], [1])
    v[touched[2] >> 6] |= 1 << (touched[2] & 63)
    out.append((m, v))                               # a wanted bit outside the mask
    out.append(([0, 0], [0, 0]))                     # every label matches
    hi = [q for q in touched if q >= 64]
    if len(hi) >= 2:
        out.append(cond(hi[:2], [1, 0]))
        out.append(cond([hi[0], touched[0]], [0, 1]))
    return out


def fused_record(st):
    return [r for r in st.profile_read() if r["kind"] == 7 and r["flags"] & 16]


@pytest.mark.parametrize("n,d,kinds,seed", [
    (20, 10, ["h"], 1), (40, 12, ["h", "h", "ry"], 2), (67, 11, ["rx", "h", "h", "h", "ry"], 3),
    (100, 9, ["ry", "h", "h"], 4), (127, 13, ["h"], 5), (33, 3, ["h"], 6)])
def test_fused_readout_matches_oracle_and_kernel(n, d, kinds, seed):
    import torch
    gates = run_gates(seed, n, d, 150, kinds)
    orc = OracleState(n)
    orc.apply(gates, eps=EPS)
    plain = sps.SparseState(n, 1 << (d + 1))
    for o, v in FORCE:
        plain.set_option(o, v)
    plain.reset()
    plain.apply(gates, EPS)
    st = sps.SparseState(n, 1 << (d + 1))
    for o, v in FORCE:
        st.set_option(o, v)
    st.set_option(sps.SPS_OPT_PROFILE, 1)
    st.set_option(sps.SPS_OPT_READOUT_MIN_PLANES, 0)   # broad conditions fused too
    for m, v in conditions(n, gates, seed):
        st.set_readout(m, v)
        st.reset()
        st.apply(gates, EPS)
        rec = fused_record(st)
        assert len(rec) == 1 and rec[0]["flags"] & 32, rec
        c0 = st.counters()
        got = st.probability(m, v)
        c1 = st.counters()
        assert c1.fused_readouts == c0.fused_readouts + 1
        assert c1.kernel_launches == c0.kernel_launches
        want = orc.probability(m, v)
        ker = plain.probability(m, v)
        assert abs(got - want) <= 1e-12, (m, v, got, want)
        assert abs(got - ker) <= 1e-13, (m, v, got, ker)
        # the same sum again, and through the enqueueing form
        assert st.probability(m, v) == got
        pin = torch.full((1,), float("nan"), dtype=torch.float64, pin_memory=True)
        st.probability_async(m, v, pin.data_ptr())
        st.sync()
        assert float(pin[0]) == got
    st.close()
    plain.close()


def test_fused_readout_goes_stale():
    """After the fused apply: another condition, a further apply, a reset, a
    set of the amplitudes and a measurement each take the readout kernel."""
    n, d = 40, 12
    gates = run_gates(7, n, d, 120, ["h"])
    touched = sorted({int(g["t0"]) for g in gates})
    m = [(1 << touched[0]) | (1 << touched[3]), 0]
    v = [1 << touched[3], 0]
    st = sps.SparseState(n, 1 << (d + 2))
    for o, val in FORCE:
        st.set_option(o, val)
    st.set_option(sps.SPS_OPT_READOUT_MIN_PLANES, 0)
    st.set_readout(m, v)
    orc = OracleState(n)
    orc.apply(gates, eps=EPS)

    def fresh():
        st.reset()
        st.apply(gates, EPS)
        f0 = st.counters().fused_readouts
        assert abs(st.probability(m, v) - orc.probability(m, v)) <= 1e-12
        assert st.counters().fused_readouts == f0 + 1

    def kernel_read(want_p, mm=m, vv=v):
        f0 = st.counters().fused_readouts
        k0 = st.counters().kernel_launches
        got = st.probability(mm, vv)
        assert st.counters().fused_readouts == f0
        # the readout kernel (after a reset, the reset's own launch first)
        assert st.counters().kernel_launches >= k0 + 1
        assert abs(got - want_p) <= 1e-12, (got, want_p)

    fresh()
    m2 = [1 << touched[1], 0]
    kernel_read(orc.probability(m2, [0, 0]), m2, [0, 0])
    # a further gate flips one tested bit
    extra = W.to_array([W.X(touched[3])])
    st.apply(extra, EPS)
    o2 = OracleState(n)
    o2.apply(np.concatenate([gates, extra]), eps=EPS)
    kernel_read(o2.probability(m, v))
    fresh()
    st.reset()
    kernel_read(1.0 if (0 & m[0]) == v[0] else 0.0)
    fresh()
    hi, lo, re, im = st.get_amplitudes()
    st.set_amplitudes(hi, lo ^ (1 << touched[3]), re, im)
    kernel_read(o2.probability(m, v))
    fresh()
    st.measure(touched[5], 0.25)
    o3 = OracleState(n)
    o3.apply(gates, eps=EPS)
    o3.measure(touched[5], 0.25)
    kernel_read(o3.probability(m, v))
    # cleared: the kernel again, even after the compiled apply
    st.set_readout(None, None)
    st.reset()
    st.apply(gates, EPS)
    kernel_read(orc.probability(m, v))
    st.close()


def test_fused_readout_not_taken_when_a_pass_follows():
    """An apply whose compiled expansion is followed by a branching pass does
    not end with it: the sum is not formed there, and the kernel reads."""
    n, d = 30, 10
    gates = run_gates(8, n, d, 100, ["h"])
    gates = np.concatenate([gates, W.to_array([W.H(25)])])
    m, v = [(1 << 25) | 1, 0], [1 << 25, 0]
    st = sps.SparseState(n, 1 << (d + 2))
    for o, val in FORCE:
        st.set_option(o, val)
    st.set_option(sps.SPS_OPT_READOUT_MIN_PLANES, 0)
    st.set_readout(m, v)
    st.reset()
    st.apply(gates, EPS)
    f0 = st.counters().fused_readouts
    got = st.probability(m, v)
    assert st.counters().fused_readouts == f0
    orc = OracleState(n)
    orc.apply(gates, eps=EPS)
    assert abs(got - orc.probability(m, v)) <= 1e-12
    st.close()


def test_fused_readout_adder67_w24():
    """The benchmark's step with its readout (the low 16 bits of the label 0):
    the fused sum against the closed form and the readout kernel."""
    from test_gpu_large import adder_closed_form
    wl = W.adder_workload(seed=1, width=24)
    n = wl.layout.nqubits
    m, v = [0xFFFF, 0], [0, 0]
    keys, cre, cim = adder_closed_form(wl)
    sel = (keys & np.uint64(0xFFFF)) == 0
    want = float(np.sum(cre[sel] ** 2 + cim[sel] ** 2))
    st = sps.SparseState(n, 1 << 25)
    st.set_readout(m, v)
    st.reset()
    st.apply(wl.gates, EPS)
    f0 = st.counters().fused_readouts
    got = st.probability(m, v)
    assert st.counters().fused_readouts == f0 + 1
    st.set_readout(None, None)
    ker = st.probability(m, v)
    st.close()
    assert abs(got - want) <= 1e-14, (got, want)
    assert abs(got - ker) <= 1e-15, (got, ker)


def test_fused_readout_min_planes():
    """By default a condition testing fewer than 8 of the launch's label bits
    is left to the readout kernel (it matches many outputs); one testing 8 or
    more, and one no label can meet, are summed by the launch. (A gate's target
    is not always a plane: gates whose controls are known 0 are dropped, and a
    bit no remaining gate touches is 0 in every label.)"""
    n, d = 40, 12
    gates = run_gates(9, n, d, 120, ["h"])
    touched = sorted({int(g["t0"]) for g in gates})
    untouched = [q for q in range(n) if q not in touched]
    orc = OracleState(n)
    orc.apply(gates, eps=EPS)
    st = sps.SparseState(n, 1 << (d + 2))
    for o, val in FORCE:
        st.set_option(o, val)
    hq = [int(g["t0"]) for g in gates[:d]]   # the expansion's qubits: each a plane
    cases = [(hq[:2], False), (hq[:7], False), (hq[:8], True), (hq[:12], True)]
    for qs, fused in cases:
        m = [sum(1 << q for q in qs), 0]
        v = [sum(1 << q for q in qs[::2]), 0]
        st.set_readout(m, v)
        st.reset()
        st.apply(gates, EPS)
        f0 = st.counters().fused_readouts
        got = st.probability(m, v)
        assert st.counters().fused_readouts == f0 + (1 if fused else 0), qs
        assert abs(got - orc.probability(m, v)) <= 1e-12
    if untouched:   # no label can match: summed (to 0) by the launch
        m = [(1 << untouched[0]) | (1 << touched[0]), 0]
        v = [1 << untouched[0], 0]
        st.set_readout(m, v)
        st.reset()
        st.apply(gates, EPS)
        f0 = st.counters().fused_readouts
        assert st.probability(m, v) == 0.0
        assert st.counters().fused_readouts == f0 + 1
    st.close()
