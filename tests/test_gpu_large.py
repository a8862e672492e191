"""GPU parity at the sizes the benchmark runs, against checkers that do not
share the product's arithmetic:

  * givens64 (64 qubits, 4 occupied modes, the benchmark's seeded layers):
    long enough for the C(64,4) = 635,376-label sector to fill and for the
    amplitude-only branching form (128-bit labels) to take runs; checked
    against the dense weight-sector simulator of the oracle.
  * the same family with 5 modes (the 7,624,512-label sector, larger than
    L2): a prefix of layers against the sector simulator.
  * adder67-w24 (67 qubits, register a over 24 bits, 16,777,216 entries, the
    bit-sliced fused pass): against the closed form of integer addition and
    the controlled-phase layer (Sec. 3.2 phases f(b) on the labels g(b)).
  * the strict prune at exactly eps^2 in every branching form.

Labels bit for bit (one-sided labels only below 10 eps), amplitudes within
1e-12 max abs."""

import math

import numpy as np
import pytest

from oracle import OracleState, sector_run
from paper_2105_01533_gb300 import sps
from paper_2105_01533_gb300 import workloads as W

from helpers import compare_states

pytestmark = pytest.mark.gpu

EPS = 1e-14
AMP_KIND = 10


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2105_01533_gb300 import build as B
    B.build()
    sps.load_library()
    yield


def sector_state(n, modes, gates):
    """Nonzero entries of the sector simulator as a sorted (hi, lo, re, im)."""
    labels, amp = sector_run(n, (1 << modes) - 1, gates[modes:])
    nz = amp != 0
    lo = labels[nz]
    return np.zeros(len(lo), np.uint64), lo, amp[nz].real.copy(), amp[nz].imag.copy()


@pytest.mark.parametrize("layers", [60])
def test_givens64_against_sector_simulator(layers):
    n, modes = 64, 4
    gates = W.givens_workload(seed=2, nqubits=n, modes=modes, layers=layers)
    st = sps.SparseState(n, 700_000)
    st.set_option(sps.SPS_OPT_PROFILE, 1)
    st.apply(gates, EPS)
    recs = st.profile_read()
    got = st.get_amplitudes()
    st.close()
    took = sum(1 for r in recs if r["kind"] == AMP_KIND and r["n_out"] > 0)
    assert took >= layers // 2, "amplitude-only runs taken: %d" % took
    assert len(got[1]) == math.comb(64, 4)
    assert np.all(got[0] == 0)
    stats = compare_states(got, sector_state(n, modes, gates), EPS)
    assert stats["common"] == math.comb(64, 4)


def test_givens64_five_modes_prefix():
    """The larger-than-L2 variant: 5 modes on 64 qubits (<= 7,624,512 labels)."""
    n, modes = 64, 5
    gates = W.givens_workload(seed=2, nqubits=n, modes=modes, layers=5)
    st = sps.SparseState(n, 8_000_000)
    st.apply(gates, EPS)
    got = st.get_amplitudes()
    st.close()
    assert {bin(int(x)).count("1") for x in got[1][:1000]} == {5}
    stats = compare_states(got, sector_state(n, modes, gates), EPS)
    assert stats["common"] > 1_000_000


def adder_closed_form(wl):
    """Keys (a, b) for a < 2^width with amplitude 2^(-width/2) prod_j e^{i phi_j}
    over the controlled-phase pairs whose bits are set after the adder
    (a in register a, (a + b) mod 2^32 in register b)."""
    n, w = wl.layout.nbits, wl.width
    avals = np.arange(1 << w, dtype=np.uint64)
    bsum = (avals + np.uint64(wl.b_const)) & np.uint64((1 << n) - 1)
    reg = avals | (bsum << np.uint64(n))
    phase = np.zeros(len(avals))
    for q1, q2, phi in wl.cp_pairs:
        both = ((reg >> np.uint64(q1)) & np.uint64(1)) & ((reg >> np.uint64(q2)) & np.uint64(1))
        phase += phi * both.astype(float)
    keys = avals | (np.uint64(wl.b_const) << np.uint64(n))
    return keys, 2.0 ** (-w / 2) * np.cos(phase), 2.0 ** (-w / 2) * np.sin(phase)


def test_adder67_w24_closed_form():
    """16,777,216 entries through the expansion and the bit-sliced fused pass."""
    wl = W.adder_workload(seed=1, width=24)
    st = sps.SparseState(wl.layout.nqubits, 1 << 25)
    st.set_option(sps.SPS_OPT_PROFILE, 1)
    st.apply(wl.gates, EPS)
    recs = st.profile_read()
    hi, lo, re, im = st.get_amplitudes()
    st.close()
    fused = [r for r in recs if r["kind"] == 1]
    assert fused and max(r["n_in"] for r in fused) == 1 << 24
    keys, cre, cim = adder_closed_form(wl)
    order = np.argsort(keys)
    assert np.all(hi == 0)
    np.testing.assert_array_equal(lo, keys[order])
    err = max(float(np.max(np.abs(re - cre[order]))), float(np.max(np.abs(im - cim[order]))))
    assert err <= 1e-12, err


@pytest.mark.parametrize("opts", [
    [(sps.SPS_OPT_BRANCH_FORM, 2), (sps.SPS_OPT_SMALL_RUN_CAP, 0), (sps.SPS_OPT_EXPAND, 0)],
    [(sps.SPS_OPT_BRANCH_FORM, 1), (sps.SPS_OPT_SMALL_RUN_CAP, 0), (sps.SPS_OPT_EXPAND, 0)],
    [(sps.SPS_OPT_SMALL_RUN_CAP, 2048), (sps.SPS_OPT_EXPAND, 0)],
    [(sps.SPS_OPT_SMALL_RUN_CAP, 0), (sps.SPS_OPT_EXPAND, 1)],
], ids=["gather", "scatter", "one-block", "expansion"])
def test_prune_keeps_exactly_eps_squared(opts):
    """eps = 2^-20: an amplitude of exactly eps stays, one an ulp below goes,
    and the exact zeros Ry(0) leaves on the partners go (strict <)."""
    eps = 2.0 ** -20
    below = float(np.nextafter(eps, 0.0))
    init = (np.zeros(4, np.uint64), np.array([0, 2, 4, 8], np.uint64),
            np.array([eps, below, 0.0, -eps]), np.array([0.0, 0.0, eps, 0.0]))
    st = sps.SparseState(8, 64)
    for o, v in opts:
        st.set_option(o, v)
    st.set_amplitudes(*init)
    st.apply(W.to_array([W.Ry(0, 0.0)]), eps)
    hi, lo, re, im = st.get_amplitudes()
    st.close()
    orc = OracleState(8)
    orc.set(*init)
    orc.apply(W.to_array([W.Ry(0, 0.0)]), eps=eps)
    ohi, olo, ore, oim = orc.get()
    assert lo.tolist() == olo.tolist() == [0, 4, 8]
    np.testing.assert_array_equal(re, ore)
    np.testing.assert_array_equal(im, oim)
