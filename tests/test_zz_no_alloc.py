"""GPU test of sps_branch_apply_static, the allocation-free branching entry
point for callers that must not allocate device memory (for example a host
framework that owns all device memory, or code inside an allocator callback).

It is called through the C ABI on device arrays this test owns, and its
output is compared with the regular entry point (sps_apply) on the same input,
within the tolerance of the other parity tests, on two calls in a row: the
second call reuses the library's fixed scratch array left by the first.
This file is collected last so that a stop at the first failure has already
run every other test."""

import numpy as np
import pytest

from paper_2105_01533_gb300 import sps
from paper_2105_01533_gb300 import workloads as W

from helpers import compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2105_01533_gb300 import build as B
    B.build()
    sps.load_library()
    return t


def device_arrays(torch, n):
    u = lambda: torch.zeros(max(n, 1), dtype=torch.int64, device="cuda")  # noqa: E731
    f = lambda: torch.zeros(max(n, 1), dtype=torch.float64, device="cuda")  # noqa: E731
    return u(), u(), f(), f()


def to_host(torch, arrs, n, kw):
    hi, lo, re, im = [a[:n].cpu().numpy() for a in arrs]
    hi = hi.view(np.uint64) if kw == 2 else np.zeros(n, np.uint64)
    lo = lo.view(np.uint64)
    order = np.lexsort((lo, hi))
    return hi[order], lo[order], re[order], im[order]


def load_state(torch, st, cap):
    """The regular path's current state copied into fresh device arrays."""
    arrs = device_arrays(torch, cap)
    n = sps.sps_get_amplitudes(st.handle, arrs[0], arrs[1], arrs[2], arrs[3], cap)
    return arrs, n


@pytest.mark.parametrize("nqubits", [40, 90])
def test_static_branch_matches_regular_path_twice(torch, nqubits):
    kw = 1 if nqubits <= 63 else 2
    eps = 1e-14
    rng = W.SplitMix64(nqubits)
    prep = W.to_array([W.H(q) for q in rng.distinct(nqubits, 11)] +
                      [W.CX(3, 70 % nqubits), W.T(5), W.Ry(7, 0.9, 2)])
    g1 = W.to_array([W.H(rng.below(nqubits))])
    g2 = W.to_array([W.Givens(1, nqubits - 1, 0.6)])
    cap = 1 << 14
    stream = torch.cuda.current_stream()
    h = int(stream.cuda_stream)

    st = sps.SparseState(nqubits, cap)
    st.apply(prep, eps)
    (inp, n0) = load_state(torch, st, cap)
    st.apply(g1, eps)
    want1 = st.get_amplitudes()
    st.apply(g2, eps)
    want2 = st.get_amplitudes()
    st.close()

    out1 = device_arrays(torch, cap)
    n1 = sps.sps_branch_apply_static(g1, nqubits, inp, n0, eps, out1, cap, h)
    got1 = to_host(torch, out1, n1, kw)
    compare_states(got1, want1, eps)

    out2 = device_arrays(torch, cap)
    n2 = sps.sps_branch_apply_static(g2, nqubits, out1, n1, eps, out2, cap, h)
    got2 = to_host(torch, out2, n2, kw)
    compare_states(got2, want2, eps)
    assert n1 == len(want1[1]) and n2 == len(want2[1])


def test_static_branch_limits(torch):
    h = int(torch.cuda.current_stream().cuda_stream)
    big = device_arrays(torch, 65_537)
    out = device_arrays(torch, 16)
    with pytest.raises(sps.SpsError) as e:
        sps.sps_branch_apply_static(W.to_array([W.H(0)]), 30, big, 65_537, 0.0, out, 16, h)
    assert e.value.status == sps.SPS_ERR_CAPACITY
    # not a branching gate
    with pytest.raises(sps.SpsError) as e:
        sps.sps_branch_apply_static(W.to_array([W.X(0)]), 30, big, 4, 0.0, out, 16, h)
    assert e.value.status == sps.SPS_ERR_ARG
    # more outputs than out_cap: H on 16 inputs gives 32 entries
    lo = torch.arange(16, dtype=torch.int64, device="cuda") << 1
    re = torch.full((16,), 0.25, dtype=torch.float64, device="cuda")
    im = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(sps.SpsError) as e:
        sps.sps_branch_apply_static(W.to_array([W.H(0)]), 30, (None, lo, re, im), 16, 0.0, out,
                                    16, h)
    assert e.value.status == sps.SPS_ERR_CAPACITY
    # and the scratch array is still usable afterwards
    out = device_arrays(torch, 64)
    n = sps.sps_branch_apply_static(W.to_array([W.H(0)]), 30, (None, lo, re, im), 16, 0.0, out,
                                    64, h)
    assert n == 32


def test_static_branch_rejects_aliased_outputs(torch):
    """Writing the result over the input would corrupt entries the pass still
    reads: such a call is refused before anything is launched."""
    h = int(torch.cuda.current_stream().cuda_stream)
    arrs = device_arrays(torch, 64)
    with pytest.raises(sps.SpsError) as e:
        sps.sps_branch_apply_static(W.to_array([W.H(0)]), 30, arrs, 8, 0.0, arrs, 64, h)
    assert e.value.status == sps.SPS_ERR_ARG


def test_static_branch_at_its_input_limit(torch):
    """Exactly 65,536 distinct inputs under H on a qubit none of them sets:
    131,072 outputs in a table at its 50% load limit, the same as sps_apply."""
    h = int(torch.cuda.current_stream().cuda_stream)
    n_in = 1 << 16
    eps = 1e-14
    gate = W.to_array([W.H(0)])
    lo = (torch.arange(n_in, dtype=torch.int64, device="cuda") << 1)
    re = torch.full((n_in,), 2.0 ** -8, dtype=torch.float64, device="cuda")
    im = torch.zeros(n_in, dtype=torch.float64, device="cuda")
    ins = (torch.zeros(n_in, dtype=torch.int64, device="cuda"), lo, re, im)
    out = device_arrays(torch, 2 * n_in)
    n = sps.sps_branch_apply_static(gate, 40, ins, n_in, eps, out, 2 * n_in, h)
    assert n == 2 * n_in
    got = to_host(torch, out, n, 1)
    st = sps.SparseState(40, 2 * n_in)
    st.set_amplitudes(None, lo.cpu().numpy().view(np.uint64), re.cpu().numpy(), im.cpu().numpy())
    st.apply(gate, eps)
    want = st.get_amplitudes()
    st.close()
    compare_states(got, want, eps)
