"""Shared test helpers: state comparison and oracle-driven workload filters."""

from __future__ import annotations

import numpy as np

from paper_2105_01533_gb300 import workloads as W

AMP_TOL = 1e-12       # max abs error per amplitude component
EDGE_FACTOR = 10.0    # one-sided keys allowed only below EDGE_FACTOR * eps


def _void_keys(hi, lo):
    k = np.empty((len(lo), 2), np.uint64)
    k[:, 0] = hi
    k[:, 1] = lo
    return np.ascontiguousarray(k).view("V16").ravel()


def compare_states(got, want, eps: float, atol: float = AMP_TOL):
    """Compare two (hi, lo, re, im) tuples. Labels must match bit for bit except
    labels present on one side only whose magnitude there is < 10*eps; shared
    labels must agree to `atol` per component. Returns a dict of statistics and
    raises AssertionError on a mismatch."""
    ghi, glo, gre, gim = got
    whi, wlo, wre, wim = want
    gk = _void_keys(ghi, glo)
    wk = _void_keys(whi, wlo)
    assert len(np.unique(gk)) == len(gk), "duplicate labels in the first state"
    common, gi, wi = np.intersect1d(gk, wk, assume_unique=True, return_indices=True)
    only_g = np.setdiff1d(np.arange(len(gk)), gi)
    only_w = np.setdiff1d(np.arange(len(wk)), wi)
    lim = EDGE_FACTOR * eps
    mag_g = np.hypot(gre[only_g], gim[only_g])
    mag_w = np.hypot(wre[only_w], wim[only_w])
    assert np.all(mag_g < lim), "labels only in the first state with |a| >= 10 eps: %d" % int(
        np.sum(mag_g >= lim))
    assert np.all(mag_w < lim), "labels only in the second state with |a| >= 10 eps: %d" % int(
        np.sum(mag_w >= lim))
    err = 0.0
    if len(common):
        err = max(float(np.max(np.abs(gre[gi] - wre[wi]))), float(np.max(np.abs(gim[gi] - wim[wi]))))
    assert err <= atol, "max amplitude error %.3e > %.1e" % (err, atol)
    return {"common": len(common), "only_first": len(only_g), "only_second": len(only_w),
            "max_err": err}


class OracleBranchFilter:
    """keep_branch predicate for the random-mix generator: keeps a branching
    gate iff the oracle says the state after it has at most `cap` nonzeros."""

    def __init__(self, nqubits: int, cap: int, eps: float):
        from oracle import OracleState
        self.st = OracleState(nqubits)
        self.cap = cap
        self.eps = eps
        self.applied = 0

    def __call__(self, accepted, cand) -> bool:
        if len(accepted) > self.applied:
            self.st.apply(W.to_array(accepted[self.applied:]), eps=self.eps)
            self.applied = len(accepted)
        trial = self.st.clone()
        trial.apply(W.to_array([cand]), eps=self.eps)
        return trial.nnz() <= self.cap


def plain24_gates(seed: int = 0, nqubits: int = 24, ngates: int = 2000, cap: int = 4096,
                  eps: float = 1e-14) -> np.ndarray:
    """The 24-qubit plain workload: H on 8 random qubits, then 2000 gates in the
    70/20/10 mix with the H restriction decided by the oracle."""
    return W.random_mix(seed, nqubits, ngates, n_initial_h=8,
                        keep_branch=OracleBranchFilter(nqubits, cap, eps))
