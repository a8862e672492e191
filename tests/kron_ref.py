"""Textbook references used to pin the oracle (tests only).

* ``full_unitary``: the 2^n x 2^n matrix of one gate record, assembled with
  Kronecker products exactly as Sec. 2.1 of arXiv 2105.01533 writes states and
  controlled gates: |i> = |i_{n-1}> (x) ... (x) |i_0> and
  CU = |0><0| (x) 1 + |1><1| (x) U (iterated for several controls). Rotations
  come from scipy's matrix exponential of their generators
  (R_P(theta) = exp(-i theta P / 2)); Givens(theta) is the exponential of
  theta (|e1><e0| - |e0><e1|) with e0 = (bit p = 0, bit q = 1) and
  e1 = (bit p = 1, bit q = 0).
* ``tensor_run``: a dense simulator that keeps the state as an n-axis tensor
  and contracts each gate's small matrix into the target axes with einsum.

Neither shares code with the oracle or with the CUDA path.
"""

from __future__ import annotations

import numpy as np
from scipy.linalg import expm

I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)   # |0><0|
P1 = np.array([[0, 0], [0, 1]], dtype=complex)   # |1><1|
SP = np.array([[0, 0], [1, 0]], dtype=complex)   # |1><0|
SM = np.array([[0, 1], [0, 0]], dtype=complex)   # |0><1|

OP_X, OP_Y, OP_Z, OP_S, OP_SDG, OP_T, OP_TDG = 1, 2, 3, 4, 5, 6, 7
OP_P, OP_RZ, OP_H, OP_RX, OP_RY, OP_GIVENS = 8, 9, 10, 11, 12, 13


def single_qubit_matrix(op: int, theta: float) -> np.ndarray:
    if op == OP_X:
        return PX
    if op == OP_Y:
        return PY
    if op == OP_Z:
        return PZ
    if op == OP_S:
        return np.diag([1, 1j])
    if op == OP_SDG:
        return np.diag([1, -1j])
    if op == OP_T:
        return np.diag([1, np.exp(1j * np.pi / 4)])
    if op == OP_TDG:
        return np.diag([1, np.exp(-1j * np.pi / 4)])
    if op == OP_P:
        return np.diag([1, np.exp(1j * theta)])
    if op == OP_RZ:
        return expm(-0.5j * theta * PZ)
    if op == OP_RX:
        return expm(-0.5j * theta * PX)
    if op == OP_RY:
        return expm(-0.5j * theta * PY)
    if op == OP_H:
        return np.sqrt(0.5) * np.array([[1, 1], [1, -1]], dtype=complex)
    raise ValueError(op)


def embed(n: int, ops: dict) -> np.ndarray:
    """Kronecker product over qubits n-1 ... 0 (leftmost factor = qubit n-1)."""
    out = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        out = np.kron(out, ops.get(q, I2))
    return out


def _mask_qubits(cmask) -> list:
    lo, hi = int(cmask[0]), int(cmask[1])
    return [q for q in range(64) if (lo >> q) & 1] + [64 + q for q in range(64) if (hi >> q) & 1]


def full_unitary(n: int, rec) -> np.ndarray:
    op, t0, t1, theta = int(rec["op"]), int(rec["t0"]), int(rec["t1"]), float(rec["theta"])
    controls = _mask_qubits(rec["cmask"])
    if op == OP_GIVENS:
        gen = embed(n, {t0: SP, t1: SM}) - embed(n, {t0: SM, t1: SP})
        target = expm(theta * gen)
    else:
        target = embed(n, {t0: single_qubit_matrix(op, theta)})
    if not controls:
        return target
    proj = embed(n, {c: P1 for c in controls})
    ident = np.eye(1 << n, dtype=complex)
    return (ident - proj) + proj @ target


def kron_run(n: int, gates) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1.0
    for rec in gates:
        psi = full_unitary(n, rec) @ psi
    return psi


def tensor_run(n: int, gates, start_index: int = 0) -> np.ndarray:
    """Dense simulation with the state as a tensor of shape (2,)*n whose axis
    n-1-q is qubit q. Returns the flat 2^n vector (index = label)."""
    psi = np.zeros((2,) * n, dtype=complex)
    idx = tuple((start_index >> (n - 1 - ax)) & 1 for ax in range(n))
    psi[idx] = 1.0
    ax = lambda q: n - 1 - q  # noqa: E731
    for rec in gates:
        op, t0, t1, theta = int(rec["op"]), int(rec["t0"]), int(rec["t1"]), float(rec["theta"])
        controls = _mask_qubits(rec["cmask"])
        sel = [slice(None)] * n
        for c in controls:
            sel[ax(c)] = 1
        sel = tuple(sel)
        sub = psi[sel]  # view with the control axes fixed to 1
        # axes of `sub`: the remaining qubits in descending order
        rest = [q for q in range(n - 1, -1, -1) if q not in controls]
        if op == OP_GIVENS:
            c, s = np.cos(theta), np.sin(theta)
            # 4x4 matrix on (bit p, bit q) ordered index 2*bp + bq
            G = np.eye(4, dtype=complex)
            e0, e1 = 0 * 2 + 1, 1 * 2 + 0
            G[e0, e0], G[e0, e1], G[e1, e0], G[e1, e1] = c, -s, s, c
            G = G.reshape(2, 2, 2, 2)
            ip, iq = rest.index(t0), rest.index(t1)
            moved = np.moveaxis(sub, (ip, iq), (0, 1))
            new = np.einsum("abcd,cd...->ab...", G, moved)
            sub[...] = np.moveaxis(new, (0, 1), (ip, iq))
        else:
            U = single_qubit_matrix(op, theta)
            it = rest.index(t0)
            moved = np.moveaxis(sub, it, 0)
            new = np.einsum("ab,b...->a...", U, moved)
            sub[...] = np.moveaxis(new, 0, it)
        psi[sel] = sub
    # flatten: axis 0 is qubit n-1 -> C-order flattening gives index = label
    return psi.reshape(-1)


def pauli_exp_unitary(n: int, x: int, z: int, controls: int, theta: float) -> np.ndarray:
    """exp(-i theta/2 P) for the Pauli string with X at x-only bits, Z at z-only
    bits and Y where both are set (qubit order as embed), as a controlled gate."""
    ops = {}
    for q in range(n):
        bx, bz = (x >> q) & 1, (z >> q) & 1
        if bx or bz:
            ops[q] = PY if (bx and bz) else (PX if bx else PZ)
    target = expm(-0.5j * theta * embed(n, ops))
    if not controls:
        return target
    proj = embed(n, {c: P1 for c in range(n) if (controls >> c) & 1})
    return (np.eye(1 << n, dtype=complex) - proj) + proj @ target
