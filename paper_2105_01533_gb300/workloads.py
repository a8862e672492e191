"""Seeded synthetic gate streams (input generators only).

This module builds gate lists; it simulates nothing. Both the CUDA path and the
CPU oracle consume what it produces. It holds no amplitude or key arithmetic
of the simulator: where a workload needs to know how many nonzeros a gate would
create (the "H restricted so nonzeros stay <= cap" rule), the caller passes a
``keep_branch`` predicate in.

Gate record (32 bytes, little-endian), the format of ``sps_gate`` in
``include/sps.h``::

    uint8  op        gate code (OP_* below)
    uint8  reserved  0
    uint16 t0        target qubit (Givens: qubit p)
    uint16 t1        Givens: qubit q; otherwise 0
    uint16 reserved  0
    uint64 cmask[2]  control qubits as a bitmask (word 0: qubits 0..63)
    double theta     rotation angle, radians

Qubit k is bit k of a basis label (|i> = |i_{n-1}> (x) ... (x) |i_0>, Sec. 2.1
of arXiv 2105.01533).

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then the 64-bit finaliser. Angles are drawn as 2*pi*(u >> 11)*2^-53, i.e.
uniform on [0, 2*pi).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence

import numpy as np

GATE_DTYPE = np.dtype([
    ("op", np.uint8), ("reserved0", np.uint8), ("t0", np.uint16), ("t1", np.uint16),
    ("reserved1", np.uint16), ("cmask", np.uint64, (2,)), ("theta", np.float64),
])
assert GATE_DTYPE.itemsize == 32

OP_X, OP_Y, OP_Z, OP_S, OP_SDG, OP_T, OP_TDG = 1, 2, 3, 4, 5, 6, 7
OP_P, OP_RZ, OP_H, OP_RX, OP_RY, OP_GIVENS = 8, 9, 10, 11, 12, 13

PERM_OPS = (OP_X, OP_Y)
DIAG_OPS = (OP_Z, OP_S, OP_SDG, OP_T, OP_TDG, OP_P, OP_RZ)
BRANCH_OPS = (OP_H, OP_RX, OP_RY, OP_GIVENS)
OP_NAMES = {OP_X: "X", OP_Y: "Y", OP_Z: "Z", OP_S: "S", OP_SDG: "Sdg", OP_T: "T",
            OP_TDG: "Tdg", OP_P: "P", OP_RZ: "Rz", OP_H: "H", OP_RX: "Rx",
            OP_RY: "Ry", OP_GIVENS: "Givens"}

_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream (Steele, Lea, Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) by the multiply-shift map."""
        return (self.next_u64() * n) >> 64

    def uniform(self) -> float:
        """Uniform double in [0, 1)."""
        return (self.next_u64() >> 11) * 2.0 ** -53

    def angle(self) -> float:
        return 2.0 * math.pi * self.uniform()

    def distinct(self, n: int, k: int) -> List[int]:
        out: List[int] = []
        while len(out) < k:
            q = self.below(n)
            if q not in out:
                out.append(q)
        return out


def _mask(qubits: Sequence[int]):
    lo = hi = 0
    for q in qubits:
        if q < 64:
            lo |= 1 << q
        else:
            hi |= 1 << (q - 64)
    return lo, hi


def gate(op: int, t0: int, controls: Sequence[int] = (), theta: float = 0.0, t1: int = 0):
    """One record as a tuple for ``np.array(..., dtype=GATE_DTYPE)``."""
    lo, hi = _mask(controls)
    return (op, 0, t0, t1, 0, (lo, hi), float(theta))


def to_array(records) -> np.ndarray:
    return np.array(list(records), dtype=GATE_DTYPE)


# Named constructors ----------------------------------------------------------
def X(t, *c): return gate(OP_X, t, c)
def Y(t, *c): return gate(OP_Y, t, c)
def Z(t, *c): return gate(OP_Z, t, c)
def S(t, *c): return gate(OP_S, t, c)
def Sdg(t, *c): return gate(OP_SDG, t, c)
def T(t, *c): return gate(OP_T, t, c)
def Tdg(t, *c): return gate(OP_TDG, t, c)
def P(t, theta, *c): return gate(OP_P, t, c, theta)
def Rz(t, theta, *c): return gate(OP_RZ, t, c, theta)
def H(t, *c): return gate(OP_H, t, c)
def Rx(t, theta, *c): return gate(OP_RX, t, c, theta)
def Ry(t, theta, *c): return gate(OP_RY, t, c, theta)
def Givens(p, q, theta, *c): return gate(OP_GIVENS, p, c, theta, t1=q)
def CX(c, t): return X(t, c)
def CCX(c1, c2, t): return X(t, c1, c2)
def CZ(c, t): return Z(t, c)
def CP(c, t, theta): return P(t, theta, c)
def CRz(c, t, theta): return Rz(t, theta, c)


_INVERSE_OP = {OP_S: OP_SDG, OP_SDG: OP_S, OP_T: OP_TDG, OP_TDG: OP_T}


def inverse(gates: np.ndarray) -> np.ndarray:
    """The inverse circuit: reversed order, each gate replaced by its inverse."""
    inv = np.array(gates[::-1], dtype=GATE_DTYPE, copy=True)
    for i in range(len(inv)):
        op = int(inv[i]["op"])
        if op in _INVERSE_OP:
            inv[i]["op"] = _INVERSE_OP[op]
        elif op in (OP_P, OP_RZ, OP_RX, OP_RY, OP_GIVENS):
            inv[i]["theta"] = -inv[i]["theta"]
    return inv


# Random mixes -----------------------------------------------------------------
KeepBranch = Callable[[List[tuple], tuple], bool]


class CountingBound:
    """keep_branch rule that needs no simulation: each branching gate at most
    doubles the number of nonzeros, so after h of them from |0..0> there are at
    most 2^h. A branching gate is kept while 2^(h+1) <= cap."""

    def __init__(self, cap: int):
        self.cap = int(cap)
        self.h = 0

    def __call__(self, accepted, cand) -> bool:
        if (1 << (self.h + 1)) <= self.cap:
            self.h += 1
            return True
        return False


def random_mix(seed: int, nqubits: int, ngates: int, n_initial_h: int = 8,
               keep_branch: Optional[KeepBranch] = None,
               p_perm: float = 0.7, p_diag: float = 0.2) -> np.ndarray:
    """Random circuit in the mix of the 24-qubit plain workload.

    ``n_initial_h`` H gates on distinct random qubits, then ``ngates`` gates:
    with probability p_perm one of X / CNOT / Toffoli (1:1:1), with p_diag one
    of Z / S / T / controlled-Rz (1:1:1:1, angle uniform on [0, 2 pi)), else
    an H candidate. An H candidate is kept iff ``keep_branch(accepted,
    candidate)`` says so (None keeps all); otherwise the gate is redrawn from
    the permutation and diagonal classes in their 70:20 proportion. Qubits are
    distinct within a gate and uniform over all qubits.
    """
    rng = SplitMix64(seed)
    out: List[tuple] = []
    for q in rng.distinct(nqubits, min(n_initial_h, nqubits)):
        g = H(q)
        if keep_branch is None or keep_branch(out, g):
            out.append(g)
    while len(out) < ngates + n_initial_h:
        u = rng.uniform()
        if u >= p_perm + p_diag:
            g = H(rng.below(nqubits))
            if keep_branch is None or keep_branch(out, g):
                out.append(g)
                continue
            u = rng.uniform() * (p_perm + p_diag)
        if u < p_perm:
            kind = rng.below(3)
            qs = rng.distinct(nqubits, kind + 1)
            out.append(gate(OP_X, qs[-1], qs[:-1]))
        else:
            kind = rng.below(4)
            if kind == 3:
                c, t = rng.distinct(nqubits, 2)
                out.append(CRz(c, t, rng.angle()))
            else:
                t = rng.below(nqubits)
                out.append(gate((OP_Z, OP_S, OP_T)[kind], t))
    return to_array(out)


def random_all_gates(seed: int, nqubits: int, ngates: int, max_controls: int = 2,
                     branch_frac: float = 0.3,
                     keep_branch: Optional[KeepBranch] = None) -> np.ndarray:
    """Random circuit drawing every gate code, with 0..max_controls controls.
    A branching candidate rejected by ``keep_branch`` becomes a
    phase/permutation gate. For parity and pin tests."""
    rng = SplitMix64(seed)
    perm_diag = list(PERM_OPS + DIAG_OPS)
    out: List[tuple] = []
    for _ in range(ngates):
        branch = rng.uniform() < branch_frac
        if branch and keep_branch is not None and not keep_branch(out, None):
            branch = False
        if branch:
            op = BRANCH_OPS[rng.below(len(BRANCH_OPS))]
        else:
            op = perm_diag[rng.below(len(perm_diag))]
        ntarg = 2 if op == OP_GIVENS else 1
        nctl = rng.below(max_controls + 1)
        nctl = min(nctl, nqubits - ntarg)
        qs = rng.distinct(nqubits, ntarg + nctl)
        theta = rng.angle()
        if op == OP_GIVENS:
            out.append(Givens(qs[0], qs[1], theta, *qs[2:]))
        else:
            out.append(gate(op, qs[0], qs[1:], theta))
    return to_array(out)


# Reversible arithmetic: the Cuccaro ripple-carry adder -------------------------
@dataclass
class AdderLayout:
    """Qubit map of the ripple-carry adder workload."""
    nbits: int = 32
    a: List[int] = field(default_factory=list)
    b: List[int] = field(default_factory=list)
    cin: int = 0
    cout: int = 0
    ancilla: int = 0
    nqubits: int = 0

    def __post_init__(self):
        n = self.nbits
        self.a = list(range(n))
        self.b = list(range(n, 2 * n))
        self.cin = 2 * n
        self.cout = 2 * n + 1
        self.ancilla = 2 * n + 2
        self.nqubits = 2 * n + 3


def cuccaro_adder(lay: AdderLayout) -> np.ndarray:
    """In-place b <- a + b (mod 2^n), cout ^= carry out, a and cin restored.

    Built from the MAJ / UMA blocks of Cuccaro, Draper, Kutin, Moulton,
    "A new quantum ripple-carry addition circuit" (quant-ph/0410184):
    MAJ(c, b, a) = CNOT(a->b), CNOT(a->c), Toffoli(c, b -> a) leaves the carry
    in a; UMA(c, b, a) = Toffoli(c, b -> a), CNOT(a->c), CNOT(c->b) undoes it
    and leaves the sum bit in b. The carry into bit i sits in cin for i = 0 and
    in a[i-1] afterwards.
    """
    n, a, b = lay.nbits, lay.a, lay.b
    recs: List[tuple] = []

    def maj(c, bb, aa):
        recs.extend([CX(aa, bb), CX(aa, c), CCX(c, bb, aa)])

    def uma(c, bb, aa):
        recs.extend([CCX(c, bb, aa), CX(aa, c), CX(c, bb)])

    carry_in = [lay.cin] + a[:-1]
    for i in range(n):
        maj(carry_in[i], b[i], a[i])
    recs.append(CX(a[n - 1], lay.cout))
    for i in reversed(range(n)):
        uma(carry_in[i], b[i], a[i])
    return to_array(recs)


@dataclass
class AdderWorkload:
    gates: np.ndarray
    layout: AdderLayout
    b_const: int
    width: int            # number of low bits of a in uniform superposition
    cp_pairs: List[tuple]  # (q1, q2, phi) of the controlled-phase layer


def adder_workload(seed: int = 1, nbits: int = 32, width: int = 16,
                   n_cp: int = 32) -> AdderWorkload:
    """Reversible-arithmetic workload: H on a[0..width-1] (2^width nonzeros),
    X gates loading a seeded constant into b, the ripple-carry adder, a layer of
    n_cp controlled-phase gates CP(phi), phi uniform on [0, 2 pi), on seeded
    pairs of distinct qubits of a and b, then the inverse adder."""
    lay = AdderLayout(nbits)
    rng = SplitMix64(seed)
    b_const = rng.next_u64() & ((1 << nbits) - 1)
    recs: List[tuple] = [H(q) for q in lay.a[:width]]
    recs += [X(lay.b[i]) for i in range(nbits) if (b_const >> i) & 1]
    add = cuccaro_adder(lay)
    pool = lay.a + lay.b
    cp_pairs = []
    for _ in range(n_cp):
        i, j = rng.distinct(len(pool), 2)
        phi = rng.angle()
        cp_pairs.append((pool[i], pool[j], phi))
    cp = to_array([CP(q1, q2, phi) for (q1, q2, phi) in cp_pairs])
    gates = np.concatenate([to_array(recs), add, cp, inverse(add)])
    return AdderWorkload(gates, lay, b_const, width, cp_pairs)


# Number-conserving workload: Givens layers ------------------------------------
def givens_workload(seed: int = 2, nqubits: int = 64, modes: int = 4,
                    layers: int = 500) -> np.ndarray:
    """X on qubits 0..modes-1 (start label with `modes` ones), then `layers`
    layers. Each layer: a seeded random perfect matching of the qubits gives
    nqubits/2 Givens(theta) on disjoint pairs, theta uniform on [0, 2 pi); then
    nqubits/2 controlled-Z on seeded random pairs of distinct qubits."""
    rng = SplitMix64(seed)
    recs: List[tuple] = [X(q) for q in range(modes)]
    for _ in range(layers):
        perm = list(range(nqubits))
        for i in range(nqubits - 1, 0, -1):  # Fisher-Yates
            j = rng.below(i + 1)
            perm[i], perm[j] = perm[j], perm[i]
        for k in range(nqubits // 2):
            recs.append(Givens(perm[2 * k], perm[2 * k + 1], rng.angle()))
        for _ in range(nqubits // 2):
            c, t = rng.distinct(nqubits, 2)
            recs.append(CZ(c, t))
    return to_array(recs)


# Batched workload -------------------------------------------------------------
@dataclass
class BatchCircuit:
    seed: int
    nqubits: int
    cap: int
    gates: np.ndarray


def batched_workload(count: int = 4096, first_seed: int = 1, qubits=(20, 100),
                     depth=(200, 5000), log2_cap=(8, 16)) -> List[BatchCircuit]:
    """Independent circuits with seeds first_seed..first_seed+count-1: qubits
    uniform on [qubits], depth uniform on [depth], nonzero cap 2^u with u
    uniform on [log2_cap] (log-uniform cap), gate mix of ``random_mix`` with the
    branching restriction enforced by :class:`CountingBound` against the cap."""
    out = []
    for s in range(first_seed, first_seed + count):
        rng = SplitMix64(s * 0x2545F4914F6CDD1D + 7)
        nq = qubits[0] + rng.below(qubits[1] - qubits[0] + 1)
        d = depth[0] + rng.below(depth[1] - depth[0] + 1)
        cap = int(2.0 ** (log2_cap[0] + (log2_cap[1] - log2_cap[0]) * rng.uniform()))
        g = random_mix(s, nq, d, keep_branch=CountingBound(cap))
        out.append(BatchCircuit(s, nq, cap, g))
    return out


# Batched workload, vectorised ----------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix_block(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Values offset+1 .. offset+count of the SplitMix64 stream of `seed`
    (the generator is counter based: value k mixes seed + k * golden)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & _M64) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _below(u: np.ndarray, n) -> np.ndarray:
    """Uniform integers in [0, n) from 64-bit draws (32-bit multiply-shift)."""
    return (((u >> np.uint64(32)) * np.asarray(n, np.uint64)) >> np.uint64(32)).astype(np.int64)


def _set_bits(q: np.ndarray):
    lo = np.where(q < 64, np.left_shift(np.uint64(1), (q % 64).astype(np.uint64)), np.uint64(0))
    hi = np.where(q >= 64, np.left_shift(np.uint64(1), (q % 64).astype(np.uint64)), np.uint64(0))
    return lo.astype(np.uint64), hi.astype(np.uint64)


def random_mix_fast(seed: int, nqubits: int, ngates: int, h_budget: int) -> np.ndarray:
    """Vectorised random mix for the batched workload: H on 8 distinct qubits,
    then `ngates` gates, each from six draws of the counter-based SplitMix64
    stream of `seed`: class u0 < 0.7 X/CNOT/Toffoli (1:1:1 by u1 % 3), < 0.9
    Z/S/T/controlled-Rz (1:1:1:1 by u1 % 4), else an H candidate. Only the
    first `h_budget` H candidates are kept (so 2^(8 + h_budget) bounds the
    nonzeros); a later one becomes X/CNOT/Toffoli or Z/S/T/CRz in the ratio
    7:2 by u1 % 9. Qubits: q0 = u2 below n, q1 = u3 below n-1 skipping q0,
    q2 = u4 below n-2 skipping both; angle = 2 pi (u5 >> 11) 2^-53."""
    n = nqubits
    rng = SplitMix64(seed)
    first = rng.distinct(n, min(8, n))
    u = splitmix_block(seed ^ 0x5DEECE66D, 6 * ngates).reshape(ngates, 6)
    f0 = (u[:, 0] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    kind = (u[:, 1] % np.uint64(36)).astype(np.int64)
    cls = np.where(f0 < 0.7, 0, np.where(f0 < 0.9, 1, 2))
    is_h = cls == 2
    h_rank = np.cumsum(is_h) - 1
    rejected = is_h & (h_rank >= h_budget)
    cls = np.where(rejected, np.where(kind % 9 < 7, 0, 1), cls)
    q0 = _below(u[:, 2], n)
    q1 = _below(u[:, 3], n - 1)
    q1 = q1 + (q1 >= q0)
    a, b = np.minimum(q0, q1), np.maximum(q0, q1)
    q2 = _below(u[:, 4], n - 2)
    q2 = q2 + (q2 >= a)
    q2 = q2 + (q2 >= b)
    theta = 2.0 * math.pi * (u[:, 5] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    g = np.zeros(ngates, dtype=GATE_DTYPE)
    op = np.zeros(ngates, np.uint8)
    t0 = np.zeros(ngates, np.int64)
    clo = np.zeros(ngates, np.uint64)
    chi = np.zeros(ngates, np.uint64)
    th = np.zeros(ngates, np.float64)
    # permutations: X(q0), CX(q0 -> q1), CCX(q0, q1 -> q2)
    pk = kind % 3
    perm = cls == 0
    op[perm] = OP_X
    t0[perm] = np.where(pk == 0, q0, np.where(pk == 1, q1, q2))[perm]
    l0, h0 = _set_bits(q0)
    l1, h1 = _set_bits(q1)
    m1 = perm & (pk >= 1)
    clo[m1] |= l0[m1]
    chi[m1] |= h0[m1]
    m2 = perm & (pk == 2)
    clo[m2] |= l1[m2]
    chi[m2] |= h1[m2]
    # diagonals: Z, S, T on q0; controlled Rz(theta) q0 -> q1
    dk = kind % 4
    diag = cls == 1
    op[diag] = np.array([OP_Z, OP_S, OP_T, OP_RZ], np.uint8)[dk[diag]]
    t0[diag] = np.where(dk == 3, q1, q0)[diag]
    m3 = diag & (dk == 3)
    clo[m3] |= l0[m3]
    chi[m3] |= h0[m3]
    th[m3] = theta[m3]
    # kept H candidates
    hk = cls == 2
    op[hk] = OP_H
    t0[hk] = q0[hk]
    g["op"] = op
    g["t0"] = t0.astype(np.uint16)
    g["cmask"][:, 0] = clo
    g["cmask"][:, 1] = chi
    g["theta"] = th
    return np.concatenate([to_array([H(q) for q in first]), g])


def batched_workload_fast(count: int = 4096, first_seed: int = 1, qubits=(20, 100),
                          depth=(200, 5000), log2_cap=(8, 16)) -> List[BatchCircuit]:
    """The batched workload: circuit s (seeds first_seed..) has qubits uniform
    on [qubits], depth uniform on [depth], nonzero cap 2^u with u uniform on
    [log2_cap], and the gates of :func:`random_mix_fast` with an H budget of
    floor(log2 cap) - 8 (so the nonzeros never exceed the cap)."""
    out = []
    for s in range(first_seed, first_seed + count):
        rng = SplitMix64(s * 0x2545F4914F6CDD1D + 7)
        nq = qubits[0] + rng.below(qubits[1] - qubits[0] + 1)
        d = depth[0] + rng.below(depth[1] - depth[0] + 1)
        cap = int(2.0 ** (log2_cap[0] + (log2_cap[1] - log2_cap[0]) * rng.uniform()))
        budget = max(0, int(math.floor(math.log2(cap))) - 8)
        out.append(BatchCircuit(s, nq, cap, random_mix_fast(s, nq, d, budget)))
    return out
