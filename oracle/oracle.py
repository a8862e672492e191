"""ctypes front end of the C++ oracle (test infrastructure only).

Gate lists are passed as contiguous numpy arrays of 32-byte records (the
layout documented in ``sps_oracle.cpp``); this module does not interpret them.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sps_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with g++ (-O2, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    u32, u64, dbl, vp, i32 = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                              ctypes.c_void_p, ctypes.c_int)
    pu64 = ctypes.POINTER(ctypes.c_uint64)
    lib.orc_create.argtypes = [u32]
    lib.orc_create.restype = vp
    lib.orc_destroy.argtypes = [vp]
    lib.orc_destroy.restype = None
    lib.orc_clone.argtypes = [vp]
    lib.orc_clone.restype = vp
    lib.orc_nqubits.argtypes = [vp]
    lib.orc_nqubits.restype = u32
    lib.orc_nnz.argtypes = [vp]
    lib.orc_nnz.restype = u64
    lib.orc_apply.argtypes = [vp, vp, u64, dbl, i32, pu64]
    lib.orc_apply.restype = i32
    lib.orc_apply_counted.argtypes = [vp, vp, u64, dbl, i32, pu64, pu64]
    lib.orc_apply_counted.restype = i32
    lib.orc_get.argtypes = [vp, vp, vp, vp, vp, u64]
    lib.orc_get.restype = i32
    lib.orc_set.argtypes = [vp, vp, vp, vp, vp, u64]
    lib.orc_set.restype = i32
    lib.orc_probability.argtypes = [vp, vp, vp]
    lib.orc_probability.restype = dbl
    lib.orc_pauli_exp.argtypes = [vp, vp, vp, vp, dbl, dbl]
    lib.orc_pauli_exp.restype = i32
    lib.orc_measure.argtypes = [vp, u32, dbl, vp]
    lib.orc_measure.restype = i32
    lib.orc_dense_run.argtypes = [u32, vp, u64, vp, vp]
    lib.orc_dense_run.restype = i32
    lib.orc_classical_eval.argtypes = [u32, vp, u64, vp, vp, u64, pu64]
    lib.orc_classical_eval.restype = i32
    lib.orc_sector_size.argtypes = [u32, u64]
    lib.orc_sector_size.restype = u64
    lib.orc_sector_run.argtypes = [u32, u64, vp, u64, vp, vp, vp, u64, pu64]
    lib.orc_sector_run.restype = i32
    _lib = lib
    return lib


def _gate_buffer(gates) -> np.ndarray:
    g = np.ascontiguousarray(gates)
    if g.size and g.dtype.itemsize != 32:
        raise ValueError("gate records must be 32 bytes each")
    return g


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else None


class OracleState:
    """Sparse state as a C++ unordered_map, updated gate by gate."""

    def __init__(self, nqubits: int, _handle=None):
        self._lib = _load()
        self._h = _handle if _handle is not None else self._lib.orc_create(nqubits)
        if not self._h:
            raise ValueError("nqubits must be in 1..127")

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            self._lib.orc_destroy(h)

    @property
    def nqubits(self) -> int:
        return int(self._lib.orc_nqubits(self._h))

    def clone(self) -> "OracleState":
        return OracleState(0, _handle=self._lib.orc_clone(self._h))

    def apply(self, gates, eps: float = 0.0, mode: int = 0) -> None:
        """Apply gate records in order. mode 0 = scatter, 1 = insert-once gather."""
        g = _gate_buffer(gates)
        bad = ctypes.c_uint64(0)
        rc = self._lib.orc_apply(self._h, _ptr(g), g.size, float(eps), int(mode),
                                 ctypes.byref(bad))
        if rc != 0:
            raise ValueError("invalid gate record at index %d" % bad.value)

    def apply_counted(self, gates, eps: float = 0.0, mode: int = 0) -> int:
        """As apply(); returns the sum over gates of the entries stored before
        each gate."""
        g = _gate_buffer(gates)
        bad = ctypes.c_uint64(0)
        upd = ctypes.c_uint64(0)
        rc = self._lib.orc_apply_counted(self._h, _ptr(g), g.size, float(eps), int(mode),
                                         ctypes.byref(bad), ctypes.byref(upd))
        if rc != 0:
            raise ValueError("invalid gate record at index %d" % bad.value)
        return int(upd.value)

    def nnz(self) -> int:
        return int(self._lib.orc_nnz(self._h))

    def get(self, sort: bool = True):
        """Return (hi, lo, re, im) arrays, sorted by (hi, lo) unless sort=False."""
        n = self.nnz()
        hi = np.empty(n, np.uint64)
        lo = np.empty(n, np.uint64)
        re = np.empty(n, np.float64)
        im = np.empty(n, np.float64)
        rc = self._lib.orc_get(self._h, _ptr(hi), _ptr(lo), _ptr(re), _ptr(im), n)
        assert rc == 0
        if sort and n:
            order = np.lexsort((lo, hi))
            hi, lo, re, im = hi[order], lo[order], re[order], im[order]
        return hi, lo, re, im

    def set(self, hi, lo, re, im) -> None:
        hi = np.ascontiguousarray(hi, np.uint64)
        lo = np.ascontiguousarray(lo, np.uint64)
        re = np.ascontiguousarray(re, np.float64)
        im = np.ascontiguousarray(im, np.float64)
        n = len(lo)
        assert len(hi) == len(re) == len(im) == n
        self._lib.orc_set(self._h, _ptr(hi), _ptr(lo), _ptr(re), _ptr(im), n)

    def probability(self, mask, value) -> float:
        m = np.ascontiguousarray(mask, np.uint64)
        v = np.ascontiguousarray(value, np.uint64)
        assert m.size == 2 and v.size == 2
        return float(self._lib.orc_probability(self._h, _ptr(m), _ptr(v)))


    def pauli_exp(self, x, z, controls, theta: float, eps: float = 0.0) -> None:
        """exp(-i theta/2 P) for the Pauli string with X-or-Y mask x and Z-or-Y
        mask z (two words each), under the control mask."""
        xs, zs, cs = (np.ascontiguousarray(v, np.uint64) for v in (x, z, controls))
        if self._lib.orc_pauli_exp(self._h, _ptr(xs), _ptr(zs), _ptr(cs), float(theta),
                                   float(eps)) != 0:
            raise ValueError("bad Pauli string")

    def measure(self, qubit: int, r: float):
        """Measures one qubit with collapse; returns (outcome, its probability)."""
        out = np.zeros(2, np.float64)
        if self._lib.orc_measure(self._h, int(qubit), float(r), _ptr(out)) != 0:
            raise ValueError("bad measurement argument")
        return int(out[0]), float(out[1])


def dense_run(nqubits: int, gates) -> np.ndarray:
    """Dense 2^n statevector of the circuit applied to |0...0> (complex128)."""
    lib = _load()
    g = _gate_buffer(gates)
    dim = 1 << nqubits
    re = np.empty(dim, np.float64)
    im = np.empty(dim, np.float64)
    rc = lib.orc_dense_run(nqubits, _ptr(g), g.size, _ptr(re), _ptr(im))
    if rc != 0:
        raise ValueError("dense_run: bad gate record or n out of range")
    return re + 1j * im


def classical_eval(nqubits: int, gates, hi, lo):
    """Push integer keys through an X/CNOT/Toffoli/MCX-only circuit."""
    lib = _load()
    g = _gate_buffer(gates)
    hi = np.array(hi, np.uint64, copy=True)
    lo = np.array(lo, np.uint64, copy=True)
    bad = ctypes.c_uint64(0)
    rc = lib.orc_classical_eval(nqubits, _ptr(g), g.size, _ptr(hi), _ptr(lo), len(lo),
                                ctypes.byref(bad))
    if rc != 0:
        raise ValueError("classical_eval: record %d is not a valid X gate" % bad.value)
    return hi, lo


def sector_run(nqubits: int, start: int, gates):
    """Dense simulation inside the weight sector of the basis state |start>
    (n <= 64): every label of that Hamming weight in increasing order and its
    amplitude (complex128, zeros included). Only Givens and diagonal gates
    (which conserve the weight) are accepted."""
    lib = _load()
    g = _gate_buffer(gates)
    size = int(lib.orc_sector_size(nqubits, start))
    if size == 0:
        raise ValueError("sector_run: n out of range")
    labels = np.empty(size, np.uint64)
    re = np.empty(size, np.float64)
    im = np.empty(size, np.float64)
    bad = ctypes.c_uint64(0)
    rc = lib.orc_sector_run(nqubits, start, _ptr(g), g.size, _ptr(labels), _ptr(re), _ptr(im),
                            size, ctypes.byref(bad))
    if rc == 1:
        raise ValueError("sector_run: record %d is invalid or leaves the sector" % bad.value)
    if rc != 0:
        raise ValueError("sector_run: bad size or start label")
    return labels, re + 1j * im
