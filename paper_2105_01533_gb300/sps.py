"""Thin ctypes binding of ``libsps.so`` (C ABI in ``include/sps.h``).

Argument marshalling only: every step of gate application runs in the CUDA
kernels of the library. The functions keep the C names (``sps_create``,
``sps_apply``, ...); :class:`SparseState` wraps them for convenience.

PyTorch supplies device memory (its caching allocator is installed as the
library's allocator hook) and streams (the current torch stream by default).
If ``libsps.so`` is missing this module raises: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import workloads

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsps.so")

SPS_OK, SPS_ERR_ARG, SPS_ERR_CAPACITY, SPS_ERR_TABLE_FULL = 0, 1, 2, 3
SPS_ERR_CUDA, SPS_ERR_OOM, SPS_ERR_NO_DEVICE, SPS_ERR_TIMEOUT = 4, 5, 6, 7
SPS_OPT_LOAD_FACTOR_PCT, SPS_OPT_PROBE_LIMIT, SPS_OPT_BLOCK_THREADS = 1, 2, 3
SPS_OPT_MAX_FUSED_OPS, SPS_OPT_COOP_WIDTH, SPS_OPT_PROFILE = 4, 5, 6
SPS_OPT_BITSLICE_MIN_OPS, SPS_OPT_SMALL_RUN_CAP, SPS_OPT_BITSLICE_MIN_NNZ = 7, 8, 9
SPS_OPT_BRANCH_FORM, SPS_OPT_BITSLICE_GROUPS, SPS_OPT_EXPAND, SPS_OPT_FOLD = 10, 11, 12, 13
SPS_OPT_COMMUTE, SPS_OPT_LAYER_GATES, SPS_OPT_EXPAND_WALK, SPS_OPT_FUSED_LABELS = 14, 15, 16, 17
SPS_OPT_AMP_ONLY, SPS_OPT_BITSLICE_JIT, SPS_OPT_PLAN_CACHE = 18, 19, 20
SPS_OPT_FALLBACK_CHAIN = 21
SPS_OPT_READOUT_MIN_PLANES = 22
KIND_SMALL_RUN, KIND_GATHER_BUILD, KIND_GATHER_EMIT = 4, 5, 6
KIND_FUSED, KIND_EMIT, KIND_COMPACT = 1, 2, 3

EXPORTS = ("sps_set_allocator", "sps_create", "sps_reset", "sps_destroy", "sps_apply", "sps_sync",
           "sps_nnz", "sps_get_amplitudes", "sps_set_amplitudes", "sps_probability",
           "sps_set_option", "sps_get_counters", "sps_profile_read", "sps_plan", "sps_status_str",
           "sps_branch_apply_static", "sps_batch_create", "sps_batch_destroy", "sps_batch_add",
           "sps_batch_run", "sps_batch_run_graph", "sps_batch_sync", "sps_batch_circuit_status",
           "sps_batch_get_amplitudes", "sps_batch_reset", "sps_batch_set_config",
           "sps_batch_get_config", "sps_batch_tune", "sps_batch_counts", "sps_batch_updates",
           "sps_get_updates", "sps_server_create", "sps_server_destroy", "sps_server_submit",
           "sps_server_tick", "sps_server_poll", "sps_server_result", "sps_server_stats",
           "sps_server_completed", "sps_probability_async", "sps_measure", "sps_pauli_exp",
           "sps_jit_selftest", "sps_device_rates", "sps_tune", "sps_tune_cache_lookup",
           "sps_barrier_selftest", "sps_set_readout",
           "sps_commute")


class SpsError(RuntimeError):
    def __init__(self, status: int, what: str, failed_gate: Optional[int] = None):
        self.status = status
        self.failed_gate = failed_gate
        msg = "%s: %s" % (what, _status_str(status))
        if failed_gate is not None:
            msg += " (gate %d)" % failed_gate
        super().__init__(msg)


class Counters(ctypes.Structure):
    _fields_ = [("gates", ctypes.c_uint64), ("fused_passes", ctypes.c_uint64),
                ("branch_passes", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("upload_bytes", ctypes.c_uint64), ("fused_readouts", ctypes.c_uint64)]


class KernelRecord(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("pass_serial", ctypes.c_uint32),
                ("ms", ctypes.c_float), ("nops", ctypes.c_uint32), ("n_in", ctypes.c_uint64),
                ("n_out", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("label_bytes", ctypes.c_uint32)]


class TuneChoice(ctypes.Structure):
    _fields_ = [("kw", ctypes.c_uint32), ("log2peak", ctypes.c_uint32),
                ("load_factor_pct", ctypes.c_uint32), ("bitslice_groups", ctypes.c_uint32),
                ("fused_labels", ctypes.c_uint32), ("max_fused_ops", ctypes.c_uint32),
                ("from_cache", ctypes.c_uint32), ("ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchConfig(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("smem_cap", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class ServerRequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int), ("failed_gate", ctypes.c_size_t),
                ("nnz", ctypes.c_uint64), ("submit_tick", ctypes.c_uint64),
                ("admit_tick", ctypes.c_uint64), ("done_tick", ctypes.c_uint64),
                ("large", ctypes.c_int), ("updates", ctypes.c_uint64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                           ctypes.c_void_p)

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libsps.so. Raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libsps.so is not built (%s); run paper_2105_01533_gb300.build" % path)
    lib = ctypes.CDLL(path)
    vp, u32, u64, sz, dbl, i64 = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                  ctypes.c_size_t, ctypes.c_double, ctypes.c_int64)
    st = ctypes.c_int
    psz = ctypes.POINTER(ctypes.c_size_t)
    pu64 = ctypes.POINTER(ctypes.c_uint64)
    lib.sps_set_allocator.argtypes = [ALLOC_FN, FREE_FN, vp]
    lib.sps_set_allocator.restype = st
    lib.sps_create.argtypes = [u32, u64, vp, ctypes.POINTER(vp)]
    lib.sps_create.restype = st
    lib.sps_reset.argtypes = [vp]
    lib.sps_reset.restype = st
    lib.sps_profile_read.argtypes = [vp, ctypes.POINTER(KernelRecord), sz, psz]
    lib.sps_profile_read.restype = st
    lib.sps_destroy.argtypes = [vp]
    lib.sps_destroy.restype = None
    lib.sps_apply.argtypes = [vp, vp, sz, dbl, psz]
    lib.sps_apply.restype = st
    lib.sps_sync.argtypes = [vp, psz]
    lib.sps_sync.restype = st
    lib.sps_nnz.argtypes = [vp, pu64]
    lib.sps_nnz.restype = st
    lib.sps_get_amplitudes.argtypes = [vp, vp, vp, vp, vp, u64, pu64]
    lib.sps_get_amplitudes.restype = st
    lib.sps_set_amplitudes.argtypes = [vp, vp, vp, vp, vp, u64]
    lib.sps_set_amplitudes.restype = st
    lib.sps_probability.argtypes = [vp, vp, vp, ctypes.POINTER(dbl)]
    lib.sps_probability.restype = st
    lib.sps_probability_async.argtypes = [vp, vp, vp, vp]
    lib.sps_probability_async.restype = st
    lib.sps_set_readout.argtypes = [vp, vp, vp]
    lib.sps_set_readout.restype = st
    lib.sps_measure.argtypes = [vp, u32, dbl, vp]
    lib.sps_measure.restype = st
    lib.sps_pauli_exp.argtypes = [vp, vp, vp, vp, dbl, dbl]
    lib.sps_pauli_exp.restype = st
    lib.sps_commute.argtypes = [vp, sz, u32, vp, sz, psz, psz]
    lib.sps_commute.restype = st
    lib.sps_set_option.argtypes = [vp, ctypes.c_int, i64]
    lib.sps_set_option.restype = st
    lib.sps_get_counters.argtypes = [vp, ctypes.POINTER(Counters)]
    lib.sps_get_counters.restype = st
    lib.sps_plan.argtypes = [vp, sz, u32, u32, vp, vp, vp, sz, psz, psz]
    lib.sps_plan.restype = st
    lib.sps_branch_apply_static.argtypes = [vp, u32, vp, vp, vp, vp, u64, dbl, vp, vp, vp, vp,
                                            u64, pu64, vp]
    lib.sps_branch_apply_static.restype = st
    lib.sps_batch_create.argtypes = [vp, ctypes.POINTER(vp)]
    lib.sps_batch_create.restype = st
    lib.sps_batch_destroy.argtypes = [vp]
    lib.sps_batch_destroy.restype = None
    lib.sps_batch_add.argtypes = [vp, u32, u64, vp, sz, dbl, ctypes.POINTER(u32), psz]
    lib.sps_batch_add.restype = st
    lib.sps_batch_run.argtypes = [vp, u32]
    lib.sps_batch_run.restype = st
    lib.sps_batch_run_graph.argtypes = [vp, u32]
    lib.sps_batch_run_graph.restype = st
    lib.sps_tune.argtypes = [vp, vp, sz, dbl, u32, ctypes.c_char_p, ctypes.POINTER(TuneChoice)]
    lib.sps_tune.restype = st
    lib.sps_tune_cache_lookup.argtypes = [ctypes.c_char_p, u32, u32, ctypes.POINTER(TuneChoice)]
    lib.sps_tune_cache_lookup.restype = st
    lib.sps_barrier_selftest.argtypes = [u32, u32, ctypes.POINTER(ctypes.c_int)]
    lib.sps_barrier_selftest.restype = st
    lib.sps_batch_sync.argtypes = [vp, ctypes.POINTER(u32)]
    lib.sps_batch_sync.restype = st
    lib.sps_batch_circuit_status.argtypes = [vp, u32, ctypes.POINTER(st), psz, pu64,
                                             ctypes.POINTER(ctypes.c_int)]
    lib.sps_batch_circuit_status.restype = st
    lib.sps_batch_get_amplitudes.argtypes = [vp, u32, vp, vp, vp, vp, u64, pu64]
    lib.sps_batch_get_amplitudes.restype = st
    lib.sps_batch_reset.argtypes = [vp]
    lib.sps_batch_reset.restype = st
    lib.sps_batch_set_config.argtypes = [vp, ctypes.POINTER(BatchConfig)]
    lib.sps_batch_set_config.restype = st
    lib.sps_batch_get_config.argtypes = [vp, ctypes.POINTER(BatchConfig)]
    lib.sps_batch_get_config.restype = st
    lib.sps_batch_tune.argtypes = [vp, u32, ctypes.POINTER(BatchConfig), ctypes.POINTER(ctypes.c_float)]
    lib.sps_batch_tune.restype = st
    lib.sps_batch_counts.argtypes = [vp, ctypes.POINTER(u32), pu64]
    lib.sps_batch_counts.restype = st
    lib.sps_batch_updates.argtypes = [vp, pu64]
    lib.sps_batch_updates.restype = st
    lib.sps_get_updates.argtypes = [vp, pu64]
    lib.sps_get_updates.restype = st
    lib.sps_server_create.argtypes = [u64, u32, u32, vp, ctypes.POINTER(vp)]
    lib.sps_server_create.restype = st
    lib.sps_server_destroy.argtypes = [vp]
    lib.sps_server_destroy.restype = None
    lib.sps_server_submit.argtypes = [vp, u32, u64, vp, sz, dbl, pu64, psz]
    lib.sps_server_submit.restype = st
    lib.sps_server_tick.argtypes = [vp, ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32)]
    lib.sps_server_tick.restype = st
    lib.sps_server_poll.argtypes = [vp, u64, ctypes.POINTER(ServerRequestInfo)]
    lib.sps_server_poll.restype = st
    lib.sps_server_result.argtypes = [vp, u64, vp, vp, vp, vp, u64, pu64]
    lib.sps_server_result.restype = st
    lib.sps_server_completed.argtypes = [vp, vp, sz, psz]
    lib.sps_server_completed.restype = st
    lib.sps_server_stats.argtypes = [vp, pu64, pu64, pu64]
    lib.sps_server_stats.restype = st
    lib.sps_status_str.argtypes = [st]
    lib.sps_status_str.restype = ctypes.c_char_p
    lib.sps_jit_selftest.argtypes = [vp, sz]
    lib.sps_jit_selftest.restype = ctypes.c_int
    lib.sps_device_rates.argtypes = [vp]
    lib.sps_device_rates.restype = st
    _lib = lib
    return lib


def _status_str(code: int) -> str:
    try:
        return load_library().sps_status_str(code).decode()
    except Exception:  # pragma: no cover - only when the library is absent
        return "status %d" % code


def _check(code: int, what: str, failed_gate: Optional[int] = None) -> None:
    if code != SPS_OK:
        raise SpsError(code, what, failed_gate)


def _ptr(a) -> Optional[int]:
    """Address of a numpy array or a torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data if a.size else None
    return a.data_ptr()  # torch.Tensor


def gate_array(gates) -> np.ndarray:
    g = np.ascontiguousarray(gates)
    if g.dtype != workloads.GATE_DTYPE:
        g = np.ascontiguousarray(g.astype(workloads.GATE_DTYPE))
    return g


# ---- torch as memory provider ---------------------------------------------------
_torch_hooks = None


def use_torch_allocator() -> bool:
    """Install torch's CUDA caching allocator as the device memory hook."""
    global _torch_hooks
    if _torch_hooks is not None:
        return True
    import torch
    if not torch.cuda.is_available():
        return False
    lib = load_library()

    def _alloc(ctx, nbytes, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream or 0))
        except Exception:
            return None

    def _free(ctx, ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(ptr)

    hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(lib.sps_set_allocator(hooks[0], hooks[1], None), "sps_set_allocator")
    _torch_hooks = hooks
    return True


def current_stream_handle() -> int:
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


# ---- C-named wrappers -------------------------------------------------------------
def sps_create(nqubits: int, capacity: int, stream: Optional[int] = None) -> int:
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.sps_create(nqubits, capacity, stream, ctypes.byref(h)), "sps_create")
    return h.value


def sps_reset(h: int) -> None:
    _check(load_library().sps_reset(h), "sps_reset")


def sps_profile_read(h: int, cap: int = 1 << 16):
    """Profiled launches since the last read, as a list of dicts."""
    recs = (KernelRecord * cap)()
    n = ctypes.c_size_t(0)
    _check(load_library().sps_profile_read(h, recs, cap, ctypes.byref(n)), "sps_profile_read")
    out = []
    for i in range(n.value):
        r = recs[i]
        out.append({"kind": r.kind, "pass": r.pass_serial, "ms": r.ms, "nops": r.nops,
                    "n_in": r.n_in, "n_out": r.n_out, "flags": r.flags,
                    "label_bytes": r.label_bytes})
    return out


def sps_destroy(h: int) -> None:
    load_library().sps_destroy(h)


def sps_apply(h: int, gates, prune_eps: float = 0.0) -> None:
    g = gate_array(gates)
    bad = ctypes.c_size_t(0)
    rc = load_library().sps_apply(h, _ptr(g), g.size, float(prune_eps), ctypes.byref(bad))
    _check(rc, "sps_apply", bad.value if rc == SPS_ERR_ARG else None)


def sps_sync(h: int) -> None:
    bad = ctypes.c_size_t(0)
    rc = load_library().sps_sync(h, ctypes.byref(bad))
    _check(rc, "sps_sync", bad.value if rc in (SPS_ERR_CAPACITY, SPS_ERR_TABLE_FULL) else None)


def sps_nnz(h: int) -> int:
    n = ctypes.c_uint64(0)
    _check(load_library().sps_nnz(h, ctypes.byref(n)), "sps_nnz")
    return n.value


def sps_get_amplitudes(h: int, key_hi, key_lo, re, im, cap: int) -> int:
    n = ctypes.c_uint64(0)
    rc = load_library().sps_get_amplitudes(h, _ptr(key_hi), _ptr(key_lo), _ptr(re), _ptr(im),
                                          cap, ctypes.byref(n))
    _check(rc, "sps_get_amplitudes")
    return n.value


def sps_set_amplitudes(h: int, key_hi, key_lo, re, im, n: int) -> None:
    _check(load_library().sps_set_amplitudes(h, _ptr(key_hi), _ptr(key_lo), _ptr(re), _ptr(im), n),
           "sps_set_amplitudes")


def sps_probability(h: int, mask: Sequence[int], value: Sequence[int]) -> float:
    m = np.array([int(mask[0]), int(mask[1])], np.uint64)
    v = np.array([int(value[0]), int(value[1])], np.uint64)
    p = ctypes.c_double(0.0)
    _check(load_library().sps_probability(h, _ptr(m), _ptr(v), ctypes.byref(p)), "sps_probability")
    return p.value


def sps_set_readout(h: int, mask: Optional[Sequence[int]], value: Optional[Sequence[int]]) -> None:
    """Register (mask, value) as the state's readout (None, None: clear it)."""
    if mask is None or value is None:
        _check(load_library().sps_set_readout(h, None, None), "sps_set_readout")
        return
    m = np.array([int(mask[0]), int(mask[1])], np.uint64)
    v = np.array([int(value[0]), int(value[1])], np.uint64)
    _check(load_library().sps_set_readout(h, _ptr(m), _ptr(v)), "sps_set_readout")


def sps_probability_async(h: int, mask: Sequence[int], value: Sequence[int], out_ptr: int) -> None:
    """Enqueue the probability; the double lands at out_ptr (pinned host or
    device memory) in stream order."""
    m = np.array([int(mask[0]), int(mask[1])], np.uint64)
    v = np.array([int(value[0]), int(value[1])], np.uint64)
    _check(load_library().sps_probability_async(h, _ptr(m), _ptr(v), ctypes.c_void_p(out_ptr)),
           "sps_probability_async")


def sps_measure(h: int, qubit: int, r: float, out_ptr: int) -> None:
    """Enqueue a measurement with collapse; {outcome, probability} land at out_ptr
    (two doubles, pinned host or device memory) in stream order."""
    _check(load_library().sps_measure(h, int(qubit), float(r), ctypes.c_void_p(out_ptr)),
           "sps_measure")


def sps_pauli_exp(h: int, x, z, controls, theta: float, eps: float = 0.0) -> None:
    xs, zs, cs = (np.array([int(v[0]), int(v[1])], np.uint64) for v in (x, z, controls))
    _check(load_library().sps_pauli_exp(h, _ptr(xs), _ptr(zs), _ptr(cs), float(theta), float(eps)),
           "sps_pauli_exp")


def sps_commute(gates, nqubits: int) -> np.ndarray:
    """Host-only gate commuting queues: the rewritten gate array (same state)."""
    g = gate_array(gates)
    cap = 4 * len(g) + 8
    out = np.zeros(cap, dtype=g.dtype)
    nout = ctypes.c_size_t(0)
    bad = ctypes.c_size_t(0)
    code = load_library().sps_commute(_ptr(g), len(g), nqubits, out.ctypes.data, cap,
                                      ctypes.byref(nout), ctypes.byref(bad))
    _check(code, "sps_commute", bad.value if code == SPS_ERR_ARG else None)
    return out[:nout.value].copy()


def sps_set_option(h: int, opt: int, value: int) -> None:
    _check(load_library().sps_set_option(h, opt, int(value)), "sps_set_option")


def sps_get_counters(h: int) -> Counters:
    c = Counters()
    _check(load_library().sps_get_counters(h, ctypes.byref(c)), "sps_get_counters")
    return c


def sps_plan(gates, nqubits: int, max_fused_ops: int = 0):
    """Host-only compilation: list of (kind, first_gate, nops); kind 1 = fused
    phase/permutation pass, 2 = branching pass."""
    lib = load_library()
    g = gate_array(gates)
    cap = max(len(g), 1)
    kind = np.zeros(cap, np.uint32)
    first = np.zeros(cap, np.uint64)
    ops = np.zeros(cap, np.uint32)
    npass = ctypes.c_size_t(0)
    bad = ctypes.c_size_t(0)
    rc = lib.sps_plan(_ptr(g), g.size, nqubits, max_fused_ops, _ptr(kind), _ptr(first), _ptr(ops),
                      cap, ctypes.byref(npass), ctypes.byref(bad))
    _check(rc, "sps_plan", bad.value if rc == SPS_ERR_ARG else None)
    n = npass.value
    return [(int(kind[i]), int(first[i]), int(ops[i])) for i in range(n)]


def sps_branch_apply_static(gate, nqubits: int, in_arrays, n_in: int, prune_eps: float,
                            out_arrays, out_cap: int, stream: Optional[int] = None) -> int:
    """One branching gate on caller-owned device arrays, without allocating.
    in_arrays / out_arrays: (hi, lo, re, im) device tensors (hi may be None
    below 64 qubits). Returns the output count."""
    g = gate_array(gate)
    if g.size != 1:
        raise ValueError("exactly one gate record")
    n = ctypes.c_uint64(0)
    ih, il, ir, ii = in_arrays
    oh, ol, orr, oi = out_arrays
    rc = load_library().sps_branch_apply_static(
        _ptr(g), nqubits, _ptr(ih), _ptr(il), _ptr(ir), _ptr(ii), n_in, float(prune_eps),
        _ptr(oh), _ptr(ol), _ptr(orr), _ptr(oi), out_cap, ctypes.byref(n), stream)
    _check(rc, "sps_branch_apply_static")
    return n.value


def sps_device_rates() -> dict:
    """Measured issue rates of the current device (lane operations per
    second): FP64 fma, FP32 fma, 3-input logic, 32-bit integer mad."""
    out = (ctypes.c_double * 4)()
    _check(load_library().sps_device_rates(out), "sps_device_rates")
    return {"fp64_fma": out[0], "fp32_fma": out[1], "lop3": out[2], "imad": out[3]}


def sps_tune_cache_lookup(path: str, kw: int, log2peak: int):
    """The choice recorded for a size class in a tuning cache file, or None
    (host only)."""
    c = TuneChoice()
    r = load_library().sps_tune_cache_lookup(path.encode(), kw, log2peak, ctypes.byref(c))
    return c.as_dict() if r == SPS_OK else None


def sps_barrier_selftest(skip_block: int, spins: int) -> int:
    """Status recorded by the cooperative launch's grid barrier with block
    skip_block missing its first arrival (>= 8: none misses)."""
    r = ctypes.c_int(-1)
    _check(load_library().sps_barrier_selftest(skip_block, spins, ctypes.byref(r)),
           "sps_barrier_selftest")
    return r.value


def sps_jit_selftest():
    """(ok, message): whether the runtime compiler builds the specialised
    bit-sliced kernel of a sample run (host only, no GPU needed)."""
    buf = ctypes.create_string_buffer(1 << 16)
    ok = load_library().sps_jit_selftest(buf, len(buf))
    return bool(ok), buf.value.decode(errors="replace")


def sps_status_str(code: int) -> str:
    return _status_str(code)


# ---- convenience class ----------------------------------------------------------
class SparseState:
    """A device-resident sparse state. ``stream`` is a cudaStream_t handle
    (int); by default the current torch stream."""

    def __init__(self, nqubits: int, capacity: int, stream: Optional[int] = None,
                 torch_memory: bool = True):
        if torch_memory:
            use_torch_allocator()
        if stream is None:
            stream = current_stream_handle()
        self.nqubits = nqubits
        self.capacity = capacity
        self.stream = stream
        self._h = sps_create(nqubits, capacity, stream)

    @property
    def handle(self) -> int:
        return self._h

    def close(self) -> None:
        h, self._h = getattr(self, "_h", None), None
        if h:
            sps_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def apply(self, gates, eps: float = 0.0) -> None:
        sps_apply(self._h, gates, eps)

    def tune(self, gates, eps: float = 0.0, repeats: int = 2, cache: Optional[str] = None) -> dict:
        """Time whole steps of `gates` under candidate settings of the plain
        path's tunable options and keep the fastest (sps_tune); with `cache`, a
        size class already recorded there is taken from the file."""
        g = gate_array(gates)
        c = TuneChoice()
        rc = load_library().sps_tune(self._h, _ptr(g), g.size, float(eps), repeats,
                                     cache.encode() if cache else None, ctypes.byref(c))
        _check(rc, "sps_tune")
        return c.as_dict()

    def sync(self) -> None:
        sps_sync(self._h)

    def reset(self) -> None:
        sps_reset(self._h)

    def profile_read(self):
        return sps_profile_read(self._h)

    def nnz(self) -> int:
        return sps_nnz(self._h)

    def updates(self) -> int:
        u = ctypes.c_uint64(0)
        _check(load_library().sps_get_updates(self._h, ctypes.byref(u)), "sps_get_updates")
        return u.value

    def set_option(self, opt: int, value: int) -> None:
        sps_set_option(self._h, opt, value)

    def counters(self) -> Counters:
        return sps_get_counters(self._h)

    def probability(self, mask, value) -> float:
        return sps_probability(self._h, mask, value)

    def probability_async(self, mask, value, out_ptr: int) -> None:
        """Enqueue the probability into out_ptr (pinned host or device memory)."""
        sps_probability_async(self._h, mask, value, out_ptr)

    def set_readout(self, mask=None, value=None) -> None:
        """Register a readout condition summed by a compiled expansion launch
        that ends an apply (None: clear it)."""
        sps_set_readout(self._h, mask, value)

    def pauli_exp(self, x, z, controls, theta: float, eps: float = 0.0) -> None:
        """exp(-i theta/2 P): x / z are the X-or-Y and Z-or-Y masks (two words)."""
        sps_pauli_exp(self._h, x, z, controls, theta, eps)

    def measure(self, qubit: int, r: float):
        """Measure one qubit with collapse (r uniform in [0, 1)); waits and
        returns (outcome, probability of the outcome)."""
        out = np.zeros(2, np.float64)
        sps_measure(self._h, qubit, r, out.ctypes.data)
        self.sync()
        return int(out[0]), float(out[1])

    def measure_async(self, qubit: int, r: float, out_ptr: int) -> None:
        """Enqueue a measurement; {outcome, probability} land at out_ptr."""
        sps_measure(self._h, qubit, r, out_ptr)

    def get_amplitudes(self, sort: bool = True):
        """(hi, lo, re, im) numpy arrays, sorted by (hi, lo) unless sort=False."""
        n = self.nnz()
        hi = np.empty(n, np.uint64)
        lo = np.empty(n, np.uint64)
        re = np.empty(n, np.float64)
        im = np.empty(n, np.float64)
        if n:
            sps_get_amplitudes(self._h, hi, lo, re, im, n)
        if sort and n:
            order = np.lexsort((lo, hi))
            hi, lo, re, im = hi[order], lo[order], re[order], im[order]
        return hi, lo, re, im

    def set_amplitudes(self, hi, lo, re, im) -> None:
        lo = np.ascontiguousarray(lo, np.uint64)
        hi = None if hi is None else np.ascontiguousarray(hi, np.uint64)
        re = np.ascontiguousarray(re, np.float64)
        im = np.ascontiguousarray(im, np.float64)
        sps_set_amplitudes(self._h, hi, lo, re, im, len(lo))


# ---- batched circuits -------------------------------------------------------------
class Batch:
    """Many independent circuits advanced by one persistent launch."""

    def __init__(self, stream: Optional[int] = None, torch_memory: bool = True):
        if torch_memory:
            use_torch_allocator()
        if stream is None:
            stream = current_stream_handle()
        self.stream = stream
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.sps_batch_create(stream, ctypes.byref(h)), "sps_batch_create")
        self._h = h.value
        self.n = 0

    @property
    def handle(self) -> int:
        return self._h

    def close(self) -> None:
        h, self._h = getattr(self, "_h", None), None
        if h:
            load_library().sps_batch_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, nqubits: int, capacity: int, gates, eps: float = 0.0) -> int:
        g = gate_array(gates)
        idx = ctypes.c_uint32(0)
        bad = ctypes.c_size_t(0)
        rc = load_library().sps_batch_add(self._h, nqubits, capacity, _ptr(g), g.size, float(eps),
                                          ctypes.byref(idx), ctypes.byref(bad))
        _check(rc, "sps_batch_add", bad.value if rc == SPS_ERR_ARG else None)
        self.n += 1
        return idx.value

    def run(self, max_passes: int = 0) -> None:
        _check(load_library().sps_batch_run(self._h, max_passes), "sps_batch_run")

    def run_graph(self, max_passes: int = 0) -> None:
        """Reset every circuit and advance it, as one replay of a captured
        CUDA graph (sps_batch_run_graph)."""
        _check(load_library().sps_batch_run_graph(self._h, max_passes), "sps_batch_run_graph")

    def sync(self) -> int:
        u = ctypes.c_uint32(0)
        _check(load_library().sps_batch_sync(self._h, ctypes.byref(u)), "sps_batch_sync")
        return u.value

    def reset(self) -> None:
        _check(load_library().sps_batch_reset(self._h), "sps_batch_reset")

    def status(self, index: int):
        st = ctypes.c_int(0)
        fg = ctypes.c_size_t(0)
        nnz = ctypes.c_uint64(0)
        fin = ctypes.c_int(0)
        _check(load_library().sps_batch_circuit_status(self._h, index, ctypes.byref(st),
                                                       ctypes.byref(fg), ctypes.byref(nnz),
                                                       ctypes.byref(fin)), "sps_batch_circuit_status")
        return {"status": st.value, "failed_gate": fg.value, "nnz": nnz.value,
                "finished": bool(fin.value)}

    def get_amplitudes(self, index: int, sort: bool = True):
        n = self.status(index)["nnz"]
        hi = np.empty(n, np.uint64)
        lo = np.empty(n, np.uint64)
        re = np.empty(n, np.float64)
        im = np.empty(n, np.float64)
        got = ctypes.c_uint64(0)
        if n:
            _check(load_library().sps_batch_get_amplitudes(self._h, index, _ptr(hi), _ptr(lo),
                                                           _ptr(re), _ptr(im), n,
                                                           ctypes.byref(got)),
                   "sps_batch_get_amplitudes")
        if sort and n:
            order = np.lexsort((lo, hi))
            hi, lo, re, im = hi[order], lo[order], re[order], im[order]
        return hi, lo, re, im

    def config(self) -> BatchConfig:
        c = BatchConfig()
        _check(load_library().sps_batch_get_config(self._h, ctypes.byref(c)), "sps_batch_get_config")
        return c

    def set_config(self, threads: int, blocks_per_sm: int, smem_cap: int) -> None:
        c = BatchConfig(threads, blocks_per_sm, smem_cap, 0)
        _check(load_library().sps_batch_set_config(self._h, ctypes.byref(c)), "sps_batch_set_config")

    def tune(self, repeats: int = 1):
        c = BatchConfig()
        ms = ctypes.c_float(0)
        _check(load_library().sps_batch_tune(self._h, repeats, ctypes.byref(c), ctypes.byref(ms)),
               "sps_batch_tune")
        return {"threads": c.threads, "blocks_per_sm": c.blocks_per_sm, "smem_cap": c.smem_cap,
                "ms": ms.value}

    def updates(self) -> int:
        t = ctypes.c_uint64(0)
        _check(load_library().sps_batch_updates(self._h, ctypes.byref(t)), "sps_batch_updates")
        return t.value

    def launches(self) -> int:
        n = ctypes.c_uint32(0)
        l = ctypes.c_uint64(0)
        _check(load_library().sps_batch_counts(self._h, ctypes.byref(n), ctypes.byref(l)),
               "sps_batch_counts")
        return l.value


# ---- serving --------------------------------------------------------------------
class Server:
    """Continuous batching of circuit requests (see include/sps.h)."""

    def __init__(self, mem_budget_bytes: int, max_active: int = 1024, passes_per_tick: int = 8,
                 stream: Optional[int] = None, torch_memory: bool = True):
        if torch_memory:
            use_torch_allocator()
        if stream is None:
            stream = current_stream_handle()
        h = ctypes.c_void_p()
        _check(load_library().sps_server_create(int(mem_budget_bytes), max_active, passes_per_tick,
                                                stream, ctypes.byref(h)), "sps_server_create")
        self._h = h.value

    def close(self) -> None:
        h, self._h = getattr(self, "_h", None), None
        if h:
            load_library().sps_server_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, nqubits: int, capacity: int, gates, eps: float = 0.0) -> int:
        g = gate_array(gates)
        rid = ctypes.c_uint64(0)
        bad = ctypes.c_size_t(0)
        rc = load_library().sps_server_submit(self._h, nqubits, capacity, _ptr(g), g.size,
                                              float(eps), ctypes.byref(rid), ctypes.byref(bad))
        _check(rc, "sps_server_submit", bad.value if rc == SPS_ERR_ARG else None)
        return rid.value

    def tick(self):
        a, p, d = ctypes.c_uint32(0), ctypes.c_uint32(0), ctypes.c_uint32(0)
        _check(load_library().sps_server_tick(self._h, ctypes.byref(a), ctypes.byref(p),
                                              ctypes.byref(d)), "sps_server_tick")
        return a.value, p.value, d.value

    def poll(self, rid: int) -> dict:
        info = ServerRequestInfo()
        _check(load_library().sps_server_poll(self._h, rid, ctypes.byref(info)), "sps_server_poll")
        return {"state": info.state, "status": info.status, "failed_gate": info.failed_gate,
                "nnz": info.nnz, "submit_tick": info.submit_tick, "admit_tick": info.admit_tick,
                "done_tick": info.done_tick, "large": bool(info.large), "updates": info.updates}

    def result(self, rid: int, sort: bool = True):
        n = self.poll(rid)["nnz"]
        hi = np.empty(n, np.uint64)
        lo = np.empty(n, np.uint64)
        re = np.empty(n, np.float64)
        im = np.empty(n, np.float64)
        got = ctypes.c_uint64(0)
        buf = lambda a: _ptr(a) if n else ctypes.c_void_p(1).value  # noqa: E731
        _check(load_library().sps_server_result(self._h, rid, buf(hi), buf(lo), buf(re), buf(im), n,
                                                ctypes.byref(got)), "sps_server_result")
        if sort and n:
            order = np.lexsort((lo, hi))
            hi, lo, re, im = hi[order], lo[order], re[order], im[order]
        return hi, lo, re, im

    def completed(self, cap: int = 65536):
        """Ids of the requests that finished in the last tick."""
        ids = np.zeros(cap, np.uint64)
        n = ctypes.c_size_t(0)
        _check(load_library().sps_server_completed(self._h, _ptr(ids), cap, ctypes.byref(n)),
               "sps_server_completed")
        return [int(x) for x in ids[:n.value]]

    def stats(self) -> dict:
        t, l, b = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
        _check(load_library().sps_server_stats(self._h, ctypes.byref(t), ctypes.byref(l),
                                               ctypes.byref(b)), "sps_server_stats")
        return {"ticks": t.value, "launches": l.value, "bytes_in_use": b.value}
