"""Benchmark: nonzero-amplitude updates/s of the sparse-state gate path.

Headline workload (default ``adder67-w24``, the larger-than-L2 reversible
arithmetic config): 67 qubits with 128-bit labels; H on the low 24 bits of
register a (16,777,216 nonzeros, a 537 MB state), X gates loading a seeded
32-bit constant into b, a 32-bit ripple-carry adder, 32 controlled-phase gates
on seeded pairs of a/b qubits, then the inverse adder; FP64 amplitudes, prune
eps 1e-14. Other workloads: ``adder67`` (a over 16 bits, L2-resident),
``adder67-w22``, ``givens64`` (64 qubits, 4 occupied modes, 500 Givens/CZ
layers), ``givens64-m5`` / ``givens64-m6`` (5 / 6 occupied modes, the
7,624,512- / 74,974,368-label sectors: a block of layers on a filled sector).

A step = reset to |0...0>, apply the whole gate stream (every branching pass
and fused phase/permutation pass), read the probability of one register value
back (registered with sps_set_readout: summed by the compiled expansion launch
when that launch ends the apply, else by the readout kernel; ``--fused-readout
0`` always takes the kernel). Updates per step U = sum over gates of the nonzero
count before the gate. ``value`` = U * steps / (sum of per-step device times);
L2 is flushed (a 512 MB write) between timed steps, outside the timed events.
The default run adds sub-lines for the other configs, the batched and the
served forms.

``--impl reference`` times the CPU oracle (the only reference this method has)
on a bounded sample of the same workload on the host cores.

Prints one JSON line on rank 0.
"""

from __future__ import annotations

import argparse
import hashlib
import math
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2105_01533_gb300 import workloads as W  # noqa: E402

METRIC = "nonzero-amplitude updates/s"
UNIT = "updates/s"
EPS = 1e-14
L2_FLUSH_BYTES = 512 << 20


# ---- workloads -------------------------------------------------------------------
def make_workload(name: str):
    """A workload: its gates, qubits, capacity and readout. Block workloads
    (``block`` set) prepare a state with ``prep`` untimed and time applies of
    ``block`` on it."""
    if name == "adder67":
        wl = W.adder_workload(seed=1, width=16)
        return dict(name=name, gates=wl.gates, nqubits=wl.layout.nqubits, capacity=1 << 17,
                    readout=((0xFFFF, 0), (0, 0)),
                    desc="adder67: 67 qubits, 128-bit labels, H on a[0..15] (65,536 nonzeros), "
                         "32-bit ripple-carry adder, 32 CP gates, inverse adder; FP64, eps 1e-14")
    if name == "adder67-w24":
        wl = W.adder_workload(seed=1, width=24)
        return dict(name=name, gates=wl.gates, nqubits=wl.layout.nqubits, capacity=1 << 25,
                    readout=((0xFFFF, 0), (0, 0)),
                    desc="adder67-w24: 67 qubits, 128-bit labels, H on a[0..23] (16,777,216 "
                         "nonzeros, 537 MB state), 32-bit ripple-carry adder, 32 CP gates, inverse "
                         "adder; FP64, eps 1e-14")
    if name == "adder67-w22":
        wl = W.adder_workload(seed=1, width=22)
        return dict(name=name, gates=wl.gates, nqubits=wl.layout.nqubits, capacity=1 << 22,
                    readout=((0xFFFF, 0), (0, 0)),
                    desc="adder67-w22: as adder67 with a over 22 bits (4,194,304 nonzeros, "
                         "134 MB state); profiling size")
    if name == "givens64":
        g = W.givens_workload(seed=2, nqubits=64, modes=4, layers=500)
        return dict(name=name, gates=g, nqubits=64, capacity=700_000,
                    readout=((0xFF, 0), (0x0F, 0)),
                    desc="givens64: 64 qubits, 4 occupied modes (<= 635,376 nonzeros), 500 layers "
                         "of 32 Givens + 32 CZ; FP64, eps 1e-14")
    if name in ("givens64-m5", "givens64-m6"):
        modes = 5 if name.endswith("m5") else 6
        prep_layers, block_layers = 12, (8 if modes == 5 else 4)
        g = W.givens_workload(seed=2, nqubits=64, modes=modes, layers=prep_layers + block_layers)
        cut = modes + 64 * prep_layers
        size = math.comb(64, modes)
        return dict(name=name, gates=g[cut:], prep=g[:cut], nqubits=64,
                    capacity=size + 4096, readout=((0xFF, 0), (0x1F, 0)), block=True,
                    desc="%s: 64 qubits, %d occupied modes (the %s-label sector, %d MB); a step "
                         "applies %d layers of 32 Givens + 32 CZ to the state left by %d seeded "
                         "layers (untimed); FP64, eps 1e-14" % (
                             name, modes, "{:,}".format(size), size * 32 >> 20, block_layers,
                             prep_layers))
    raise SystemExit("unknown workload %s" % name)


# ---- distributed plumbing --------------------------------------------------------
def dist_init(ngpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        dist.init_process_group(backend=backend)
        return dist, int(os.environ.get("RANK", "0")), world, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---- clocks ----------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id_for_smi() -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        u = u if u.startswith("GPU-") else "GPU-" + u
        out = subprocess.run(["nvidia-smi", "--query-gpu=uuid", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout
        if u in out:
            return u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    return vis.split(",")[torch.cuda.current_device()] if vis else str(torch.cuda.current_device())


# ---- roofline ----------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


KIND_NAMES = {1: "k_fused", 2: "k_branch_emit", 3: "k_branch_compact", 4: "k_small_run",
              5: "k_gather_build", 6: "k_gather_emit", 7: "k_expand", 8: "k_measure",
              9: "k_amp_index", 10: "k_amp_layer", 11: "k_chain", 12: "k_probability"}
MOVED_ACCOUNTING = ("bytes the launch must move: B*n read and written by a fused pass that "
                    "permutes and changes phases (labels only or amplitudes only when it does "
                    "one of the two), B*(n_in + n_out) by a branching pass or an expansion, "
                    "(B + 16)*n by an amplitude-only run (labels read, amplitudes read and "
                    "written); B = 24 or 32 bytes per entry")
ACCOUNTING = ("bytes of the method's passes: 2*B*n per fused phase/permutation pass, "
              "B*(n_in + n_out) per branching pass, B = 24 (64-bit labels) or 32 (128-bit) "
              "bytes per entry; index builds count the labels they read")


def kernel_name(r) -> str:
    if r["kind"] == 7 and r["flags"] & 16:   # expansion and bit-sliced run, compiled together
        return "k_bs_jit_expand"
    if r["kind"] == 1 and r["flags"] & 16:
        return "k_bs_jit"
    if r["kind"] == 1 and r["flags"] & 8:
        return "k_fused_bs"
    return KIND_NAMES[r["kind"]]


def algorithmic_bytes(r) -> float:
    """Bytes of the passes of the method one launch carries out: a fused
    phase/permutation pass reads and writes the state (2*B*n), a branching
    pass reads the old state and writes the new one (B*(n_in + n_out)); a
    launch that carries out several passes (an expansion of d gates, an
    amplitude-only run of d gates, a layer) is credited with each of them."""
    lb = r["label_bytes"]
    B = lb + 16
    k, n_in, n_out, d = r["kind"], r["n_in"], r["n_out"], max(1, r["nops"])
    if k == 1:
        return 2.0 * B * n_in
    if k == 7:   # d gates, each doubling the entries: B * (m + 2m) for m = n_in, 2 n_in, ...
        b = 3.0 * B * n_in * ((1 << min(d, 60)) - 1)
        if r["flags"] & 4:   # and the fused run walked on its outputs
            b += 2.0 * B * n_out
        return b
    if k == 10:   # d gates on a state whose labels stay (n_out > 0: the attempt took them)
        b = 2.0 * B * n_out * d
        if r["flags"] & 4:
            b += 2.0 * B * n_out
        return b
    if k == 6 and d > 1 and n_in > 0:   # a layer: d passes from n_in to n_out entries
        q = (n_out / n_in) ** (1.0 / d) if n_out > 0 else 1.0
        return sum(B * n_in * q ** j * (1.0 + q) for j in range(d))
    if k in (5, 9):   # label index of a gather or amplitude-only pass
        return float(lb * n_in)
    if k == 11:   # an attempted run's d passes (none when the attempt took it: n_in 0)
        return float(B * (n_in + n_out) * d) if n_in > 0 else 0.0
    if k == 12:   # readout: the labels (and the matching entries' amplitudes) read
        return float(lb * n_in)
    if k == 2:
        return float(B * n_in)
    if k == 3:
        return float(B * n_out)
    return float(B * (n_in + n_out))


def moved_bytes(r) -> float:
    """The least traffic the launch itself needs: every entry it reads read
    once, every entry it writes written once."""
    lb = r["label_bytes"]
    B = lb + 16
    k, n_in, n_out = r["kind"], r["n_in"], r["n_out"]
    if k == 1:
        return float((lb + (lb if r["flags"] & 1 else 0) + (32 if r["flags"] & 2 else 0)) * n_in)
    if k == 10:   # labels stay: amplitudes read and written, labels read by the lookups
        return float((32 + lb) * n_out)
    return algorithmic_bytes(r) if k in (2, 3, 5, 9, 11, 12) else float(B * (n_in + n_out))


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_2105_01533_gb300", "csrc"))):
        with open(os.path.join(ROOT, "paper_2105_01533_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str, n_per_launch: float):
    """DRAM bytes per launch from the committed ncu summary, scaled to this
    launch size, or None if the summary is missing or the kernels changed."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(kernel, {}).get(workload)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e["dram_bytes_per_entry"] * n_per_launch


def roofline(records, workload: str, steps: int):
    """The dominant kernel (by time over `steps` profiled steps) against the
    HBM roofline: the bytes a launch must move (every entry it reads read once,
    every entry it writes written once) over its average launch time. The
    bytes of the method's passes the launch carries out (2*B*n per fused pass,
    B*(n_in + n_out) per branching pass) are reported beside it: a launch that
    does several passes without writing the states between them is credited
    with more bytes than it moves, so that figure is a rate of work, not a
    fraction of the memory bound."""
    peak, which = measured_peaks()
    by = {}
    for r in records:
        b = by.setdefault(kernel_name(r), {"ms": 0.0, "bytes": 0.0, "moved": 0.0, "n": 0,
                                           "entries": 0})
        b["ms"] += r["ms"]
        b["bytes"] += algorithmic_bytes(r)
        b["moved"] += moved_bytes(r)
        b["n"] += 1
        # entries a launch processes: outputs for a compaction or an expansion
        b["entries"] += r["n_out"] if r["kind"] in (3, 7, 10) else r["n_in"]
    total = sum(b["ms"] for b in by.values()) or 1.0
    kern = max(by, key=lambda k: by[k]["ms"])
    b = by[kern]
    avg_ms = b["ms"] / b["n"]
    moved = b["moved"] / b["n"]
    method = b["bytes"] / b["n"]
    achieved = moved / (avg_ms * 1e-3) / 1e9
    method_rate = method / (avg_ms * 1e-3) / 1e9
    share = {k: round(v["ms"] / total, 4) for k, v in by.items()}
    traffic = ncu_traffic(kern, workload, b["entries"] / b["n"])
    return {"bound": "hbm", "kernel": kern, "achieved": round(achieved, 2), "peak": peak,
            "peak_source": which + " (MEASURED_PEAKS.json hbm_gbs)" if which == "measured"
            else "fallback 6800 GB/s", "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": traffic, "bytes_per_launch": round(moved),
            "accounting": MOVED_ACCOUNTING,
            "method_passes": {"bytes_per_launch": round(method), "rate": round(method_rate, 2),
                              "unit": "GB/s", "accounting": ACCOUNTING},
            "avg_launch_ms": round(avg_ms, 5),
            "launches_per_step": round(b["n"] / max(1, steps), 2),
            "time_share": share}


# ---- our arm ---------------------------------------------------------------------
def updates_per_step(sps, wl, st) -> tuple:
    """Untimed: nonzeros before every gate, from the product path itself."""
    plan = sps.sps_plan(wl["gates"], wl["nqubits"])
    bounds = [p[1] for p in plan] + [len(wl["gates"])]
    st.reset()
    u = 0
    nnz = 1
    for j, (kind, first, _) in enumerate(plan):
        u += nnz * (bounds[j + 1] - first)
        st.apply(wl["gates"][first:bounds[j + 1]], EPS)
        nnz = st.nnz()
    return u, nnz


def profiled_steps(sps, torch, st, step, flush, stream, nsteps):
    """Per-kernel records of `nsteps` steps, every launch bracketed by CUDA
    events on the state's stream (kept out of the headline timing)."""
    st.set_option(sps.SPS_OPT_PROFILE, 1)
    st.profile_read()
    records = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(nsteps)]
    for i in range(nsteps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        records += st.profile_read()
    torch.cuda.synchronize()
    st.set_option(sps.SPS_OPT_PROFILE, 0)
    return records, sum(a.elapsed_time(b) for a, b in ev) / max(1, nsteps)


def run_ours(args, dist, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2105_01533_gb300 import sps

    wl = make_workload(args.workload)
    st = sps.SparseState(wl["nqubits"], wl["capacity"])
    for kv in args.opt:
        name, val = kv.split("=")
        st.set_option(getattr(sps, "SPS_OPT_" + name.upper()), int(val))
    stream = torch.cuda.current_stream()
    U, nnz_final = updates_per_step(sps, wl, st)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    mask, val = wl["readout"]
    if args.fused_readout:   # summed by the launch that ends the apply, where it can be
        st.set_readout(mask, val)
    # each step's readout lands in its own pinned slot, in stream order: the host
    # does not wait for step i before enqueueing step i + 1
    nslots = args.warmup + args.steps + min(args.steps, 20)
    probs = torch.full((nslots,), float("nan"), dtype=torch.float64, pin_memory=True)
    slot = [0]

    def step():
        st.reset()
        st.apply(wl["gates"], EPS)
        st.probability_async(mask, val, probs.data_ptr() + 8 * slot[0])
        slot[0] += 1

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_id_for_smi()) if rank == 0 else None
    barrier(dist)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    c0 = st.counters().kernel_launches
    f0 = st.counters().fused_readouts
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if args.profile_range:   # a profiler started with capture off records the timed steps only
        torch.cuda.profiler.start()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.profiler.stop()
    launches = st.counters().kernel_launches - c0
    fused = st.counters().fused_readouts - f0
    st.sync()   # raises if any timed step failed on the device
    p = probs[:slot[0]].numpy()
    if not np.all(np.abs(p - p[0]) <= 1e-9):
        raise SystemExit("readouts of identical steps differ: %r" % p[:8])
    # the same state read by the readout kernel
    st.set_readout(None, None)
    p_kernel = st.probability(mask, val)
    if abs(p_kernel - p[0]) > 1e-13:
        raise SystemExit("fused readout %r differs from the readout kernel's %r" % (p[0], p_kernel))
    readout = {"probability": float(p[0]), "kernel_probability": p_kernel,
               "fused_per_step": round(fused / args.steps, 3),
               "what": "sum of |a|^2 over labels with (label & mask) == value; fused: formed by "
                       "the compiled expansion launch as it stores the outputs "
                       "(sps_set_readout), else the readout kernel"}
    if args.fused_readout:
        st.set_readout(mask, val)
    barrier(dist)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(b) for a, b in ev]

    prof_steps = min(args.steps, 20)
    records, prof_ms = profiled_steps(sps, torch, st, step, flush, stream, prof_steps)
    if args.dump_profile and rank == 0:
        per_step = len(records) // prof_steps
        with open(args.dump_profile, "w") as f:
            json.dump({"workload": wl["name"], "options": args.opt,
                       "step_records": records[-per_step:] if per_step else []}, f, indent=1)
    total_ms = max_over_ranks(dist, sum(step_ms))
    units = sum_over_ranks(dist, float(U) * args.steps)
    value = units / (total_ms * 1e-3)

    # end to end through the public API with host buffers
    e2e = run_e2e(args, sps, torch, wl, st, flush, U, dist)

    rl = roofline(records, wl["name"], prof_steps)
    rl["profiled_steps"] = prof_steps
    rl["profiled_ms_per_step"] = round(prof_ms, 5)
    res = None
    if rank == 0:
        res = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": round(total_ms / args.steps, 5), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": wl["desc"], "nqubits": wl["nqubits"],
                          "gates": int(len(wl["gates"])), "nnz_final": int(nnz_final),
                          "updates_per_step": int(U), "prune_eps": EPS,
                          "l2": "flushed between timed steps (512 MB write)",
                          "parallelism": "replicas" if world > 1 else "single"},
               "roofline": rl, "e2e": e2e, "gpu_launches": int(launches * world),
               "readout": readout,
               "device_rates": device_rates(sps),
               "clocks": clocks, "p50_step_ms": round(float(np.median(step_ms)), 5),
               "p99_step_ms": round(float(np.percentile(step_ms, 99)), 5)}
        if world == 1 and not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline(wl, budget_s=args.cpu_seconds)
    st.close()
    del flush
    if args.sublines and rank == 0:
        subs = {}
        for name in args.sublines.split(","):
            if name and name != wl["name"]:
                subs[name] = run_sub(args, sps, torch, name)
        if res is not None:
            res["sublines"] = subs
    if args.branch_forms and rank == 0:
        bf = branch_forms(args, sps, torch)
        if res is not None:
            res["branch_forms"] = bf
    if args.batched:
        bres = run_batched(args, sps, torch, args.batch_count, steps=args.batch_steps,
                           warmup=1, dist=dist, rank=rank, world=world)
        if res is not None:
            res["batched"] = bres
    if args.served and rank == 0:
        sres = run_served(args, sps, torch, args.serve_count, args.serve_seconds)
        if res is not None:
            res["served"] = sres
    return res


def device_rates(sps) -> dict:
    """Issue rates measured by the library's probe (lane operations per second):
    the denominators for kernels bound by FP64 or by instruction issue."""
    try:
        r = sps.sps_device_rates()
    except Exception as e:   # a measurement aid: never fail the bench line for it
        return {"error": str(e)}
    return {k: round(v / 1e9, 1) for k, v in r.items()} | {"unit": "G lane-ops/s"}


def branch_forms(args, sps, torch):
    """One branching-heavy workload under the gather form (the paper's
    insert-once rule: index, look up, write each pair once) and the scatter form
    (atomic accumulation into a 128-bit open-addressing table) with 1 and 4
    lanes probing each insert: 40 qubits, H on 20 of them (1,048,576 nonzeros),
    then 24 Ry / controlled-Ry / Givens gates on the same qubits (labels meet
    partners; nothing grows), one pass per gate (no layers, no amplitude-only
    runs). Per-pass time by CUDA events over whole applies."""
    from paper_2105_01533_gb300 import workloads as W
    rng = W.SplitMix64(31)
    recs = [W.H(q) for q in range(20)]
    for _ in range(24):
        q = rng.distinct(20, 3)
        k = rng.below(3)
        if k == 0:
            recs.append(W.Ry(q[0], rng.angle()))
        elif k == 1:
            recs.append(W.Ry(q[0], rng.angle(), q[1]))
        else:
            recs.append(W.Givens(q[0], q[1], rng.angle()))
    gates = W.to_array(recs)
    stream = torch.cuda.current_stream()
    out = {}
    for name, opts in (("gather", [(sps.SPS_OPT_BRANCH_FORM, 2)]),
                       ("scatter_w1", [(sps.SPS_OPT_BRANCH_FORM, 1), (sps.SPS_OPT_COOP_WIDTH, 1)]),
                       ("scatter_w4", [(sps.SPS_OPT_BRANCH_FORM, 1), (sps.SPS_OPT_COOP_WIDTH, 4)])):
        st = sps.SparseState(40, 1 << 21)
        for o, v in opts + [(sps.SPS_OPT_LAYER_GATES, 1), (sps.SPS_OPT_AMP_ONLY, 0)]:
            st.set_option(o, v)
        prep = gates[:20]
        body = gates[20:]
        times = []
        for rep_i in range(4):
            st.reset()
            st.apply(prep, EPS)
            st.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st.apply(body, EPS)
            e1.record(stream)
            st.sync()
            if rep_i:
                times.append(e0.elapsed_time(e1))
        n = st.nnz()
        st.close()
        out[name] = {"ms_per_pass": round(float(np.median(times)) / len(body), 4), "nnz": int(n)}
    out["workload"] = ("40 qubits, H on 20 (1,048,576 nonzeros), 24 Ry / CRy / Givens on those "
                       "qubits, one pass per gate; FP64, eps 1e-14")
    return out


def run_sub(args, sps, torch, name: str):
    """One more config on its own state: the same step (or, for a block
    workload, applies of the block on the prepared state), its own roofline."""
    wl = make_workload(name)
    st = sps.SparseState(wl["nqubits"], wl["capacity"])
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    mask, val = wl["readout"]
    if args.fused_readout:
        st.set_readout(mask, val)
    out = torch.zeros(4096, dtype=torch.float64, device="cuda")
    slot = [0]
    block = wl.get("block", False)
    t0 = time.perf_counter()
    if block:
        st.apply(wl["prep"], EPS)
        st.sync()

    def step():
        if not block:
            st.reset()
        st.apply(wl["gates"], EPS)
        st.probability_async(mask, val, out.data_ptr() + 8 * (slot[0] % 4096))
        slot[0] += 1

    warm = 2 if block else 3
    for _ in range(warm):
        step()
    torch.cuda.synchronize()
    prep_s = time.perf_counter() - t0
    steps = args.sub_steps
    u0 = st.updates()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    c0 = st.counters().kernel_launches
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    launches = st.counters().kernel_launches - c0
    U = st.updates() - u0 if block else None
    if not block:   # the update counter restarts at each reset: one step's count
        U = st.updates() * steps
    nnz = st.nnz()
    ms = [a.elapsed_time(b) for a, b in ev]
    prof = min(steps, 3)
    records, prof_ms = profiled_steps(sps, torch, st, step, flush, stream, prof)
    st.close()
    del flush
    total = sum(ms)
    rl = roofline(records, name, prof)
    rl["profiled_steps"] = prof
    return {"workload": wl["desc"], "value": round(U / (total * 1e-3), 1), "unit": UNIT,
            "ms_per_step": round(total / steps, 5), "steps": steps,
            "updates_per_step": int(U // steps), "nnz": int(nnz),
            "gpu_launches_per_step": round(launches / steps, 1), "roofline": rl,
            "p50_step_ms": round(float(np.median(ms)), 5),
            "min_step_ms": round(float(np.min(ms)), 5), "max_step_ms": round(float(np.max(ms)), 5),
            "prepare_s": round(prep_s, 2)}


def run_e2e(args, sps, torch, wl, st, flush, U, dist):
    """Same metric through the public calls with host buffers: every step
    compiles the gate records from host memory and uploads the plan from pinned
    staging (the apply-plan cache is off, so nothing of the previous step is
    reused), and copies the step's result (the probability) to pinned host
    memory. Two loops: steps enqueued back to back, every result on the host
    when the clock stops (the host compiles step i + 1 while the GPU runs step
    i: the throughput a caller with many circuits sees), and steps one at a
    time, each result read before the next step starts (`serial`)."""
    mask, val = wl["readout"]
    st.set_option(sps.SPS_OPT_PLAN_CACHE, 0)
    for _ in range(3):
        st.reset()
        st.apply(wl["gates"], EPS)
        st.probability(mask, val)
    # back to back
    k = max(8, args.steps)
    res = torch.full((k,), float("nan"), dtype=torch.float64, pin_memory=True)
    b0 = st.counters().upload_bytes
    torch.cuda.synchronize()
    barrier(dist)
    t0 = time.perf_counter()
    for i in range(k):
        st.reset()
        st.apply(wl["gates"], EPS)
        st.probability_async(mask, val, res.data_ptr() + 8 * i)
    st.sync()   # every step's result is in pinned host memory
    total = time.perf_counter() - t0
    up = (st.counters().upload_bytes - b0) / k
    r = res.numpy()
    if not (np.all(np.isfinite(r)) and np.all(np.abs(r - r[0]) <= 1e-9)):
        raise SystemExit("end-to-end readouts differ: %r" % r[:8])
    # one at a time
    ks = max(3, args.steps // 4)
    serial = 0.0
    for _ in range(ks):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        st.reset()
        st.apply(wl["gates"], EPS)
        st.probability(mask, val)
        serial += time.perf_counter() - t1
    st.set_option(sps.SPS_OPT_PLAN_CACHE, 1)
    total = max_over_ranks(dist, total)
    serial = max_over_ranks(dist, serial)
    units = sum_over_ranks(dist, float(U) * k)
    units_s = sum_over_ranks(dist, float(U) * ks)
    return {"value": round(units / total, 1), "unit": UNIT,
            "h2d_bytes_per_step": int(up), "d2h_bytes_per_step": 8,
            "gate_record_bytes": int(wl["gates"].nbytes), "steps": k,
            "ms_per_step": round(1e3 * total / k, 5),
            "what": "steps enqueued back to back: reset, sps_apply of host gate records "
                    "(compiled and the plan uploaded from pinned staging each step), "
                    "sps_probability_async into pinned host memory; wall clock from the first "
                    "enqueue until every result is on the host (state larger than L2, no flush)",
            "serial": {"value": round(units_s / serial, 1), "unit": UNIT, "steps": ks,
                       "ms_per_step": round(1e3 * serial / ks, 5),
                       "what": "one step at a time: the same calls with sps_probability, "
                               "the result read before the next step; L2 flushed before "
                               "each step, outside the clock"}}


# ---- batched form -----------------------------------------------------------------------
def run_batched(args, sps, torch, count: int, steps: int, warmup: int, sample_every: int = 32,
                dist=None, rank: int = 0, world: int = 1):
    """4,096 independent circuits (qubits 20..100, depth 200..5000, caps
    2^8..2^16) in one persistent launch per step, against the plain per-circuit
    path on every `sample_every`-th circuit of the same set. With several ranks
    each runs its longest-processing-time share; only totals are reduced."""
    from paper_2105_01533_gb300 import shard
    from paper_2105_01533_gb300 import workloads as W
    t0 = time.perf_counter()
    circs = W.batched_workload_fast(count, first_seed=1)
    if world > 1:
        circs = shard.my_share(circs, rank, world)
    gen_s = time.perf_counter() - t0
    b = sps.Batch()
    for c in circs:
        b.add(c.nqubits, c.cap, c.gates, EPS)
    tuned = b.tune(repeats=1)
    stream = torch.cuda.current_stream()
    # a step (every circuit reset, then the persistent launch) is one replay of
    # a captured CUDA graph
    for _ in range(max(1, warmup)):
        b.run_graph()
        b.sync()
    upd = b.updates()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for i in range(steps):
        ev[i][0].record(stream)
        b.run_graph()
        ev[i][1].record(stream)
        left = b.sync()
        assert left == 0
    ms = [a.elapsed_time(e) for a, e in ev]
    failed = sum(1 for i in range(len(circs)) if b.status(i)["status"] != 0)
    # the same launches timed by the host clock (the clock the plain path uses)
    torch.cuda.synchronize()
    tw = time.perf_counter()
    for i in range(steps):
        b.run_graph()
        b.sync()
    wall_s = time.perf_counter() - tw
    b.close()
    tot_upd, tot_s = shard.reduce_totals(float(upd) * steps, sum(ms) * 1e-3)
    batched_rate = tot_upd / tot_s
    batched_wall_rate = float(upd) * steps / wall_s
    # the plain path on a sample of the same circuits, one circuit at a time
    sample = circs[::sample_every]
    sb = sps.Batch()
    for c in sample:
        sb.add(c.nqubits, c.cap, c.gates, EPS)
    sb.run()
    sb.sync()
    upd_s = sb.updates()
    sb.close()
    states = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in sample:
        st = states.get((c.nqubits, c.cap))
        if st is None:
            st = states[(c.nqubits, c.cap)] = sps.SparseState(c.nqubits, c.cap)
        st.reset()
        st.apply(c.gates, EPS)
        st.sync()
    plain_s = time.perf_counter() - t0
    for st in states.values():
        st.close()
    plain_rate = upd_s / plain_s
    cpu = batch_cpu_baseline(circs, args.batch_cpu_every) if rank == 0 and args.batch_cpu_every else None
    return {"workload": "batched%d: qubits U{20..100}, depth U{200..5000}, caps 2^U[8,16], "
                        "mix 70%% X/CNOT/Toffoli, 20%% Z/S/T/CRz, 10%% H within the cap; FP64, "
                        "eps 1e-14" % count,
            "circuits": count, "gates": int(sum(len(c.gates) for c in circs)),
            "updates_per_step": int(tot_upd / steps), "value": round(batched_rate, 1), "unit": UNIT,
            "scaling": "weak" if world > 1 else None, "ranks": world,
            "ms_per_step": round(float(np.median(ms)), 3), "steps": steps,
            "launches_per_step": 1, "graph": "each step one launch of a captured CUDA graph "
                                              "(reset kernel + persistent batch kernel)",
            "failed_circuits": failed, "tuned_config": tuned,
            "value_wall_clock": round(batched_wall_rate, 1),
            "plain_value": round(plain_rate, 1),
            "plain_sample": "every %dth circuit (%d circuits), one sps_apply + sync each, "
                            "host wall clock" % (sample_every, len(sample)),
            "batched_vs_plain": round(batched_wall_rate / plain_rate, 2),
            "batched_vs_plain_clock": "both by the host wall clock (batched: graph launch + "
                                      "sync per step)",
            "cpu_baseline": cpu, "generate_s": round(gen_s, 1)}


def _oracle_circuit(job):
    """One circuit on the CPU oracle (worker process): (updates, seconds)."""
    from oracle import OracleState
    nq, gates = job
    t0 = time.perf_counter()
    orc = OracleState(nq)
    u = orc.apply_counted(gates, eps=EPS)
    return u, time.perf_counter() - t0


def batch_cpu_baseline(circs, every: int):
    """The oracle over a sample of the batch (every `every`-th circuit) on a
    pool of all host cores, one circuit per task, largest first; updates per
    second of wall clock."""
    import multiprocessing as mp
    sample = sorted(circs[::every], key=lambda c: -len(c.gates) * c.cap)
    jobs = [(c.nqubits, c.gates) for c in sample]
    ncores = os.cpu_count() or 1
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(ncores) as pool:
        pool.map(_oracle_circuit, [(20, jobs[0][1][:1])] * ncores)   # workers up
        t0 = time.perf_counter()
        res = pool.map(_oracle_circuit, jobs, chunksize=1)
        wall = time.perf_counter() - t0
    upd = sum(u for u, _ in res)
    return {"value": round(upd / wall, 1), "unit": UNIT, "cores": ncores, "kind": "oracle",
            "sample": "every %dth circuit of the batch (%d circuits, %d gates), one circuit per "
                      "task on a pool of %d processes, wall clock %.1f s" % (
                          every, len(jobs), sum(len(j[1]) for j in jobs), ncores, wall),
            "cpu": cpu_model()}


# ---- served form ------------------------------------------------------------------------
def serve_requests(count: int, seed: int = 77):
    """Request families: random mixes (70%), ripple-carry adders with a
    log-uniform superposition width 6..26 (20%: peaks 2^6..2^26 nonzeros),
    Givens circuits (10%)."""
    from paper_2105_01533_gb300 import workloads as W
    rng = W.SplitMix64(seed)
    out = []
    randoms = W.batched_workload_fast(count, first_seed=10_000 + seed, depth=(200, 2000),
                                      log2_cap=(8, 14))
    for i in range(count):
        u = rng.uniform()
        if u < 0.7:
            c = randoms[i]
            out.append(("random", c.nqubits, c.cap, c.gates))
        elif u < 0.9:
            w = int(round(math.exp(math.log(6) + (math.log(26) - math.log(6)) * rng.uniform())))
            wl = W.adder_workload(seed=1000 + i, nbits=32, width=w, n_cp=16)
            out.append(("adder", wl.layout.nqubits, 1 << w, wl.gates))
        else:
            n = (32, 48, 64)[rng.below(3)]
            k = 2 + rng.below(3)
            layers = 5 + rng.below(26)
            g = W.givens_workload(seed=2000 + i, nqubits=n, modes=k, layers=layers)
            out.append(("givens", n, math.comb(n, k), g))
    return out


def run_served(args, sps, torch, count: int, arrive_s: float):
    """Continuous batching under a Poisson stream: capacity at saturation, then
    arrivals at 0.5, 0.8 and 1.0 times that rate; latency = completion -
    scheduled arrival."""
    import random as _random
    reqs = serve_requests(count)
    free, _total = torch.cuda.mem_get_info()
    budget = int(free * 0.9) - (8 << 30)

    def drive(arrivals):
        srv = sps.Server(mem_budget_bytes=budget, max_active=2048, passes_per_tick=32)
        t0 = time.perf_counter()
        ids, done_at, upd = {}, {}, 0
        k = 0
        while k < len(arrivals) or len(done_at) < len(arrivals):
            now = time.perf_counter() - t0
            while k < len(arrivals) and arrivals[k] <= now:
                nm, nq, cap, g = reqs[k % len(reqs)]
                ids[srv.submit(nq, cap, g, EPS)] = k
                k += 1
            if not ids or len(done_at) == len(ids):
                time.sleep(0.0005)
                continue
            _, _, nd = srv.tick()
            if nd:
                t = time.perf_counter() - t0
                for rid in srv.completed():
                    done_at[ids[rid]] = t
                    upd += srv.poll(rid)["updates"]
        elapsed = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lat = [done_at[j] - arrivals[j] for j in range(len(arrivals))]
        return elapsed, upd, lat, st

    # saturation: everything arrives at once
    sat_n = min(count, 256)
    el, upd, lat, _ = drive([0.0] * sat_n)
    cap_rps = sat_n / el
    sat_rate = upd / el
    # Poisson arrivals at 0.5, 0.8 and 1.0 times the saturation rate
    loads = {}
    for f in (0.5, 0.8, 1.0):
        lam = f * cap_rps
        rnd = _random.Random(5)
        t, arr = 0.0, []
        while t < arrive_s and len(arr) < count:
            t += rnd.expovariate(lam)
            arr.append(t)
        el2, upd2, lat2, st2 = drive(arr)
        loads[f] = {"lambda_rps": round(lam, 2), "requests": len(arr),
                    "value": round(upd2 / el2, 1),
                    "p50_latency_ms": round(1e3 * float(np.percentile(lat2, 50)), 3),
                    "p99_latency_ms": round(1e3 * float(np.percentile(lat2, 99)), 3),
                    "ticks": st2["ticks"], "batched_launches": st2["launches"]}
    # the plain path, one request at a time, on the saturation set: each
    # request's state created, the circuit applied, the result copied to the
    # host (what the server hands back)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pu = 0
    for (nm, nq, cap, g) in reqs[:sat_n]:
        s1 = sps.SparseState(nq, cap)
        s1.apply(g, EPS)
        s1.get_amplitudes(sort=False)
        pu += s1.updates()
        s1.close()
    plain_s = time.perf_counter() - t0
    fam = {}
    for r in reqs[:sat_n]:
        fam[r[0]] = fam.get(r[0], 0) + 1
    mid = loads[0.8]
    return {"workload": "served: Poisson stream of random mixes (70%), adders with log-uniform "
                        "superposition width 6..26 (20%), Givens circuits n 32..64, 2..4 modes "
                        "(10%); peak nonzeros up to 2^26; FP64, eps 1e-14",
            "families_in_saturation_set": fam, "capacity_rps": round(cap_rps, 2),
            "saturation_requests": sat_n, "saturation_value": round(sat_rate, 1),
            "saturation_p99_latency_ms": round(1e3 * float(np.percentile(lat, 99)), 3),
            "value": mid["value"], "unit": UNIT, "lambda_rps": mid["lambda_rps"],
            "p50_latency_ms": mid["p50_latency_ms"], "p99_latency_ms": mid["p99_latency_ms"],
            "loads": {"%.1fx" % f: v for f, v in loads.items()},
            "plain_value": round(pu / plain_s, 1),
            "served_vs_plain": round(sat_rate / (pu / plain_s), 2),
            "served_vs_plain_set": "the same %d requests, one state, sps_apply and result "
                                   "read-back each" % sat_n,
            "memory_budget_gb": round(budget / 2 ** 30, 1)}


# ---- the oracle on the host ------------------------------------------------------------
def oracle_rate(wl, budget_s: float):
    """Run the oracle over the gate stream (gate by gate, single thread) until
    the budget is used; returns (updates, seconds, gates_done)."""
    from oracle import OracleState
    gates = wl["gates"]
    orc = OracleState(wl["nqubits"])
    if wl.get("block"):
        orc.apply(wl["prep"], eps=EPS)
    u, done, t = 0, 0, 0.0
    while done < len(gates) and t < budget_s:
        t0 = time.perf_counter()
        u += orc.apply_counted(gates[done:done + 1], eps=EPS)
        t += time.perf_counter() - t0
        done += 1
    return u, t, done


def cpu_baseline(wl, budget_s: float):
    """The oracle on one host thread, median of three runs of the same bounded
    sample (the first gates of the stream, as many as fit the budget)."""
    runs = [oracle_rate(wl, budget_s / 3.0) for _ in range(3)]
    rates = sorted(u / t for u, t, _ in runs)
    done = min(d for _, _, d in runs)
    return {"value": round(rates[1], 1), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "first %d of %d gates of %s from |0..0>, gate by gate, one host thread; "
                      "median of 3 runs (%.1f s each)" % (done, len(wl["gates"]), wl["name"],
                                                          budget_s / 3.0),
            "runs": [round(r, 1) for r in rates], "cpu": cpu_model(), "nproc": os.cpu_count()}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo; Arm parts are
    named from their part number)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                if name and name != "-":
                    return name
    except (OSError, subprocess.SubprocessError):
        pass
    arm_parts = {"0xd4f": "Arm Neoverse-V2", "0xd40": "Arm Neoverse-V1", "0xd0c": "Arm Neoverse-N1"}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.lower()
                if key.startswith("model name"):
                    return line.split(":", 1)[1].strip()
                if key.startswith("cpu part"):
                    part = line.split(":", 1)[1].strip()
                    return arm_parts.get(part, "Arm CPU part " + part)
    except OSError:
        pass
    return "unknown"


def run_reference(args, dist, rank, world):
    if rank != 0:
        return None
    import oracle
    oracle.build()
    wl = make_workload(args.workload)
    per_step = max(0.05, min(5.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_rate(wl, per_step)
    us, ts, gates = 0, 0.0, 0
    times = []
    for _ in range(args.steps):
        u, t, g = oracle_rate(wl, per_step)
        us += u
        ts += t
        gates = g
        times.append(t)
    value = us / ts
    return {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * ts / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"], "nqubits": wl["nqubits"],
                       "parallelism": "single host thread"},
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "each step: the first %d gates of %s from |0..0>, gate by "
                                       "gate" % (gates, wl["name"]), "cpu": cpu_model()},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="adder67-w24",
                    choices=["adder67", "adder67-w22", "adder67-w24", "givens64", "givens64-m5",
                             "givens64-m6"])
    ap.add_argument("--sublines", default="adder67,givens64,givens64-m5,givens64-m6",
                    help="comma-separated configs measured after the headline ('' for none)")
    ap.add_argument("--sub-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fused-readout", type=int, default=1,
                    help="register the step's readout so that a compiled expansion launch "
                         "ending the apply sums it (0: the readout kernel every step)")
    ap.add_argument("--opt", action="append", default=[],
                    help="library option NAME=VALUE (e.g. bitslice_min_ops=0), repeatable")
    ap.add_argument("--batched", type=int, default=1,
                    help="also measure the batched form (1) or not (0)")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--served", type=int, default=1,
                    help="also measure the served form (1) or not (0)")
    ap.add_argument("--serve-count", type=int, default=2000)
    ap.add_argument("--branch-forms", type=int, default=1,
                    help="1: time one branching workload under the gather and scatter forms")
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--batch-cpu-every", type=int, default=8,
                    help="all-core oracle baseline on every k-th batched circuit (0: skip)")
    ap.add_argument("--dump-profile", default=None,
                    help="write the per-launch records of one profiled step to this JSON file")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for a profiler "
                         "started with capture off, e.g. ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        # rank 0 alone times the host oracle; other ranks exit without work
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        res = run_reference(args, None, rank, world)
        if rank == 0 and res is not None:
            print(json.dumps(res), flush=True)
        return
    dist, rank, world, local_rank = dist_init(args.gpus)
    if True:
        res = run_ours(args, dist, rank, world, local_rank)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
