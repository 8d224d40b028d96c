"""Benchmark: amplitude-steps/s of a reversible wiring diagram on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload adder_m32|mixed_m28|cnot_m16|...] [--also mixed_m28]

One timed step = one pass of the whole hot path over the resident state:
validate + plan the circuit, apply all of its steps and compute the FP64
basis-state probabilities into device memory, through
qsim_apply_circuit_probabilities (the last pass writes the probabilities
beside the state; --separate-probs times qsim_apply_circuit followed by
qsim_probabilities_device instead).  value = 2^M * L * K / (device time of
K steps).

Default workload: M=32 complex64 (32 GiB state, in place, larger than L2):
the ripple-carry adder of two 15-bit registers with carry-in and carry-out,
two additions per unit, unit repeated 8 times (1456 CNOT / Toffoli steps),
lines placed on address bits by a seeded permutation; seeded synthetic
state.  Adjacent-equal-step cancellation is switched off, so every one of the
L steps is applied.  The same line also carries the M=28 complex128 workload
of 1000 NOT / CNOT / Toffoli / 3-5-control NOT steps (key "also", resident
timing only) and the batched-vs-plain comparison on 4096 circuits of both
gate mixes (key "batch").

Also reported on the same JSON line:
  e2e          the same metric through the C ABI with host buffers: each step
               copies the state in from pinned host memory, applies the
               circuit, computes probabilities and copies them back.
  roofline     the dominant kernel's algorithmic bytes per launch over its
               average CUDA-event duration, against the measured HBM copy
               bandwidth (MEASURED_PEAKS.json).
  cpu_baseline the CPU oracle on the host cores, on a bounded prefix of the
               same circuit and state.
  clocks       nvidia-smi samples taken during the timed region.

``--impl reference`` times the CPU oracle alone (the reference arm).
Under torchrun (N > 1) every rank runs an independent replica of the
workload; value is the sum over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_quant_ph_0308158_gb300 import workloads as W  # noqa: E402

METRIC = "amplitude-steps/s"
UNIT = "amp-steps/s"
FALLBACK_HBM_GBS = 6800.0
CSRC = os.path.join(ROOT, "paper_quant_ph_0308158_gb300", "csrc")
# source files that define a kernel's code (every other kernel: kernels.cu)
KERNEL_SOURCE = {"qsim_jit_gather": ("jit.cu", "prob_math.cuh"), "qsim_jit_closed": ("jit.cu", "prob_math.cuh"),
                 "qsim_jit_delta": ("jit.cu",)}
KERNELS_CU = ("kernels.cu", "prob_math.cuh", "qsim_internal.h")


def workload(name: str):
    if name == "mixed_m28":
        return W.config_mixed_m28()
    if name == "adder_m32":
        return W.config_adder_m32()
    if name == "cnot_m16":
        return W.config_small_cnot()
    if name == "mixed_m24":  # 256 MiB: the small case for ncu captures
        return W.config_mixed(24)
    if name == "cnot_m28":  # CNOT-only: one affine gather pass
        return W.config_cnot(28)
    if name == "cnot_m26":  # 1 GiB: the small case for coset-gather captures
        return W.config_cnot(26)
    if name == "adder_m28":  # 2 GiB in-place adder: the small case for tile-kernel captures
        return W.config_adder(13)
    if name == "hybrid_m28":  # register arithmetic then a CNOT layer: strategies mixed per segment
        return W.config_hybrid(28)
    if name == "parity_m32":  # Sec. 4 example, input generated on the device (App. 1)
        return W.config_parity(32)
    if name == "parity_m28":  # 2 GiB: the small case for product-input captures
        return W.config_parity(28)
    raise SystemExit("unknown workload " + name)


def strategy_for(name: str) -> str:
    # the adder workload is specified in place
    return "inplace" if name.startswith("adder") else "auto"


# ----------------------------------------------------------------------------
# distributed plumbing (replicas only; no data-path collective)
# ----------------------------------------------------------------------------

def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    on_gpu = dist.get_backend() == "nccl"
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if on_gpu else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# roofline inputs
# ----------------------------------------------------------------------------

def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(kernel: str) -> str:
    """First 16 hex digits of the SHA-256 of the source files of a kernel."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCE.get(kernel, KERNELS_CU):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, wl: str):
    """DRAM bytes per launch recorded from an ncu capture of the current kernel
    source (profiles/traffic.json), scaled to the benchmarked launch; None if
    absent or taken on a different kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    e = rec.get(wl, {}).get(kernel)
    if not e or e.get("kernel_source_sha256_16") != kernel_source_hash(kernel):
        return None
    return float(e["dram_bytes_per_launch"])


# ----------------------------------------------------------------------------
# reference arm / CPU baseline: the oracle
# ----------------------------------------------------------------------------

def _host_free_bytes() -> int:
    try:
        return os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        return 0


def oracle_state(cfg, k1=None):
    """The workload's state in the oracle's FP64 complex storage (built before
    any timing), or None when the host lacks the memory for it."""
    M = cfg["M"]
    need = 16 << M
    if k1 is None:
        need += np.dtype(cfg["dtype"]).itemsize << M
    if _host_free_bytes() and _host_free_bytes() < need + (4 << 30):
        return None
    if k1 is None:
        k1 = W.random_state(M, cfg["dtype"], cfg["state_seed"])
    return np.asarray(k1).astype(np.complex128)


def oracle_steps_rate(M: int, k: np.ndarray, steps):
    """Time the CPU oracle's step-by-step loop (single thread) applying steps
    in place to the full FP64 state.  Returns (amp-steps/s, seconds)."""
    import oracle
    t0 = time.perf_counter()
    oracle.apply_circuit_inplace(M, k, steps)
    dt = time.perf_counter() - t0
    return (1 << M) * len(steps) / dt, dt


def oracle_rows_rate(cfg, k1, rows: int = 1 << 18):
    """Fallback sample for a host without room for an FP64 copy of the state:
    the oracle's single-row evaluation k2(i) = k1(x(i)) through all L steps on
    seeded rows (k1: the input state, or a function of the source rows).
    Returns (amp-steps/s, seconds)."""
    import oracle
    M, steps = cfg["M"], cfg["steps"]
    r = np.random.default_rng(7).integers(0, 1 << M, size=rows, dtype=np.uint64)
    get = k1 if callable(k1) else (lambda src: k1[src])
    t0 = time.perf_counter()
    oracle.sample_outputs(M, get, steps, r)
    dt = time.perf_counter() - t0
    return rows * len(steps) / dt, dt


def run_reference(args, rank, ws):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    cfg = workload(args.workload)
    M, steps = cfg["M"], cfg["steps"]
    L = len(steps)
    per = args.ref_steps_per_step if args.ref_steps_per_step > 0 else (1 if M >= 31 else 2)
    per = max(1, min(L, per))
    k = oracle_state(cfg)
    pos = 0

    def one():
        nonlocal pos
        sl = [steps[(pos + j) % L] for j in range(per)]
        pos = (pos + per) % L
        return oracle_steps_rate(M, k, np.array(sl, dtype=steps.dtype))[1]

    rows = 1 << 18
    if k is None:  # no room for an FP64 copy of the state: single rows through all L steps
        def one():
            return oracle_rows_rate(cfg, lambda src: src.astype(np.float64).astype(np.complex128), rows)[1]
    for _ in range(args.warmup):
        one()
    total = sum(one() for _ in range(args.steps))
    if k is None:
        value = rows * L * args.steps / total
        sample = ("host too small for a %d GiB FP64 copy: single-row evaluation k2(i) = k1(x(i)) "
                  "through all %d steps on 2^18 seeded rows per timed step" % ((16 << M) >> 30, L))
    else:
        value = (1 << M) * per * args.steps / total
        sample = ("%d successive circuit steps per timed step (cycling through the %d steps) on the "
                  "full 2^%d-amplitude state in FP64, in place" % (per, L, M))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128" if np.dtype(cfg["dtype"]) == np.complex128 else "c64",
        "data": "synthetic", "config": {"workload": cfg["name"], "M": M, "L": L},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def _roofline(passes, wl_name):
    """Roofline record of the dominant kernel (most device time) of a list of
    traced passes (kernel, ms, algorithmic bytes)."""
    by_kind = {}
    for kind, ms, by in passes:
        a = by_kind.setdefault(kind, [0, 0.0, 0.0])
        a[0] += 1
        a[1] += ms
        a[2] += by
    dkernel, (dlaunch, dms, dbytes) = max(by_kind.items(), key=lambda kv: kv[1][1])
    peak, peak_src = hbm_peak()
    achieved = (dbytes / dlaunch) / (dms / dlaunch * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": ncu_traffic(dkernel, wl_name), "kernel": dkernel,
                "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                else "fallback 6800 GB/s",
                "algorithmic_bytes_per_launch": dbytes / dlaunch,
                "avg_launch_ms": dms / dlaunch, "launches": dlaunch,
                "share_of_device_time": dms / max(1e-30, sum(v[1] for v in by_kind.values()))}
    kernel_ms = {k: v[1] / max(1, v[0]) for k, v in by_kind.items()}
    kernel_launches = {k: v[0] for k, v in by_kind.items()}
    return roofline, kernel_ms, kernel_launches


class Resident:
    """One workload timed with its state resident in HBM: the context, its
    host input and what the timed region measured."""


def measure_resident(args, cfg, strategy, use_jit, local, ws, steps_k, warmup, sample_clocks=True,
                     for_e2e=True):
    """Time steps_k steps of one workload on a resident state (after warmup
    untimed steps), CUDA events on the context's stream, max over ranks.

    A step is one pass of the whole hot path: validate and plan the circuit,
    every pass, and the FP64 probabilities into device memory (written by the
    last pass, or by their own pass with --separate-probs)."""
    import torch
    from paper_quant_ph_0308158_gb300 import Simulator

    r = Resident()
    M, dtype, steps = cfg["M"], np.dtype(cfg["dtype"]), cfg["steps"]
    n = 1 << M
    tdt = torch.complex64 if dtype == np.complex64 else torch.complex128
    # seeded state in pinned host memory (also the e2e input buffer), or the
    # qubits of a product-state input generated on the device (App. 1); the
    # end-to-end leg copies that state in from the host all the same
    qubits = cfg.get("qubits")
    h_in = None
    if qubits is None or (for_e2e and not args.no_e2e):
        h_in = torch.empty(n, dtype=tdt, pin_memory=True).numpy()
        if qubits is None:
            W.random_state(M, dtype, cfg["state_seed"], out=h_in)
        else:  # the only product-state workload is the Sec. 4 alternating input
            assert np.array_equal(qubits, W.sec4_qubits(M)), "host copy of this product state"
            W.alternating_state(M, dtype, out=h_in)
    scratch = strategy in ("auto", "gather")  # the other strategies work in place
    sim = Simulator(M, dtype, scratch=scratch)
    sim.set_strategy(strategy, args.tile_bits, args.low_bits)
    sim.set_canonicalize(False)
    sim.set_coset(not args.no_coset, args.coset_run_bits, args.coset_stage_kib)

    def load_input():
        if qubits is None:
            sim.load_state(h_in)
        else:
            sim.load_product_state(qubits)

    jit_ms = None
    if use_jit:
        # compiled kernels: gathers are compiled here, before any timing; a
        # closed tile pass (in place) is compiled by the first apply, which
        # also finds the bits the circuit changes -- both outside the timing
        if scratch:
            from paper_quant_ph_0308158_gb300 import jit_precompile
            jit_ms = jit_precompile(M, dtype, steps, canonicalize=False)
        sim.set_jit(True)
    probs = torch.empty(n, dtype=torch.float64, device="cuda")
    tuned = None
    if args.autotune:  # measured plan choice, before warm-up (not timed, like compilation)
        load_input()
        t0 = time.perf_counter()
        cands = sim.autotune(steps, reps=1)
        tuned = {"seconds": time.perf_counter() - t0, "chosen": cands[0], "candidates": cands}

    def step():
        if qubits is not None:  # App. 1 input generated within the step (first pass)
            sim.apply_product(qubits, steps, probs.data_ptr())
        elif args.separate_probs:
            sim.apply(steps)
            sim.probabilities_device(probs.data_ptr())
        else:
            sim.apply_probabilities(steps, probs.data_ptr())

    stream = torch.cuda.current_stream()
    load_input()
    t0 = time.perf_counter()
    step()  # the first apply plans the circuit (and compiles what it needs)
    sim.synchronize()
    r.first_step_s = time.perf_counter() - t0
    for _ in range(warmup):
        step()
    sim.synchronize()
    sim.set_profiling(True)
    sim.pass_times()  # clear
    clocks = ClockSampler(local) if sample_clocks else None
    if clocks:
        clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps_k):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    r.clocks = clocks.stop() if clocks else None
    ms_total = max_over_ranks(e0.elapsed_time(e1), ws)
    passes = sim.pass_times()
    sim.set_profiling(False)
    r.stats = sim.plan_stats()
    r.ms_step = ms_total / steps_k
    r.value = ws * n * len(steps) * steps_k / (ms_total * 1e-3)
    r.roofline, r.kernel_ms, r.kernel_launches = _roofline(passes, cfg["name"])
    r.launches = len(passes)  # every pass kernel and probabilities kernel in the timed region
    r.sim, r.h_in, r.qubits, r.scratch, r.jit_ms, r.tuned, r.probs = sim, h_in, qubits, scratch, jit_ms, tuned, probs
    r.jit = bool(use_jit)
    return r


def measure_e2e(args, cfg, r, local, ws, steps_k):
    """The same metric end to end through the C ABI with host buffers: each
    step copies its state in from pinned host memory, applies the circuit and
    copies the FP64 probabilities out to pinned host memory.  Two contexts on
    two streams alternate steps, so one step's copies overlap the other's
    kernels (each context waits for its previous step before reusing its
    buffers); copies in go one after the other over the host link."""
    import torch
    from paper_quant_ph_0308158_gb300 import Simulator

    M, dtype, steps = cfg["M"], np.dtype(cfg["dtype"]), cfg["steps"]
    n = 1 << M
    L = len(steps)
    need = n * dtype.itemsize + 2 * n * 8 + (8 << 30)  # input, two outputs, headroom
    budget = getattr(args, "host_budget", 0)
    if budget and need > budget:
        return {"unavailable": "host memory: the end-to-end leg page-locks %.0f GiB per rank, "
                               "this rank's share of the node is %.0f GiB" % (need / 2**30, budget / 2**30)}
    outs_block = torch.empty(2 * n, dtype=torch.float64, pin_memory=True)
    stream = torch.cuda.current_stream()
    s2 = torch.cuda.Stream()
    with torch.cuda.stream(s2):
        sim2 = Simulator(M, dtype, scratch=r.scratch)
    sim2.set_strategy(args.strategy or strategy_for(args.workload), args.tile_bits, args.low_bits)
    sim2.set_canonicalize(False)
    if r.jit:
        sim2.set_jit(True)
    sims = (r.sim, sim2)
    streams = (stream, s2)
    outs = [outs_block[:n].numpy(), outs_block[n:].numpy()]
    loaded = [torch.cuda.Event() for _ in range(2)]

    def e2e_step(i):
        c = i & 1
        sm = sims[c]
        if i >= 2:
            sm.synchronize()  # this context's previous step is done
        if i >= 1:  # copies in go one after the other over the host link
            streams[c].wait_event(loaded[1 - c])
        sm.load_state_async(r.h_in)
        loaded[c].record(streams[c])
        sm.apply_probabilities_async(steps, outs[c])

    for i in range(2):  # warm both contexts
        e2e_step(i)
    for sm in sims:
        sm.synchronize()
    torch.cuda.synchronize()
    barrier(ws)
    f0 = torch.cuda.Event(enable_timing=True)
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ke = max(2, steps_k)
    f0.record(stream)
    s2.wait_event(f0)
    for i in range(ke):
        e2e_step(i)
    for sm in sims:
        sm.synchronize()
    for j in range(2):
        ends[j].record(streams[j])
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(max(f0.elapsed_time(e) for e in ends), ws)
    sim2.close()
    del outs, outs_block
    return {"value": ws * n * L * ke / (ms_e2e * 1e-3), "unit": UNIT,
            "h2d_bytes_per_step": n * dtype.itemsize, "d2h_bytes_per_step": n * 8,
            "ms_per_step": ms_e2e / ke, "steps": ke,
            "pipelining": "two contexts on two streams alternate steps; copies in are serialised"}


def cpu_baseline_for(args, cfg, h_in):
    """The oracle, as it stands, on the first steps of the same circuit and
    state (single thread, full state in FP64, widened before timing)."""
    import oracle
    oracle.build()
    M, steps = cfg["M"], cfg["steps"]
    L = len(steps)
    nst = min(L, args.cpu_steps if args.cpu_steps > 0 else (2 if M >= 31 else 24))
    k = oracle_state(cfg, h_in)
    if k is None:
        rate, secs = oracle_rows_rate(cfg, h_in)
        sample = ("host too small for a %d GiB FP64 copy: single-row evaluation of all %d steps "
                  "on 2^18 seeded rows (%.1f s)" % ((16 << M) >> 30, L, secs))
    else:
        rate, secs = oracle_steps_rate(M, k, steps[:nst])
        sample = "first %d of the %d steps on the full 2^%d-amplitude state, FP64 (%.1f s)" % (
            nst, L, M, secs)
    del k
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
            "host_threads": os.cpu_count()}


def run_ours(args, rank, ws, local):
    import torch
    from paper_quant_ph_0308158_gb300 import build

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    # host memory this rank may page-lock: the ranks of one node share it
    free0 = _host_free_bytes()
    args.host_budget = free0 // max(1, int(os.environ.get("LOCAL_WORLD_SIZE", "1"))) if free0 else 0
    build.build()
    torch.cuda.set_device(local)
    cfg = workload(args.workload)
    M, dtype, L = cfg["M"], np.dtype(cfg["dtype"]), len(cfg["steps"])
    n = 1 << M
    strategy = args.strategy or strategy_for(args.workload)
    r = measure_resident(args, cfg, strategy, args.jit, local, ws, args.steps, args.warmup)

    # ---- CPU baseline: the oracle on a bounded prefix (rank 0, N=1) -----------
    # (before the end-to-end leg, whose pinned buffers stay cached)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and r.h_in is not None:
        cpu = cpu_baseline_for(args, cfg, r.h_in)

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(args, cfg, r, local, ws, args.steps)
    h_in_bytes = 0 if r.h_in is None else r.h_in.nbytes
    r.sim.close()
    r.h_in = None
    del r.probs

    # ---- the other single-circuit workload, on the same line ------------------
    also = {}
    for wl in args.also:
        if wl == args.workload:
            continue
        c2 = workload(wl)
        r2 = measure_resident(args, c2, strategy_for(wl), args.jit, local, ws, args.steps,
                              args.warmup, sample_clocks=False, for_e2e=False)
        r2.sim.close()
        pure = None
        if wl == "hybrid_m28":  # the same circuit forced into one strategy
            pure = {}
            for strat in ("gather", "inplace"):
                r3 = measure_resident(args, c2, strat, args.jit, local, ws, max(3, args.steps // 2),
                                      args.warmup, sample_clocks=False)
                r3.sim.close()
                pure[strat] = {"ms_per_step": r3.ms_step, "passes": r3.stats["passes"],
                               "kernel_ms": r3.kernel_ms}
        also[wl] = {"workload": c2["name"], "value": r2.value, "unit": UNIT, "pure_plans": pure,
                    "plan_est_ms": r2.stats["est_ms"], "kernel_launches": r2.kernel_launches,
                    "ms_per_step": r2.ms_step, "M": c2["M"], "L": len(c2["steps"]),
                    "dtype": "c128" if np.dtype(c2["dtype"]) == np.complex128 else "c64",
                    "passes_per_step": r2.stats["passes"], "jit": r2.jit,
                    "first_step_s": r2.first_step_s,
                    "jit_compile_ms": r2.jit_ms, "kernel_ms": r2.kernel_ms,
                    "roofline": r2.roofline, "gpu_launches": r2.launches}

    # ---- batched vs one launch per circuit (part of the metric) ----------------
    batch = None
    if not args.no_batch:
        batch = [batch_speedup(args.batch_compare, mix, 10, 3) for mix in ("cnot", "mixed")]

    # ---- serving (bounded open-loop sample, its own process) -------------------
    serve = None
    if rank == 0 and ws == 1 and args.serve_in_line > 0:
        serve = serve_sample(args)
    if rank == 0:
        stats = r.stats
        line = {
            "metric": METRIC, "value": r.value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r.ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128" if dtype == np.complex128 else "c64",
            "data": "synthetic (seeded random state and circuit)",
            "config": {"workload": cfg["name"], "M": M, "L": L, "strategy": strategy,
                       "tile_bits": args.tile_bits, "low_bits": args.low_bits,
                       "state_bytes": n * dtype.itemsize, "l2": "inputs larger than L2",
                       "parallelism": "replicas" if ws > 1 else "single",
                       "passes_per_step": stats["passes"],
                       "gather_passes": stats["gather_passes"],
                       "tile_passes": stats["tile_passes"],
                       "sweep_passes": stats["sweep_passes"],
                       "steps_cancelled": stats["steps_cancelled"],
                       "full_pass_equiv": stats["full_pass_equiv"],
                       "step_includes": "plan + all passes + FP64 probabilities",
                       "probabilities": "separate pass" if args.separate_probs
                       else "written by the last pass",
                       "in_place": not r.scratch,
                       "jit": r.jit,
                       "first_step_s": r.first_step_s,
                       "plan_est_ms": r.stats["est_ms"],
                       "autotune": r.tuned,
                       "jit_compile_ms": r.jit_ms,
                       "host_input_bytes": h_in_bytes,
                       "kernel_ms": r.kernel_ms, "kernel_launches": r.kernel_launches},
            "roofline": r.roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": r.launches,
            "clocks": r.clocks,
            "also": also or None,
            "batch": batch,
            "serve": serve,
        }
        print(json.dumps(line), flush=True)
    return 0


def serve_sample(args):
    """A bounded serving run for the benchmark line: the open-loop Poisson
    stream of --workload serve at its 200 requests/s (over capacity, so the
    rate served is the server's capacity and compares with one request at a
    time through the plain API) with fewer requests and states up to M = 28,
    in a child process (its page-locked pools and HBM budget come and go with
    it; this process's cached device memory is released first).  Returns the
    child's key figures, or a reason it has none."""
    import torch
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    n = args.serve_in_line
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", "serve", "--serve-requests", str(n),
           "--serve-rate", "200", "--serve-m-max", "28", "--serve-host-gb", "16",
           "--serve-plain-requests", str(max(20, n // 12))]
    try:
        out = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
    except subprocess.TimeoutExpired:
        return {"unavailable": "serving sample timed out"}
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    if out.returncode != 0 or not lines:
        return {"unavailable": "serving sample exited %d: %s" % (out.returncode, out.stderr[-300:])}
    d = json.loads(lines[-1])
    c = d["config"]
    keys = ("requests_per_s", "offered_requests_per_s", "latency_ms_p50", "latency_ms_p99", "wall_s",
            "h2d_gbs_while_busy", "d2h_gbs_while_busy", "compute_busy_frac", "served_over_plain")
    r = {"workload": c["workload"] + "_M12-28", "value": d["value"], "unit": d["unit"], "e2e": d["e2e"],
         "gpu_launches": d["gpu_launches"], "clocks": d["clocks"]}
    r.update({k: c.get(k) for k in keys})
    return r


def batch_speedup(n: int, mix: str, steps: int, warmup: int):
    """Time one batch run (graph of persistent launches) against one plain
    launch per circuit pass on n circuits of the batched workload; returns a
    dict for the JSON line.  Used by the default benchmark for the
    batched-vs-plain part of the metric.  For NOT/CNOT circuits the size from
    which gathers read in coset-tile order is chosen by timing (every
    candidate is measured and reported; the fastest is the batched number,
    and the plain path uses the same plans)."""
    import torch
    from paper_quant_ph_0308158_gb300 import Batch
    specs = W.batch_specs(n, seed=4, mix=mix)
    dtype = np.dtype(np.complex64)
    states = [W.random_state(sp["M"], dtype, sp["state_seed"]) for sp in specs]

    def measure(coset_min):
        b = Batch([(s["M"], s["steps"]) for s in specs], dtype, coset_min_qubits=coset_min)
        for i, st in enumerate(states):
            b.load_state(i, st)
        info = b.info()
        stream = torch.cuda.ExternalStream(info["stream"])

        def timed(fn, k):
            for _ in range(warmup):
                fn()
            b.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(k):
                fn()
            e1.record(stream)
            b.synchronize()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / k

        ms_b = timed(b.run, steps)
        b.close()
        return ms_b, info

    cands = [14, 18, 64] if mix == "cnot" else [18]
    tuned = {c: measure(c) for c in cands}
    best = min(tuned, key=lambda c: tuned[c][0])
    ms_b, info = tuned[best]
    b = Batch([(s["M"], s["steps"]) for s in specs], dtype, coset_min_qubits=best)
    for i, st in enumerate(states):
        b.load_state(i, st)
    stream = torch.cuda.ExternalStream(b.info()["stream"])
    for _ in range(warmup):
        b.run_plain()
    b.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        b.run_plain()
    e1.record(stream)
    b.synchronize()
    torch.cuda.synchronize()
    ms_p = e0.elapsed_time(e1) / steps
    b.close()
    return {"circuits": n, "mix": mix, "amplitude_steps_per_run": info["amplitude_steps"],
            "batched_ms": ms_b, "plain_ms": ms_p, "batched_over_plain": ms_p / ms_b,
            "batched_value": info["amplitude_steps"] / (ms_b * 1e-3),
            "plain_value": info["amplitude_steps"] / (ms_p * 1e-3),
            "coset_min_qubits": best,
            "coset_min_qubits_ms": {str(c): v[0] for c, v in tuned.items()},
            "passes": {k: info[k] for k in ("coset_passes", "affine_passes", "sliced_passes", "sweep_passes")},
            "levels": info["levels"]}


def run_batch(args, rank, ws, local):
    """Batched circuits: one captured graph of persistent launches per run,
    against one plain launch per circuit pass (same plans, same states)."""
    import torch
    from paper_quant_ph_0308158_gb300 import Batch, build

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    build.build()
    torch.cuda.set_device(local)
    mix = "mixed" if args.workload.endswith("mixed") else "cnot"
    n = args.batch_size
    specs = W.batch_specs(n, seed=4, mix=mix)
    dtype = np.dtype(np.complex64)
    t0 = time.perf_counter()
    b = Batch([(s["M"], s["steps"]) for s in specs], dtype)
    create_s = time.perf_counter() - t0
    for i, sp in enumerate(specs):
        b.load_state(i, W.random_state(sp["M"], dtype, sp["state_seed"]))
    info = b.info()
    stream = torch.cuda.ExternalStream(info["stream"])
    amp_steps = info["amplitude_steps"]

    def timed(fn, k):
        for _ in range(args.warmup):
            fn()
        b.synchronize()
        barrier(ws)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        b.synchronize()
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), ws) / k

    clocks = ClockSampler(local)
    clocks.start()
    ms_batch = timed(b.run, args.steps)
    clk = clocks.stop()
    ms_plain = timed(b.run_plain, max(1, args.steps // 4))
    peak, peak_src = hbm_peak()
    achieved = info["algorithmic_bytes"] / (ms_batch * 1e-3) / 1e9
    value = ws * amp_steps / (ms_batch * 1e-3)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_batch, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64",
            "data": "synthetic (seeded random states and circuits)",
            "config": {"workload": "batch%d_%s" % (n, mix), "circuits": n, "M_range": [10, 22],
                       "L_range": [50, 2000], "levels": info["levels"], "items": info["items"],
                       "arena_bytes": info["arena_bytes"], "create_s": create_s,
                       "plain_ms_per_run": ms_plain,
                       "plain_value": ws * amp_steps / (ms_plain * 1e-3),
                       "batched_over_plain": ms_plain / ms_batch,
                       "step": "one run of every circuit (graph replay)",
                       "l2": "inputs larger than L2 (%.1f GB of states)" % (info["arena_bytes"] / 2e9)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "batch_kernel",
                         "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": info["algorithmic_bytes"] / max(1, info["levels"]),
                         "avg_launch_ms": ms_batch / max(1, info["levels"])},
            "cpu_baseline": None, "e2e": None,
            "gpu_launches": args.steps * info["levels"],
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    b.close()
    return 0


def serve_plain_baseline(specs, pool):
    """The same requests one at a time through the plain API, back to back:
    load the state from pinned host memory, apply the circuit, copy the FP64
    probabilities to pinned host memory, then the next request (one context
    per M, created before timing)."""
    import torch
    from paper_quant_ph_0308158_gb300 import Simulator

    sims, outs = {}, {}
    ms = sorted({sp["M"] for sp in specs})
    block = torch.empty(sum(1 << M for M in ms), dtype=torch.float64, pin_memory=True).numpy()
    off = 0
    for M in ms:
        sims[M] = Simulator(M, np.complex128)
        outs[M] = block[off: off + (1 << M)]
        off += 1 << M
    for sp in specs[:3]:  # warm-up
        sims[sp["M"]].load_state(pool[sp["M"]][1])
        sims[sp["M"]].apply(sp["steps"])
        sims[sp["M"]].probabilities(out=outs[sp["M"]])
    torch.cuda.synchronize()
    amp_steps = 0.0
    t0 = time.perf_counter()
    for sp in specs:
        sim = sims[sp["M"]]
        sim.load_state(pool[sp["M"]][1])
        sim.apply(sp["steps"])
        sim.probabilities(out=outs[sp["M"]])
        amp_steps += float(1 << sp["M"]) * sp["L"]
    wall = time.perf_counter() - t0
    for sim in sims.values():
        sim.close()
    return {"requests": len(specs), "wall_s": wall, "value": amp_steps / wall,
            "requests_per_s": len(specs) / wall,
            "how": "first requests of the same stream, one at a time, closed loop"}


def run_gather_floor(args, rank, ws, local):
    """The random-read floor of the gather pass: the M=28 complex128 mixed
    circuit's row array (qsim_row_array) applied by qsim_gather_rows -- the
    same 2^28 scattered 16-byte reads and coalesced stores and probabilities
    as the compiled gather, with no index arithmetic -- at several reads in
    flight per thread, beside the compiled gather itself and the coset and
    direct affine gathers of the 1000-CNOT circuit."""
    import torch
    from paper_quant_ph_0308158_gb300 import Simulator, build, gather_rows, jit_precompile

    build.build()
    torch.cuda.set_device(local)
    cfg = workload("mixed_m28") if args.floor_m == 28 else W.config_mixed(args.floor_m)
    M, steps = cfg["M"], cfg["steps"]
    n = 1 << M
    stream = torch.cuda.current_stream()
    k1 = torch.empty(n, dtype=torch.complex128, pin_memory=True)
    W.random_state(M, np.complex128, cfg["state_seed"], out=k1.numpy())
    d_in = k1.to("cuda")
    d_out = torch.empty_like(d_in)
    probs = torch.empty(n, dtype=torch.float64, device="cuda")
    rows = torch.empty(n, dtype=torch.int64, device="cuda")
    peak, _ = hbm_peak()
    alg = n * (16 + 16 + 8)

    def timed(fn, k=args.steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    out = {}
    with Simulator(M, np.complex128) as sim:
        sim.row_array(steps, rows.data_ptr())
        sim.synchronize()
    for U in (4, 8, 16):
        ms = timed(lambda: gather_rows(d_in.data_ptr(), d_out.data_ptr(), rows.data_ptr(), M,
                                       np.complex128, probs.data_ptr(), U, stream.cuda_stream))
        out["rows_U%d" % U] = {"ms": ms, "alg_GBps": alg / ms / 1e6,
                               "alg_GBps_with_rows": (alg + 8 * n) / ms / 1e6}
    del rows
    out["copy_4GiB"] = {"ms": timed(lambda: d_out.copy_(d_in))}
    out["copy_4GiB"]["GBps"] = 2 * 16 * n / out["copy_4GiB"]["ms"] / 1e6
    jit_precompile(M, np.complex128, steps, canonicalize=False)
    cn = workload("cnot_m28") if args.floor_m == 28 else W.config_cnot(args.floor_m)
    for name, st, jit, coset in (("jit_gather_mix1000", steps, True, True),
                                 ("coset_gather_cnot1000", cn["steps"], False, True),
                                 ("affine_gather_cnot1000", cn["steps"], False, False)):
        with Simulator(M, np.complex128) as sim:
            sim.set_canonicalize(False)
            sim.set_jit(jit)
            sim.set_coset(coset)
            sim.load_state(k1.numpy())
            ms = timed(lambda: sim.apply_probabilities(st, probs.data_ptr()))
        out[name] = {"ms": ms, "alg_GBps": alg / ms / 1e6, "frac": alg / ms / 1e6 / peak}
    if rank == 0:
        print(json.dumps({"workload": "gather_floor_M%d_c128" % M, "peak_GBps": peak,
                          "alg_bytes_per_pass": alg, "results": out}), flush=True)
    return 0


def run_parity_scan(args, rank, ws, local):
    """Sec. 4 computational example at every M of a range: the parity program
    on the alternating input (generated on the device from its qubits, App. 1),
    probabilities included, timed per M.  The paper reports its run time
    growing about 3.4x per added qubit at M = 30-31 on modi4 (Sec. 4)."""
    import torch
    from paper_quant_ph_0308158_gb300 import Simulator, build

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    build.build()
    torch.cuda.set_device(local)
    lo, hi = args.scan_m_min, args.scan_m_max
    rows = []
    clocks = ClockSampler(local)
    clocks.start()
    for M in range(lo, hi + 1):
        cfg = W.config_parity(M)
        steps = cfg["steps"]
        sim = Simulator(M, np.complex64, scratch=False)
        sim.set_strategy("inplace")
        sim.set_canonicalize(False)
        sim.set_jit(args.jit)  # compiled closed pass (--no-jit: tile pass)
        probs = torch.empty(1 << M, dtype=torch.float64, device="cuda")
        sim.load_product_state(cfg["qubits"])
        for _ in range(args.warmup):
            sim.apply_probabilities(steps, probs.data_ptr())
        sim.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            sim.apply_probabilities(steps, probs.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        sim.set_profiling(True)
        sim.apply_probabilities(steps, probs.data_ptr())
        sim.synchronize()
        passes = sim.pass_times()
        sim.set_profiling(False)
        rows.append({"M": M, "L": len(steps), "ms": ms,
                     "amp_steps_per_s": (1 << M) * len(steps) / (ms * 1e-3),
                     "kernels": [k for k, _, _ in passes],
                     "gb_per_s": (1 << M) * (8 + 8 + 8) / (ms * 1e-3) / 1e9})
        sim.close()
        del probs
        torch.cuda.empty_cache()
    clk = clocks.stop()
    growth = [rows[i + 1]["ms"] / rows[i]["ms"] for i in range(len(rows) - 1)]
    top = rows[-1]
    line = {
        "metric": METRIC, "value": top["amp_steps_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": top["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
        "data": "synthetic (the Sec. 4 alternating input from its qubits)",
        "config": {"workload": "parity_scan_M%d_%d" % (lo, hi),
                   "step_includes": "one in-place pass (closed pass, or tile pass with --no-jit) + FP64 probabilities",
                   "per_M": rows,
                   "time_growth_per_qubit": growth,
                   "time_growth_per_qubit_top4_mean": float(np.mean(growth[-4:])) if growth else None,
                   "paper_growth_per_qubit_modi4": 3.4},
        "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": len(rows) *
        (args.steps + args.warmup), "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args, rank, ws, local):
    """Serving: a Poisson stream of simulation requests through qsim_server
    (continuous batching under an HBM budget), FP64 probabilities out.
    Each distinct M uses one seeded random input state from a pinned pool."""
    import torch
    from paper_quant_ph_0308158_gb300 import Server, build

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    build.build()
    torch.cuda.set_device(local)
    m_hi = args.serve_m_max
    dtype = np.dtype(np.complex128)
    # Input states: one pinned block, taken before anything else churns host
    # memory and sliced per M.  Copies from pinned memory scattered over many
    # small physical pieces ran at 25-45 GB/s instead of 211 GB/s on the
    # GB300's host link, so a client should pin large blocks early.
    sizes = {M: 1 << M for M in range(12, m_hi + 1)}
    block = torch.empty(sum(sizes.values()) + 256 * len(sizes), dtype=torch.complex128,
                        pin_memory=True)
    pool, off = {}, 0
    for M in sorted(sizes, reverse=True):
        t = block[off: off + sizes[M]]
        off += sizes[M] + 256
        W.random_state(M, dtype, 5000 + M, out=t.numpy())
        pool[M] = (t, t.numpy())
    specs = W.serving_requests(n=args.serve_requests, rate=args.serve_rate, seed=5,
                               m_range=(12, m_hi), l_range=(100, 5000), mix="cnot")
    budget = int(args.serve_budget_gb * 1e9)
    host_bytes = int(args.serve_host_gb * 1e9)
    srv = Server(budget, host_bytes, dtype)
    srv.set_backfill(args.serve_backfill_ms)
    srv.set_copy_streams(args.serve_copy_streams)
    if args.serve_upload_chunk_mb:
        srv.set_upload_chunk(args.serve_upload_chunk_mb << 20)
    if args.serve_trace:
        srv.set_tracing(True)
    lat = []
    amp_steps = 0.0
    done = 0
    mbytes = {}
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    for sp in specs:
        while True:
            for rid, ms in srv.drain():
                lat.append(ms)
                srv.release(rid)
                done += 1
            if time.perf_counter() - t0 >= sp["arrival"]:
                break
            time.sleep(0.0002)
        srv.submit(sp["M"], pool[sp["M"]][1], sp["steps"])
        amp_steps += float(1 << sp["M"]) * sp["L"]
    while done < len(specs):
        got = srv.drain()
        for rid, ms in got:
            lat.append(ms)
            srv.release(rid)
            done += 1
        if not got:
            time.sleep(0.0005)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    st = srv.stats()
    uploads = None
    if args.serve_trace:
        tr = srv.trace()
        np.savetxt(args.serve_trace, np.column_stack([tr[f] for f in tr.dtype.names]),
                   delimiter=",", header=",".join(tr.dtype.names), comments="", fmt="%.6g")
        # per-copy rates of the state uploads: by request size and over time
        dur = tr["upload_end_ms"] - tr["upload_start_ms"]
        ok = dur > 0
        gbs = (16.0 * np.exp2(tr["M"][ok].astype(np.float64))) / dur[ok] / 1e6
        ms = tr["M"][ok]
        t_mid = 0.5 * (tr["upload_start_ms"][ok] + tr["upload_end_ms"][ok])
        uploads = {"by_M_median_gbs": {int(m): float(np.median(gbs[ms == m])) for m in np.unique(ms)},
                   "p10_p50_p90_gbs": [float(np.percentile(gbs, q)) for q in (10, 50, 90)]}
        if len(t_mid):
            edges = np.linspace(t_mid.min(), t_mid.max() + 1e-9, 11)
            idx = np.digitize(t_mid, edges) - 1
            big = ms >= 26
            uploads["M26plus_median_gbs_by_tenth_of_run"] = [
                float(np.median(gbs[(idx == b) & big])) if np.any((idx == b) & big) else None
                for b in range(10)]
    srv.close()
    lat_a = np.array(lat)
    value = amp_steps / wall
    plain = serve_plain_baseline(specs[:args.serve_plain_requests], pool) \
        if args.serve_plain_requests > 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": len(specs),
        "warmup": 0, "ms_per_step": 1e3 * wall / len(specs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic (seeded Poisson arrivals, circuits and input states)",
        "config": {"workload": "serve%d_poisson%g" % (len(specs), args.serve_rate),
                   "M_range": [12, m_hi], "L_range": [100, 5000], "mix": "cnot",
                   "hbm_budget_bytes": budget, "host_result_bytes": host_bytes,
                   "requests_per_s": len(specs) / wall, "offered_requests_per_s": args.serve_rate,
                   "latency_ms_p50": float(np.percentile(lat_a, 50)),
                   "latency_ms_p99": float(np.percentile(lat_a, 99)),
                   "latency_ms_max": float(lat_a.max()), "wall_s": wall,
                   "rounds": st["rounds"], "peak_hbm_in_use": st["peak_in_use_bytes"],
                   "backfill_ms": args.serve_backfill_ms, "backfilled": st["backfilled"],
                   "copy_streams": args.serve_copy_streams,
                   "upload_chunk_mb": args.serve_upload_chunk_mb, "uploads": uploads,
                   "h2d_gbs_while_busy": st["h2d_bytes"] / max(st["h2d_busy_ms"], 1e-9) / 1e6,
                   "d2h_gbs_while_busy": st["d2h_bytes"] / max(st["d2h_busy_ms"], 1e-9) / 1e6,
                   "h2d_busy_frac": st["h2d_busy_ms"] / (1e3 * wall),
                   "d2h_busy_frac": st["d2h_busy_ms"] / (1e3 * wall),
                   "compute_busy_frac": st["compute_busy_ms"] / (1e3 * wall),
                   "copy_issue_ms_total": st["issue_ms"], "copy_issue_ms_max": st["issue_ms_max"],
                   "step": "one request (submit to FP64 probabilities in host memory)",
                   "plain": plain,
                   "served_over_plain": value / plain["value"] if plain else None},
        "roofline": None, "cpu_baseline": None, "e2e": {"value": value, "unit": UNIT,
                   "h2d_bytes_per_step": float(np.mean([16 << sp["M"] for sp in specs])),
                   "d2h_bytes_per_step": float(np.mean([8 << sp["M"] for sp in specs]))},
        "gpu_launches": st["launches"], "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="adder_m32", choices=["mixed_m28", "adder_m32", "adder_m28", "cnot_m16", "mixed_m24", "cnot_m28", "cnot_m26", "parity_m32", "parity_m28", "hybrid_m28",
                             "batch_cnot", "batch_mixed", "serve", "parity_scan", "gather_floor"])
    ap.add_argument("--batch-size", type=int, default=4096)
    ap.add_argument("--tile-bits", type=int, default=0, help="tile width k (0: default)")
    ap.add_argument("--low-bits", type=int, default=0, help="contiguous low tile bits l (0: default)")
    ap.add_argument("--separate-probs", action="store_true",
                    help="compute probabilities in their own pass after the circuit")
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-m-max", type=int, default=30)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-host-gb", type=float, default=48.0)
    ap.add_argument("--serve-backfill-ms", type=float, default=100.0,
                    help="admit later requests ahead of a head that waited less (-1: FIFO)")
    ap.add_argument("--serve-upload-chunk-mb", type=int, default=0,
                    help="upload each state in copies of this many MiB (0: one copy)")
    ap.add_argument("--serve-copy-streams", type=int, default=2, choices=[1, 2],
                    help="copies in and out on two overlapping streams or on one")
    ap.add_argument("--serve-trace", default="",
                    help="write a per-request timeline (CSV) of the serving run to this path")
    ap.add_argument("--serve-plain-requests", type=int, default=400,
                    help="requests timed one at a time for the plain comparison (0: skip)")
    ap.add_argument("--strategy", default="", choices=["", "auto", "sweep", "tile", "gather", "inplace"],
                    help="force a strategy (default: the workload's)")
    ap.add_argument("--autotune", action="store_true",
                    help="time candidate plans first and keep the fastest (qsim_autotune)")
    ap.add_argument("--scan-m-min", type=int, default=16)
    ap.add_argument("--scan-m-max", type=int, default=33)
    ap.add_argument("--cpu-steps", type=int, default=0,
                    help="oracle steps for cpu_baseline (0: 2 at M >= 31, else 24)")
    ap.add_argument("--ref-steps-per-step", type=int, default=0,
                    help="oracle steps per timed reference step (0: 1 at M >= 31, else 2)")
    ap.add_argument("--no-jit", dest="jit", action="store_false",
                    help="use the general bit-sliced gather instead of compiled kernels")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-coset", action="store_true", help="affine gathers read rows directly")
    ap.add_argument("--coset-run-bits", type=int, default=0, help="coset tile run length r (0: 512 B)")
    ap.add_argument("--coset-stage-kib", type=int, default=0, help="coset pipeline stage (0: 32 KiB)")
    ap.add_argument("--serve-in-line", type=int, default=1200,
                    help="requests of the bounded serving sample on the default line (0: none)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-vs-plain comparison of the default run")
    ap.add_argument("--also", default="mixed_m28,cnot_m28,hybrid_m28,parity_m32",
                    help="comma-separated single-circuit workloads also timed on the same line "
                         "(device-resident, no e2e); empty: none")
    ap.add_argument("--batch-compare", type=int, default=4096,
                    help="circuits in the default run's batched-vs-plain comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--floor-m", type=int, default=28,
                    help="gather_floor: state size (the mixed and CNOT circuits at this M)")
    args = ap.parse_args()
    args.also = [w for w in args.also.split(",") if w]
    if args.warmup < 3 and args.impl == "ours":
        print("note: timing rules want >= 3 warm-up steps", file=sys.stderr)
    rank, ws, local = dist_init()
    if args.impl == "reference":
        rc = run_reference(args, rank, ws)
    elif args.workload.startswith("batch"):
        rc = run_batch(args, rank, ws, local)
    elif args.workload == "serve":
        rc = run_serve(args, rank, ws, local) if rank == 0 else 0
    elif args.workload == "gather_floor":
        rc = run_gather_floor(args, rank, ws, local) if rank == 0 else 0
    elif args.workload == "parity_scan":
        rc = run_parity_scan(args, rank, ws, local) if rank == 0 else 0
    else:
        rc = run_ours(args, rank, ws, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
