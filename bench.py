#!/usr/bin/env python3
"""Benchmark: checkerboard-Metropolis sweeps of the 2D Ising beta scan.

Workload (default): 2D square lattice L = 8192 (67,108,864 sites), 16 betas
evenly spaced in [0.30, 0.60], cold start (all +1), seeds 20031109 + j, E and M
recorded after every sweep, run in the int8 layout and again in the
bit-packed layout.  One step = one sweep (black pass, white pass, fused E/M)
of each of the 16 lattices in turn, so the 1 GiB of int8 spin state that a
step touches is far larger than the 129 MB L2 between timed iterations.  The
default K = 2000 steps is the full run of the workload; the lattices are
re-initialised (cold) inside the timed region; `value` covers both layouts.

Metric: site updates per second (attempted single-spin Metropolis updates,
one per site per sweep), whole job over all ranks.

Arms
  default          the CUDA engine (C ABI via ctypes), device-timed with CUDA
                   events; plus an end-to-end figure through the same public
                   API with host buffers (initial spins uploaded from pinned
                   host memory, E/M read back to the host every step, final
                   spins read back), a roofline object for the int8 pass
                   kernel, clock samples, and the CPU oracle timed on a
                   bounded sample (rank 0, N = 1).
  --impl reference the CPU oracle (single-threaded C) on the same workload,
                   each step a bounded sample sized so the run ends in
                   minutes.

Multi-GPU (torchrun): every rank runs its own 16 independent lattices (seeds
offset by 16 * rank), no collective on the data path; scaling "weak".

--rule heatbath runs the same workload with the heat-bath update rule (every
site draws; flip iff u < floor(2^32 / (1 + exp(beta dE)))) instead of the
Metropolis rule, in the engine and in the oracle arms alike.  --rule demon
runs Creutz's deterministic demon dynamics: cold spins and demons (qmax 3)
drawn at each lattice's beta; no draws; 5 bytes per update in int8, 7 bits
in the bit-packed layout.
"""
from __future__ import annotations

import argparse
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

L_SCAN = 8192
N_BETA = 16
BASE_SEED = 20031109
BYTES_PER_UPDATE_INT8 = 3  # per colour pass: read own N/2, read other N/2, write own N/2
BYTES_PER_UPDATE_DEMON = 5  # and read + write the own colour's demons (1 byte per site)
BYTES_PER_UPDATE_DEMON_PACKED = 7 / 8  # bits: own, other, 2 demon planes read; own, 2 written
DEMON_QMAX = 3


# DRAM bytes per site update of the pass kernels, from one
# `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum` capture of the
# bench's own run per workload (profiles/dram_traffic_bench_scan_L8192.md,
# profiles/dram_traffic_bench_big_L65536.md, profiles/dram_traffic_bench_demon.md).  They describe the kernel sources
# whose code hash (comments left out) is recorded; any change to that code
# makes the bench report "traffic": null until the capture is redone.
TRAFFIC = {
    ("scan", "int8"): {"bytes_per_update": 1.9506,
        "sha1": "1abb33311d8df4c6572058f296e0a0424c106a7f",
        "sources": ["sweep_int8_tma.cu", "pass_bodies.cuh", "ising_device.cuh"]},
    ("scan", "bitpack"): {"bytes_per_update": 0.2146,
        "sha1": "a8e8b2f4bd8de47a7be802a2cd50b7ee8649b8f8",
        "sources": ["sweep_bitpack.cu", "pass_bodies.cuh", "ising_device.cuh"]},
    ("big", "int8"): {"bytes_per_update": 3.0130,
        "sha1": "26576c343dcce05b584d2b0a6f7f410a779ff5a4",
        "sources": ["sweep_int8.cu", "pass_bodies.cuh", "ising_device.cuh"]},
    ("big", "bitpack"): {"bytes_per_update": 0.3900,
        "sha1": "a8e8b2f4bd8de47a7be802a2cd50b7ee8649b8f8",
        "sources": ["sweep_bitpack.cu", "pass_bodies.cuh", "ising_device.cuh"]},
    ("scan", "demon"): {"bytes_per_update": 4.4847,
        "sha1": "194d7a49755ca93f859297cf549f9ac9b7c89468",
        "sources": ["sweep_demon.cu", "pass_bodies.cuh", "ising_device.cuh"]},
    ("scan", "demon_packed"): {"bytes_per_update": 0.6969,
        "sha1": "194d7a49755ca93f859297cf549f9ac9b7c89468",
        "sources": ["sweep_demon.cu", "pass_bodies.cuh", "ising_device.cuh"]},
    ("big", "demon"): {"bytes_per_update": 5.0088,
        "sha1": "194d7a49755ca93f859297cf549f9ac9b7c89468",
        "sources": ["sweep_demon.cu", "pass_bodies.cuh", "ising_device.cuh"]},
    ("big", "demon_packed"): {"bytes_per_update": 0.8672,
        "sha1": "194d7a49755ca93f859297cf549f9ac9b7c89468",
        "sources": ["sweep_demon.cu", "pass_bodies.cuh", "ising_device.cuh"]},
}


def code_only(text: str) -> str:
    """Source text without comments, with runs of blanks collapsed and empty
    lines dropped, so that a comment or layout edit does not mark a traffic
    capture stale."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    lines = (" ".join(re.sub(r"//.*$", "", ln).split()) for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln)


def kernel_sources_sha1(names) -> str:
    """Hash of the code (comments left out) of the kernel sources a traffic
    capture describes."""
    import hashlib
    h = hashlib.sha1()
    for n in names:
        with open(os.path.join(ROOT, "paper_cs_0312006_gb300", "csrc", n), encoding="utf-8") as f:
            h.update(code_only(f.read()).encode())
    return h.hexdigest()


def measured_traffic(workload: str, layout: str, updates_per_launch: int,
                     rule: str = "metropolis"):
    t = TRAFFIC.get((workload, layout))
    if t is None:
        return None
    if rule != "metropolis":  # the capture covers the Metropolis instances only
        return None
    if t["bytes_per_update"] is None or kernel_sources_sha1(t["sources"]) != t["sha1"]:
        return None
    return t["bytes_per_update"] * updates_per_launch


def issue_schedule(n_lattices: int, steps: int, order: str = "wave"):
    """The e2e leg's issue order: a list of wavefronts, each a list of
    (lattice, sweep) pairs.  "step": wavefront k holds every lattice's sweep
    k.  "wave": lattice j's sweep k is in wavefront k + j, so lattice j starts
    j wavefronts after lattice 0 (its upload has more of the others' sweeps to
    hide behind) and every lattice still runs its sweeps in order."""
    skew = 1 if order == "wave" else 0
    waves = []
    for wave in range(steps + skew * (n_lattices - 1)):
        waves.append([(j, wave - skew * j) for j in range(n_lattices)
                      if 0 <= wave - skew * j < steps])
    return waves


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest of every rank's value (the job's time is its slowest rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def scan_betas():
    return [round(0.30 + 0.02 * j, 10) for j in range(N_BETA)]


def workload_config(L: int, steps: int, lattices: int = N_BETA,
                    rule: str = "metropolis", big: bool = False) -> dict:
    name = {"metropolis": "checkerboard Metropolis", "heatbath": "checkerboard heat-bath",
            "demon": f"deterministic demon dynamics, qmax={DEMON_QMAX}"}[rule]
    if big:
        text = (f"2D Ising single lattice ({name}): L={L} square lattice ({L * L} sites, "
                f"{L * L // 2 // 2 ** 20} MiB per colour in int8), beta=0.30, cold start, "
                f"{steps} sweeps, E/M every sweep, int8 and bit-packed layouts")
    else:
        text = (f"2D Ising beta scan ({name}): L={L} square lattice, 16 betas evenly spaced in "
                f"[0.30,0.60], cold start, {steps} sweeps, E/M every sweep, int8 and bit-packed "
                f"layouts")
    return {"workload": text,
            "rule": rule,
            "lattices_per_gpu": lattices,
            "l2": f"inputs larger than L2: a step touches {lattices} x L^2 bytes of int8 spins",
            "step": "one sweep (black pass, white pass, fused E/M) of each lattice"}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []
        self.times = []

    def start(self, wait_s: float = 5.0):
        """Start sampling every 50 ms and wait (at most wait_s) for the first
        sample, so that a short timed region that follows is covered."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
            return
        t_end = time.time() + wait_s
        while not self.lines and time.time() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.times.append(time.time())

    def count_since(self, t0: float) -> int:
        return sum(1 for t in list(self.times) if t >= t0)

    def stop(self, since: float = 0.0):
        """Summarise the samples taken at or after `since` (time.time())."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln, t in zip(list(self.lines), list(self.times)):
            if t < since:
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_demon_rate(budget_s: float, L: int, betas, n_lattices: int):
    """The oracle's demon dynamics on cold lattices with demons at each beta."""
    import oracle
    from paper_cs_0312006_gb300 import workloads
    oracle.build()
    done, j, spent = 0, 0, 0.0
    while True:
        b = betas[j % len(betas)]
        q = workloads.demon_field(L * L, DEMON_QMAX, b, BASE_SEED + (j % len(betas)))
        s = np.ones(L * L, dtype=np.int8)
        t0 = time.perf_counter()
        oracle.run_demon(2, L, s, q, DEMON_QMAX, 1, measure_every=1)
        spent += time.perf_counter() - t0
        done += L * L
        j += 1
        if spent >= budget_s or j >= n_lattices:
            break
    return done / spent, f"{j} single demon sweeps (E/M after each) of 2D L={L} lattices"


def oracle_sample_rate(budget_s: float, L: int, betas, n_lattices: int, heatbath: bool = False):
    """Time the oracle (as it stands) sweeping cold-started lattices of size L
    with E/M recomputed after each sweep; returns (updates/s, description)."""
    import oracle
    oracle.build()
    done = 0
    t0 = time.perf_counter()
    j = 0
    while True:
        b = betas[j % len(betas)]
        oracle.run(2, L, b, BASE_SEED + (j % len(betas)), 1, measure_every=1,
                   start=oracle.COLD_UP, heatbath=heatbath)
        done += L * L
        j += 1
        if time.perf_counter() - t0 >= budget_s or j >= n_lattices:
            break
    dt = time.perf_counter() - t0
    return done / dt, (f"{j} single sweeps (cold start, E/M after each) of 2D L={L} lattices"
                       + (", heat-bath rule" if heatbath else ""))


def host_description() -> dict:
    """The host the CPU baseline ran on: logical cores and the CPU model."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    import platform
    return {"nproc": os.cpu_count(), "machine": platform.machine(), "cpu": model}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    betas = scan_betas()
    total_steps = args.steps + args.warmup
    # each step sweeps one lattice once; pick the largest L <= 8192 whose whole
    # run stays within ~90 s at the oracle's ~2.5e7 updates/s
    L = args.L
    while L > 64 and total_steps * L * L / 2.5e7 > 90.0:
        L //= 2
    import oracle
    oracle.build()
    hb = args.rule == "heatbath"
    if args.rule == "demon":
        from paper_cs_0312006_gb300 import workloads
        # every lattice's demons are drawn before the clock starts
        fields = [workloads.demon_field(L * L, DEMON_QMAX, b, BASE_SEED + j)
                  for j, b in enumerate(betas)]
        cold = np.ones(L * L, dtype=np.int8)

        def step(j):
            oracle.run_demon(2, L, cold, fields[j], DEMON_QMAX, 1)

        for w in range(args.warmup):
            step(w % N_BETA)
        t0 = time.perf_counter()
        for k in range(args.steps):
            step(k % N_BETA)
        dt = time.perf_counter() - t0
        return _reference_line(args, world, L, dt, "demon sweep")
    for w in range(args.warmup):
        oracle.run(2, L, betas[w % N_BETA], BASE_SEED + w, 1, measure_every=1,
                   start=oracle.COLD_UP, heatbath=hb)
    t0 = time.perf_counter()
    for k in range(args.steps):
        j = k % N_BETA
        oracle.run(2, L, betas[j], BASE_SEED + j, 1, measure_every=1, start=oracle.COLD_UP,
                   heatbath=hb)
    dt = time.perf_counter() - t0
    return _reference_line(args, world, L, dt, "sweep")


def _reference_line(args, world, L, dt, what):
    total_steps = args.steps + args.warmup
    value = args.steps * L * L / dt
    sample = (f"each step: one {what} (cold start, E/M recomputed) of one 2D L={L} lattice "
              f"of the 16-beta scan (beta cycling), single-threaded C oracle; the workload's "
              f"L={args.L} is sampled at L={L} so that {total_steps} steps end in minutes")
    line = {
        "impl": "reference", "metric": "site updates/s", "value": value,
        "unit": "site updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": workload_config(args.L, args.steps, args.lattices, args.rule),
        "cpu_baseline": {"value": value, "unit": "site updates/s", "cores": 1,
                         "kind": "oracle", "sample": sample, "host": host_description()},
        "e2e": {"value": value, "unit": "site updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args, world, rank, local):
    import torch

    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the engine has no CPU path)")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_cs_0312006_gb300 import _build, engine
    _build.build()
    engine.load_library()

    L = args.L
    n_sites = L * L
    betas = scan_betas()[:args.lattices]
    layouts = [("int8", engine.INT8), ("bitpack", engine.BITPACK)]
    if args.layout != "both":
        layouts = [x for x in layouts if x[0] == args.layout]

    stream = torch.cuda.current_stream()
    int8_kernel = {"auto": engine.KERNEL_AUTO, "strip": engine.KERNEL_STRIP,
                   "tma": engine.KERNEL_TMA}[args.int8_kernel]
    int8_tuned = None
    if int8_kernel == engine.KERNEL_AUTO and args.layout in ("both", "int8"):
        # the int8 pass configuration for this lattice shape, measured (or read
        # from the cache) and registered so that ISING_KERNEL_AUTO runs it
        from paper_cs_0312006_gb300 import autotune
        int8_tuned = autotune.tune_int8(2, L, use_cache=not args.retune)
    rule = {"metropolis": engine.RULE_METROPOLIS, "heatbath": engine.RULE_HEATBATH,
            "demon": engine.RULE_METROPOLIS}[args.rule]
    sets = {name: [engine.Lattice(2, L, b, BASE_SEED + 16 * rank + j, layout=lay,
                                  start=engine.COLD_UP, stream=stream, kernel=int8_kernel,
                                  rule=rule)
                   for j, b in enumerate(betas)] for name, lay in layouts}

    if args.rule == "demon":
        from paper_cs_0312006_gb300 import workloads
        fields = [workloads.demon_field(n_sites, DEMON_QMAX, b, BASE_SEED + 16 * rank + j)
                  for j, b in enumerate(betas)]
        for lats in sets.values():
            for j, lat in enumerate(lats):
                lat.set_demons(fields[j], qmax=DEMON_QMAX)
                lat.set_rule(engine.RULE_DEMON)
        del fields
    int8_ran = sets["int8"][0].kernel() if "int8" in sets else -1
    int8_cfg = sets["int8"][0].int8_config() if "int8" in sets else None

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---------------- warm-up ----------------
    sampler = ClockSampler(local)
    sampler.start()
    for lats in sets.values():
        for _ in range(args.warmup):
            for lat in lats:
                lat.sweep(1, 1)
    # the same sweeps for a moment more (at least 0.3 s and 5 clock samples,
    # at most 3 s), so that the clock record covers the GPU under this load:
    # the timed region of a short run is shorter than the sampling interval
    soak_from = time.time()
    while time.time() - soak_from < 3.0:
        for lats in sets.values():
            for lat in lats:
                lat.sweep(1, 1)
        torch.cuda.synchronize()
        if time.time() - soak_from >= 0.3 and sampler.count_since(soak_from) >= 5:
            break
    for lats in sets.values():
        for lat in lats:
            lat.observables()
    torch.cuda.synchronize()

    # ---------------- device-timed value ----------------
    barrier()
    torch.cuda.synchronize()
    marks = {}
    pairs = {name: [] for name in sets}
    start = torch.cuda.Event(enable_timing=True)
    # at least ~20 timed steps per layout, however short the run
    every = max(1, min(args.time_every, args.steps // 20))
    start.record(stream)
    for name, lats in sets.items():
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for lat in lats:
            lat.init(engine.COLD_UP)
        for k in range(args.steps):
            # a timed step is bracketed as a whole: its 2 x 16 passes run back
            # to back, so the events break no chained launch inside it
            time_this = k % every == 0
            if time_this:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            for lat in lats:
                lat.sweep(1, 1)
            if time_this:
                e1.record(stream)
                pairs[name].append((e0, e1))
        b1.record(stream)
        marks[name] = (b0, b1)
    stop = torch.cuda.Event(enable_timing=True)
    stop.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop(since=soak_from)
    if clocks is not None:
        clocks["window"] = "the same sweeps just before the timed region, and the timed region"
    ms_all = max_over_ranks(start.elapsed_time(stop), world, device="cuda")
    per_layout_updates = world * len(betas) * n_sites * args.steps
    # the headline is the int8 layout's whole job (its own bracket of events),
    # the other layout is reported beside it
    head = "int8" if "int8" in sets else next(iter(sets))
    ms = max_over_ranks(marks[head][0].elapsed_time(marks[head][1]), world, device="cuda")
    value = per_layout_updates / (ms / 1e3)
    for lats in sets.values():  # every step recorded one (E, M) per lattice
        n_rec = [len(lat.observables()[0]) for lat in lats]
        assert all(n == args.steps for n in n_rec), n_rec

    peak_hbm, peak_kind = load_peaks()
    # the integer ceiling: the device generator alone, measured here (outside
    # the timed region) -- every site with dE > 0 needs one 32-bit draw
    ceiling = measure_philox_ceiling(engine, torch)
    layout_stats = {}
    rooflines = {}
    for name in sets:
        part_ms = marks[name][0].elapsed_time(marks[name][1])
        # average launch: the timed steps' time over their passes (2 per lattice)
        pass_ms = (sum(a.elapsed_time(b) for a, b in pairs[name]) /
                   (2 * len(sets[name]) * len(pairs[name])))
        updates_per_pass = n_sites // 2
        layout_stats[name] = {"value": world * len(betas) * n_sites * args.steps / (part_ms / 1e3),
                              "ms": part_ms, "pass_ms": pass_ms,
                              "pass_updates_per_s": updates_per_pass / (pass_ms / 1e3)}
        if name == "int8" and args.rule == "demon":
            bytes_per_pass = BYTES_PER_UPDATE_DEMON * updates_per_pass
            achieved = bytes_per_pass / (pass_ms / 1e3) / 1e9
            rooflines[name] = {"kernel": "pass_demon_strip<2,measure>", "bound": "hbm",
                               "achieved": achieved, "peak": peak_hbm, "unit": "GB/s",
                               "frac": achieved / peak_hbm,
                               "traffic": measured_traffic(args.workload, "demon",
                                                           updates_per_pass),
                               "bytes_per_launch": bytes_per_pass, "launch_ms": pass_ms,
                               "peak_source": f"{peak_kind} hbm_gbs (copy)"}
        elif name == "int8":
            bytes_per_pass = BYTES_PER_UPDATE_INT8 * updates_per_pass
            achieved = bytes_per_pass / (pass_ms / 1e3) / 1e9
            rtag = "" if args.rule == "metropolis" else ",heatbath"
            kname = (f"pass_int8_tma<2,measure{rtag}>" if int8_ran == engine.KERNEL_TMA else
                     f"pass_int8_strip<2,measure{rtag}>")
            upd_s = updates_per_pass / (pass_ms / 1e3)
            rooflines[name] = {"kernel": kname, "bound": "hbm",
                               "achieved": achieved, "peak": peak_hbm, "unit": "GB/s",
                               "frac": achieved / peak_hbm,
                               "traffic": measured_traffic(args.workload, "int8",
                                                           updates_per_pass, args.rule),
                               "bytes_per_launch": bytes_per_pass, "launch_ms": pass_ms,
                               "peak_source": f"{peak_kind} hbm_gbs (copy)",
                               "philox_ceiling_updates_per_s": ceiling["draws_per_s"],
                               "frac_of_philox_ceiling": upd_s / ceiling["draws_per_s"]}
        elif args.rule == "demon":  # bit-packed demons: 7 bits per update, no draws
            bytes_per_pass = BYTES_PER_UPDATE_DEMON_PACKED * updates_per_pass
            achieved = bytes_per_pass / (pass_ms / 1e3) / 1e9
            kname = ("pass_demon_packed4<2,measure>" if (L // 2) % 128 == 0 else
                     "pass_demon_packed<2,measure>")
            rooflines[name] = {"kernel": kname, "bound": "hbm",
                               "achieved": achieved, "peak": peak_hbm, "unit": "GB/s",
                               "frac": achieved / peak_hbm,
                               "traffic": measured_traffic(args.workload, "demon_packed",
                                                           updates_per_pass),
                               "bytes_per_launch": bytes_per_pass, "launch_ms": pass_ms,
                               "peak_source": f"{peak_kind} hbm_gbs (copy)"}
        else:
            peak = ceiling["draws_per_s"]
            achieved = updates_per_pass / (pass_ms / 1e3)
            rtag = "" if args.rule == "metropolis" else ",heatbath"
            rooflines[name] = {"kernel": f"pass_packed<2,measure{rtag}>", "bound": "alu",
                               "achieved": achieved, "peak": peak, "unit": "site updates/s",
                               "frac": achieved / peak,
                               "traffic": measured_traffic(args.workload, "bitpack",
                                                           updates_per_pass, args.rule),
                               "launch_ms": pass_ms,
                               "peak_source": "measured in this run: Philox4x32-10 calls/s of "
                                              "the generator alone (ising_philox_probe) x 4 "
                                              "draws per call (one draw per site update)"}

    # ---------------- end to end through the C ABI, host buffers ----------------
    e2e = None
    if not args.no_e2e:
        e2e = {}
        e2e_steps = args.e2e_steps or args.steps
        # every lattice's initial and final spins live in pinned host memory.
        # The host<->device copies run on the copy engines of a second stream
        # and overlap the other lattices' sweeps: lattice j's upload lands in a
        # device buffer that ising_set_spins_async reads once its copy event
        # has passed, and its final spins (ising_get_spins_async into a device
        # buffer) go down while the later lattices finish their last sweep.
        # Each wavefront's (E, M) pairs land in one half of a pinned double
        # buffer (one gather kernel) and are summed on the host while the next
        # wavefront runs.  By default lattice j's sweep k runs in wavefront
        # k + j (--e2e-order wave): the first lattices sweep while the later
        # ones are still uploaded, and the last ones while the first go down
        # (measured 0.92 of the device-timed rate against 0.72 in step order,
        # whose first and last steps wait on the copies).
        host_init = torch.ones(n_sites, dtype=torch.int8).pin_memory()
        host_out = [torch.empty(n_sites, dtype=torch.int8).pin_memory() for _ in betas]
        dev_in = [torch.empty(n_sites, dtype=torch.int8, device="cuda") for _ in betas]
        dev_out = [torch.empty(n_sites, dtype=torch.int8, device="cuda") for _ in betas]
        pairs = torch.zeros((2, len(betas), 2), dtype=torch.int64).pin_memory().numpy()
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        copy_streams = [torch.cuda.Stream() for _ in range(max(1, args.e2e_copy_streams))]
        # each layout's leg runs three times (host wall clock over a ~30 ms leg
        # at 20 steps is exposed to host scheduling); the median is reported
        # and every repeat listed
        for name, lats in [(n, l) for n, l in sets.items() for _ in range(3)]:
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h2d = d2h = 0
            host_sum = 0
            n_valid = [0, 0]  # records gathered into each half of the pinned buffer
            uploaded = []
            direct = args.e2e_mode == "direct"
            if not direct:
                for j in range(len(lats)):  # H2D: every lattice's initial configuration
                    cs = copy_streams[j % len(copy_streams)]
                    with torch.cuda.stream(cs):
                        dev_in[j].copy_(host_init, non_blocking=True)
                        ev = torch.cuda.Event()
                        ev.record(cs)
                        uploaded.append(ev)
            last = None
            # wave order: lattice j runs its sweep k in wavefront k + j, so that
            # the lattices whose uploads have landed run ahead while the later
            # ones are still copied (the lattices are independent: the same
            # sweeps and results, only their interleaving differs); one
            # records gather per wavefront
            for wave, work in enumerate(issue_schedule(len(lats), e2e_steps, args.e2e_order)):
                for j, k in work:
                    lat = lats[j]
                    if k == 0:
                        if direct:  # the import kernel reads the pinned host buffer itself
                            lat.set_spins_async(host_init.data_ptr(), 0)
                        else:
                            stream.wait_event(uploaded[j])
                            lat.set_spins_async(dev_in[j].data_ptr(), 0)
                        h2d += n_sites
                    lat.sweep(1, 1)
                    if k == e2e_steps - 1:  # D2H of the final configuration
                        if direct:  # the export kernel writes the pinned host buffer
                            lat.get_spins_async(host_out[j].data_ptr())
                        else:
                            lat.get_spins_async(dev_out[j].data_ptr())
                            done = torch.cuda.Event()
                            done.record(stream)
                            cs = copy_streams[j % len(copy_streams)]
                            cs.wait_event(done)
                            with torch.cuda.stream(cs):
                                host_out[j].copy_(dev_out[j], non_blocking=True)
                        d2h += n_sites
                half = wave % 2
                n_valid[half] = int(engine.observables_gather(lats, pairs[half]).sum())
                d2h += 16 * n_valid[half]
                ready[half].record(stream)
                if last is not None:
                    ready[last].synchronize()
                    host_sum += int(pairs[last, :n_valid[last], 0].sum())
                last = half
            torch.cuda.synchronize()
            host_sum += int(pairs[last, :n_valid[last], 0].sum())
            dt = max_over_ranks(time.perf_counter() - t0, world, device="cuda")
            for lat in lats:
                lat.synchronize()  # a bounded wait or an invalid input would be reported here
            e2e.setdefault(name, []).append(
                {"value": world * len(betas) * n_sites * e2e_steps / dt,
                 "seconds": dt, "h2d_bytes": h2d, "d2h_bytes": d2h,
                 "h2d_bytes_per_step": h2d / e2e_steps,
                 "d2h_bytes_per_step": d2h / e2e_steps,
                 # the copies' bytes over the leg's wall time (they overlap
                 # the sweeps, so this is what the job moved, not a link rate)
                 "h2d_gb_per_s": h2d / dt / 1e9, "d2h_gb_per_s": d2h / dt / 1e9,
                 # the host's own sum of every E record it read (same for every leg)
                 "records_E_sum": host_sum})
        for name, legs in e2e.items():
            med = sorted(legs, key=lambda x: x["value"])[len(legs) // 2]
            e2e[name] = dict(med, repeats=[x["value"] for x in legs])
        del dev_in, dev_out
        head_e2e = e2e[head]
        e2e = {"value": head_e2e["value"], "unit": "site updates/s",
               "h2d_bytes_per_step": head_e2e["h2d_bytes_per_step"],
               "d2h_bytes_per_step": head_e2e["d2h_bytes_per_step"],
               "h2d_gb_per_s": head_e2e["h2d_gb_per_s"],
               "d2h_gb_per_s": head_e2e["d2h_gb_per_s"], "steps": e2e_steps,
               "mode": args.e2e_mode, "order": args.e2e_order,
               "layout": head, "layouts": e2e,
               "over_device_value": head_e2e["value"] / value,
               "note": "per layout: every lattice's initial spins copied from pinned host "
                       "memory on a copy stream and loaded with ising_set_spins_async, then per "
                       "step one sweep of each lattice and one ising_observables_gather of "
                       "every lattice's (E, M) into pinned host memory (read on the host while "
                       "the next step runs); each lattice's final spins written by "
                       "ising_get_spins_async and copied to pinned host memory on the copy "
                       "stream while the later lattices finish"}

    for lats in sets.values():
        for lat in lats:
            lat.close()

    if rank != 0:
        return 0

    cpu = None
    if world == 1 and not args.no_cpu_baseline and args.rule == "demon":
        rate, sample = oracle_demon_rate(args.cpu_seconds, L_SCAN, betas, 64)
        cpu = {"value": rate, "unit": "site updates/s", "cores": 1, "kind": "oracle",
               "sample": sample, "host": host_description()}
    elif world == 1 and not args.no_cpu_baseline:
        rate, sample = oracle_sample_rate(args.cpu_seconds, L_SCAN, betas, 64,
                                          heatbath=args.rule == "heatbath")
        cpu = {"value": rate, "unit": "site updates/s", "cores": 1, "kind": "oracle",
               "sample": sample, "host": host_description()}

    forms = {}
    if world == 1 and not args.no_forms and args.rule == "metropolis":
        forms["small"] = small_form(args)
        forms["cubic"] = cubic_form(args, peak_hbm, ceiling)
        forms["batched"] = batched_form(args)
        forms["serving"] = serving_form(args)

    line = {
        "metric": "site updates/s", "value": value, "unit": "site updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
        "data": "synthetic",
        "config": workload_config(L, args.steps, len(betas), args.rule,
                                  big=args.workload == "big"),
        "pass_timing": f"CUDA events around each lattice's sweep on every {every}th step of "
                       f"the timed region (the events sit between sweeps, so fewer of them "
                       f"disturb the chained launches less)",
        "headline_layout": head,
        "layouts": layout_stats,
        "both_layouts": {"value": per_layout_updates * len(sets) / (ms_all / 1e3),
                         "ms": ms_all},
        "roofline": rooflines.get("int8") or rooflines.get("bitpack"),
        "roofline_bitpack": rooflines.get("bitpack"),
        "philox_ceiling": ceiling,
        "int8_config": {"ran": int8_cfg,
                        "tuned": None if int8_tuned is None else
                        {"config": int8_tuned["config"],
                         "candidates": [{"config": r["config"],
                                         "site_updates_per_s": r["site_updates_per_s"]}
                                        for r in int8_tuned["results"]]}},
        "gpu_launches": len(sets) * len(betas) * 2 * args.steps,
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    line.update(forms)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def batched_form(args) -> dict:
    """The batched form on its full workload (2048 lattices x 500 sweeps):
    one persistent launch against one ising_sweep per lattice (one stream and
    eight streams); every lattice bit-identical across the forms."""
    import torch
    from paper_cs_0312006_gb300 import autotune, batched, engine, workloads
    specs = workloads.batched_mix(n=args.batch_lattices, sweeps=args.batch_sweeps)
    tuned = autotune.tune(specs, use_cache=not args.retune)
    opts, layout = tuned["opts"], tuned["layout"]
    batched.run_batched(batched.scaled(specs[:64], 2), opts, 1, layout)  # warm-up
    res = batched.compare_forms(specs, opts, layout)
    if res["mismatches"]:
        raise SystemExit(f"batched and plain forms differ on {res['mismatches']} lattices")
    return {"config": {"workload": f"batched: {res['lattices']} lattices, {args.batch_sweeps} "
                                   "sweeps each, 70% 2D L log-uniform [16,1024] beta U[0.2,0.6], "
                                   "30% 3D L log-uniform [8,128] beta U[0.15,0.30], hot start, "
                                   "E/M every 10 sweeps"},
            "value": res["batched_updates_per_s"], "unit": "site updates/s",
            "plain_value": res["plain_updates_per_s"],
            "batched_over_plain": res["batched_over_plain"],
            "batched_over_plain_8_streams": res["batched_over_plain_8_streams"],
            "detail": res,
            "autotune": {"opts": opts, "layout": layout, "candidates": len(tuned["results"]),
                         "choice": tuned.get("choice")}}


def serving_form(args) -> dict:
    """The serving form on its full workload (Poisson job stream) against the
    plain form (each job alone through ising_sweep, in arrival order)."""
    from paper_cs_0312006_gb300 import serve, workloads
    jobs = workloads.poisson_jobs(args.serve_jobs, rate_per_s=args.serve_rate)
    warm = workloads.poisson_jobs(8, rate_per_s=1e6, seed=99, l2d=(32, 128), l3d=(16, 32),
                                  sweeps=(10, 20))
    serve.Server(round_s=args.round_s).run(warm)  # load and warm the kernels
    srv = serve.Server(hbm_budget_bytes=int(args.hbm_budget_gb * 1e9), round_s=args.round_s,
                       keep_spins=False)
    summ = srv.run(jobs)
    skip = max(0, len(jobs) // 10)
    pct = serve.percentile_summary(srv.results, skip)
    psum, pres = serve.run_plain_fifo(jobs)
    plain = dict(psum, **serve.percentile_summary(pres, skip))
    return {"config": {"workload": f"serving: {len(jobs)} Poisson jobs at {args.serve_rate}/s, "
                                   "dims 2/3, L log-uniform (2D 32-4096, 3D 16-256), beta_c +- "
                                   "0.05, sweeps log-uniform 100-20000, E/M every 10, HBM budget "
                                   f"{args.hbm_budget_gb} GB; first {skip} jobs left out of the "
                                   "percentiles"},
            "value": summ["updates_per_s"], "unit": "site updates/s",
            "p50_latency_s": pct["p50_latency_s"], "p99_latency_s": pct["p99_latency_s"],
            "plain_value": plain["updates_per_s"],
            "plain_p50_latency_s": plain["p50_latency_s"],
            "plain_p99_latency_s": plain["p99_latency_s"],
            "served_over_plain": summ["updates_per_s"] / plain["updates_per_s"],
            "offered_load_updates_per_s": serve.offered_load(jobs, args.serve_rate),
            "detail": dict(summ, **pct)}


def cubic_form(args, peak_hbm: float, ceiling: dict) -> dict:
    """3D cubic L=256 (16.8 M sites) at beta 0.2216544, hot start, seed
    20031109, 1000 sweeps with E/M every 10 sweeps, in both layouts; the int8
    pass configuration tuned for this shape; the int8 pass against the HBM
    roofline (3 B per update) and the Philox ceiling."""
    import torch
    from paper_cs_0312006_gb300 import autotune, engine
    L, beta, n = args.cubic_L, 0.2216544, args.cubic_sweeps
    sites = L ** 3
    tuned = autotune.tune_int8(3, L, use_cache=not args.retune)
    out = {}
    for name, lay in (("int8", engine.INT8), ("bitpack", engine.BITPACK)):
        lat = engine.Lattice(3, L, beta, BASE_SEED, layout=lay)
        lat.sweep(3, 10)  # warm-up
        lat.observables()
        lat.init(engine.HOT)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        lat.sweep(n, 10)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b)
        E, M = lat.observables()
        cfg = lat.int8_config()
        lat.close()
        rate = sites * n / (ms / 1e3)
        out[name] = {"value": rate, "ms": ms, "records": len(E), "us_per_sweep": ms * 1e3 / n,
                     "int8_config": cfg if name == "int8" else None}
    int8_rate = out["int8"]["value"]
    achieved = BYTES_PER_UPDATE_INT8 * int8_rate / 1e9
    return {"config": {"workload": f"3D cubic L={L}, beta 0.2216544, hot start, seed "
                                   f"{BASE_SEED}, {n} sweeps, E/M every 10 sweeps, int8 and "
                                   "bit-packed layouts"},
            "value": int8_rate, "unit": "site updates/s", "layouts": out,
            "int8_tuned": tuned["config"],
            "roofline": {"kernel": "int8 pass (tuned configuration), 3D", "bound": "hbm",
                         "achieved": achieved, "peak": peak_hbm, "unit": "GB/s",
                         "frac": achieved / peak_hbm, "traffic": None,
                         "frac_of_philox_ceiling": int8_rate / ceiling["draws_per_s"],
                         "note": "whole sweeps timed (both passes, fused E/M every 10 "
                                 "sweeps); the lattice (16 MiB in int8) stays resident in "
                                 "the 129 MB L2, so HBM is not what its passes stream from"}}


def small_form(args) -> dict:
    """The critical 2D L=64 run: beta 0.4406868, hot start, seed 20031109,
    1000 sweeps with E/M every sweep, one single-CTA launch, in both layouts;
    median of five runs.  (Its parity with the oracle is a test,
    tests/test_gpu_parity.py; here the two layouts are checked against each
    other, bit for bit.)"""
    import numpy as np
    import torch
    from paper_cs_0312006_gb300 import engine
    L, beta, n = 64, 0.4406868, 1000
    out, states = {}, []
    for name, lay in (("int8", engine.INT8), ("bitpack", engine.BITPACK)):
        lat = engine.Lattice(2, L, beta, BASE_SEED, layout=lay)
        lat.sweep(n, 1)  # warm-up run
        lat.observables()
        times = []
        for _ in range(5):
            lat.init(engine.HOT)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            lat.sweep(n, 1)
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b))
        E, M = lat.observables()
        states.append((lat.get_spins(), E[-n:], M[-n:]))
        lat.close()
        ms = sorted(times)[len(times) // 2]
        out[name] = {"value": L * L * n / (ms / 1e3), "us_per_sweep": ms * 1e3 / n}
    agree = all(np.array_equal(x, y) for x, y in zip(states[0], states[1]))
    return {"config": {"workload": "2D L=64, beta 0.4406868, hot start, seed 20031109, 1000 "
                                   "sweeps, E/M every sweep, int8 and bit-packed layouts"},
            "value": out["int8"]["value"], "unit": "site updates/s",
            "us_per_sweep": out["int8"]["us_per_sweep"], "layouts_bit_identical": agree,
            "layouts": out}

def run_batched_workload(args):
    """2048 independent lattices (70% 2D L in [16,1024], 30% 3D L in [8,128],
    log-uniform), 500 sweeps each: one persistent CUDA-graph launch (launch
    shape from the autotuner) against one ising_sweep call per lattice."""
    import torch
    from paper_cs_0312006_gb300 import _build, autotune, batched, engine, workloads
    _build.build()
    engine.load_library()
    specs = workloads.batched_mix(n=args.batch_lattices, sweeps=args.batch_sweeps)
    if args.no_tune:
        tuned = {"opts": dict(block_threads=256, cluster_size=8, big_sites=65536),
                 "layout": "auto", "results": []}
    else:
        tuned = autotune.tune(specs, use_cache=not args.retune)
    opts, layout = tuned["opts"], tuned["layout"]
    if args.batch_layout:
        layout = args.batch_layout
    batched.run_batched(batched.scaled(specs[:64], 2), opts, 1, layout)  # warm-up
    res = batched.compare_forms(specs, opts, layout)
    line = {"metric": "site updates/s", "value": res["batched_updates_per_s"],
            "unit": "site updates/s", "n_gpus": 1, "higher_is_better": True,
            "workload": f"batched: {res['lattices']} lattices, {args.batch_sweeps} sweeps each, "
                        "70% 2D L log-uniform [16,1024], 30% 3D L log-uniform [8,128], E/M every "
                        "10 sweeps",
            "batched": res, "autotune": {"opts": opts, "layout": layout,
                                         "candidates": len(tuned["results"])},
            "device": torch.cuda.get_device_name()}
    print(json.dumps(line), flush=True)
    if res["mismatches"]:
        raise SystemExit(f"batched and plain forms differ on {res['mismatches']} lattices")
    return 0


def run_serving_workload(args):
    """Poisson job stream (200 jobs/s): dims in {2,3}; L log-uniform (2D
    32-4096, 3D 16-256); beta within 0.05 of the critical point; sweeps
    log-uniform 100-20000; E/M every 10 sweeps; HBM budget 120 GB.  Reports
    aggregate site updates/s and p50/p99 job latency (arrival to completion),
    the first tenth of the jobs excluded from the percentiles."""
    import torch
    from paper_cs_0312006_gb300 import _build, autotune, engine, serve, workloads
    _build.build()
    engine.load_library()
    jobs = workloads.poisson_jobs(args.serve_jobs, rate_per_s=args.serve_rate)
    warm = workloads.poisson_jobs(8, rate_per_s=1e6, seed=99, l2d=(32, 128), l3d=(16, 32),
                                  sweeps=(10, 20))
    serve.Server(round_s=args.round_s).run(warm)  # load and warm the kernels
    srv = serve.Server(hbm_budget_bytes=int(args.hbm_budget_gb * 1e9),
                       round_s=args.round_s, keep_spins=False,
                       batch_opts=dict(cluster_size=8, big_sites=65536))
    summ = srv.run(jobs)
    skip = max(0, len(jobs) // 10)
    pct = serve.percentile_summary(srv.results, skip)
    plain = None
    if not args.no_plain:
        psum, pres = serve.run_plain_fifo(jobs)
        plain = dict(psum, **serve.percentile_summary(pres, skip))
    line = {"metric": "site updates/s", "value": summ["updates_per_s"],
            "unit": "site updates/s", "n_gpus": 1, "higher_is_better": True,
            "workload": f"serving: {len(jobs)} Poisson jobs at {args.serve_rate}/s, dims 2/3, "
                        "L log-uniform (2D 32-4096, 3D 16-256), beta_c +- 0.05, sweeps "
                        "log-uniform 100-20000, E/M every 10, HBM budget "
                        f"{args.hbm_budget_gb} GB",
            "serving": dict(summ, **pct), "plain_fifo": plain,
            "offered_load_updates_per_s": serve.offered_load(jobs, args.serve_rate),
            "device": torch.cuda.get_device_name()}
    print(json.dumps(line), flush=True)
    return 0


def run_small_workload(args):
    """The small critical run (small_form): 2D L=64 at beta_c, hot start, seed
    20031109, 1000 sweeps with E/M every sweep, both layouts."""
    import torch
    from paper_cs_0312006_gb300 import _build, engine
    _build.build()
    engine.load_library()
    form = small_form(args)
    line = {"metric": "site updates/s", "value": form["value"], "unit": "site updates/s",
            "workload": form["config"]["workload"], "us_per_sweep": form["us_per_sweep"],
            "layouts_bit_identical": form["layouts_bit_identical"], "layouts": form["layouts"],
            "device": torch.cuda.get_device_name()}
    print(json.dumps(line), flush=True)
    return 0 if form["layouts_bit_identical"] else 1

def run_cubic_workload(args):
    """3D cubic L=256 (16.8 M sites) at beta 0.2216544, hot start, seed
    20031109, 1000 sweeps with E/M every 10 sweeps, in both layouts."""
    import torch
    from paper_cs_0312006_gb300 import _build, engine
    _build.build()
    engine.load_library()
    from paper_cs_0312006_gb300 import autotune
    L, beta, n = args.cubic_L, 0.2216544, args.cubic_sweeps
    sites = L ** 3
    # the int8 pass configuration tuned for this shape, as in the default line
    tuned = autotune.tune_int8(3, L, use_cache=not args.retune)
    out = {}
    for name, lay in (("int8", engine.INT8), ("bitpack", engine.BITPACK)):
        lat = engine.Lattice(3, L, beta, BASE_SEED, layout=lay)
        if name == "int8":
            out_cfg = lat.int8_config()
        lat.sweep(3, 10)  # warm-up
        torch.cuda.synchronize()
        lat.init(engine.HOT)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        lat.sweep(n, 10)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        E, M = lat.observables()
        lat.close()
        out[name] = {"value": sites * n / (ms / 1e3), "ms": ms, "records": len(E),
                     "us_per_sweep": ms * 1e3 / n}
    total = 2 * sites * n / ((out["int8"]["ms"] + out["bitpack"]["ms"]) / 1e3)
    line = {"metric": "site updates/s", "value": total, "unit": "site updates/s",
            "workload": f"3D cubic L={L}, beta 0.2216544, hot start, {n} sweeps, E/M every 10 "
                        "sweeps, int8 and bit-packed layouts",
            "layouts": out, "int8_config": out_cfg, "int8_tuned": tuned,
            "device": torch.cuda.get_device_name()}
    print(json.dumps(line), flush=True)
    return 0


def run_percolation_workload(args):
    """Site percolation (Sec. 2.3), two forms:
    medium -- one 2D medium L = 16384 (268 M sites) at porosity 0.6 (above the
              threshold, so the cluster is deep): porosity field, then face
              invasion by synchronous growth passes to the steady state;
    batch  -- 8192 media of 2D L = 128 at the paper's threshold 0.592746, one
              CTA per medium (spanning fraction reported);
    scan   -- spanning fractions over seven porosities around the threshold
              for L = 64, 128, 256, 512 and the fitted porosity where half
              the media span.
    The oracle runs on bounded samples of both as the CPU baseline."""
    import torch
    from paper_cs_0312006_gb300 import _build, percolation
    _build.build()
    L, P = args.perc_L, 0.6
    sites = L * L
    m = percolation.Medium(2, L, BASE_SEED)
    m.generate(P)  # warm-up
    m.invade(percolation.FACE)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    m.generate(P)
    b.record()
    torch.cuda.synchronize()
    gen_ms = a.elapsed_time(b)
    t0 = time.perf_counter()
    r = m.invade(percolation.FACE)
    inv_s = time.perf_counter() - t0
    m.close()
    words = L * ((L + 31) // 32)
    medium = {"L": L, "porosity": P, "generate_ms": gen_ms,
              "generate_sites_per_s": sites / (gen_ms / 1e3),
              "invade_s": inv_s, "steps": r.steps, "cluster_sites": r.size,
              "spans": bool(r.spans),
              "us_per_pass": inv_s * 1e6 / max(1, r.steps),
              "site_passes_per_s": sites * r.steps / inv_s,
              "pass_bytes": 5 * 4 * words,
              "note": "a growth pass reads the pore, cluster and last-front bitmaps (with "
                      "halo words from L2) and writes the next front (and the cluster where "
                      "it grew): ~5 x 4 B per 32-site word"}
    # batch of small media
    Lb, Pb, n = 128, 0.592746, args.perc_media
    seeds = [BASE_SEED + k for k in range(n)]
    percolation.batch(2, Lb, Pb, seeds[:256])  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = percolation.batch(2, Lb, Pb, seeds)
    bt = time.perf_counter() - t0
    frac = sum(x.spans for x in res) / n
    batch = {"L": Lb, "porosity": Pb, "media": n, "seconds": bt, "media_per_s": n / bt,
             "sites_per_s": n * Lb * Lb / bt, "spanning_fraction": frac,
             "mean_steps": sum(x.steps for x in res) / n}
    # spanning probability against porosity for growing L: where half the media
    # span approaches the threshold (0.592746 in Sec. 5) as L grows; the
    # porosities are spread over the transition, whose width falls as L^(-3/4)
    scan = []
    pc = 0.592746
    for k_L, Ls in enumerate((64, 128, 256, 512)):
        width = 0.012 * (Ls / 128) ** -0.75
        Ps = [pc + width * x for x in (-2.0, -1.0, -0.5, 0.0, 0.5, 1.0, 2.0)]
        ns = args.perc_scan_media
        t0 = time.perf_counter()
        fr = []
        for j, Pj in enumerate(Ps):
            sd_seeds = [BASE_SEED + 10_000_000 * (k_L + 1) + 100_000 * j + q for q in range(ns)]
            fr.append(sum(x.spans for x in percolation.batch(2, Ls, Pj, sd_seeds)) / ns)
        st = time.perf_counter() - t0
        p_half, p_sd = percolation.spanning_threshold(Ps, fr, ns)
        scan.append({"L": Ls, "media_per_porosity": ns, "porosities": Ps,
                     "spanning_fraction": fr, "p_half": p_half, "p_half_sd": p_sd,
                     "seconds": st})
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < args.cpu_seconds / 2 and k < n:
            oracle.perc_invade(2, Lb, oracle.perc_pores(2, Lb, seeds[k], Pb))
            k += 1
        ct = time.perf_counter() - t0
        cpu = {"value": k / ct, "unit": "media/s", "cores": 1, "kind": "oracle",
               "sample": f"{k} media of 2D L={Lb} at P={Pb} (porosity field + face invasion)",
               "host": host_description()}
    line = {"metric": "media/s", "value": batch["media_per_s"], "unit": "media/s",
            "workload": "site percolation, 2D: one L=16384 medium at P=0.6 (porosity field "
                        "+ face invasion to the steady state) and a batch of L=128 media at "
                        "P=0.592746",
            "medium": medium, "batch": batch, "threshold_scan": scan, "cpu_baseline": cpu,
            "device": torch.cuda.get_device_name()}
    print(json.dumps(line), flush=True)
    return 0


def measure_philox_ceiling(engine, torch, reps: int = 5) -> dict:
    """Calls/s of the device Philox4x32-10 alone (ising_philox_probe): every
    resident thread folds 8192 calls into one register and stores one word,
    so the launch measures the generator's integer arithmetic only.  Both
    multiply forms, 4 and 8 independent calls in flight per thread."""
    sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    threads, blocks = 256, sm * 8
    out = torch.empty(blocks * threads, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    for variant in (0, 1):
        for chains in (4, 8):
            iters = 8192 // chains
            calls = blocks * threads * iters * chains
            for _ in range(2):
                engine.philox_probe(out.data_ptr(), blocks, threads, iters, variant, chains,
                                    BASE_SEED, stream)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                engine.philox_probe(out.data_ptr(), blocks, threads, iters, variant, chains,
                                    BASE_SEED, stream)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b) / reps
            res[f"{'wide' if variant == 0 else 'split'}_x{chains}"] = {
                "calls_per_s": calls / (ms / 1e3), "ms_per_launch": ms, "calls": calls}
    best = max(res.values(), key=lambda r: r["calls_per_s"])
    engine_form = max(res["wide_x4"]["calls_per_s"], res["wide_x8"]["calls_per_s"])
    return {"forms": res, "best_calls_per_s": best["calls_per_s"],
            "engine_form_calls_per_s": engine_form,
            "draws_per_s": 4 * engine_form, "sm_count": sm,
            "how": f"{blocks} CTAs x {threads} threads, 8192 calls folded per thread, "
                   f"CUDA events over {reps} launches"}


def run_philox_workload(args):
    """Throughput of the device generator alone: the integer ceiling that the
    Metropolis draws put on any pass kernel (one 32-bit draw per site with
    dE > 0; a quarter of a call per site)."""
    import torch
    from paper_cs_0312006_gb300 import _build, engine
    _build.build()
    engine.load_library()
    res = measure_philox_ceiling(engine, torch, reps=args.probe_reps)
    line = {"metric": "Philox4x32-10 calls/s", "value": res["engine_form_calls_per_s"],
            "unit": "calls/s", "probe": res, "device": torch.cuda.get_device_name()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["engine", "reference"], default="engine")
    ap.add_argument("--L", type=int, default=L_SCAN)
    ap.add_argument("--layout", choices=["both", "int8", "bitpack"], default="both")
    ap.add_argument("--rule", choices=["metropolis", "heatbath", "demon"], default="metropolis",
                    help="local update rule of the scan workload")
    ap.add_argument("--int8-kernel", choices=["auto", "strip", "tma"], default="auto",
                    help="int8 pass: register-window strips or shared-memory tiles staged by "
                         "bulk (TMA) copies")
    ap.add_argument("--workload", choices=["scan", "batched", "serving", "philox", "small",
                                           "cubic", "big", "percolation"],
                    default="scan",
                    help="scan: the 2D L=8192 beta scan (default line); batched: 2048 "
                         "lattices in one launch vs one launch per lattice; serving: Poisson "
                         "job stream; philox: the device generator alone; small: 2D L=64, "
                         "1000 sweeps; cubic: 3D L=256; big: one 2D lattice of --big-L "
                         "(default 65536, out of L2); percolation: an L=16384 medium and a "
                         "batch of L=128 media")
    ap.add_argument("--batch-lattices", type=int, default=2048)
    ap.add_argument("--batch-sweeps", type=int, default=500)
    ap.add_argument("--batch-layout", choices=["auto", "int8", "bitpack", "mixed"], default=None,
                    help="batched: override the tuned layout policy")
    ap.add_argument("--retune", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="batched: fixed launch shape")
    ap.add_argument("--big-L", type=int, default=65536,
                    help="big: linear size of the single 2D lattice")
    ap.add_argument("--perc-L", type=int, default=16384)
    ap.add_argument("--perc-media", type=int, default=8192)
    ap.add_argument("--perc-scan-media", type=int, default=8192,
                    help="media per porosity in the percolation threshold scan")
    ap.add_argument("--cubic-L", type=int, default=256)
    ap.add_argument("--cubic-sweeps", type=int, default=1000)
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--hbm-budget-gb", type=float, default=120.0)
    ap.add_argument("--round-s", type=float, default=0.05)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--lattices", type=int, default=N_BETA,
                    help="how many of the 16 betas to run (profiling uses fewer)")
    ap.add_argument("--time-every", type=int, default=20,
                    help="bracket every k-th step with events (an event between two passes "
                         "keeps the second from being scheduled early, so only step "
                         "boundaries carry them)")
    ap.add_argument("--probe-reps", type=int, default=5,
                    help="philox: timed launches of each probe form")
    ap.add_argument("--e2e-steps", type=int, default=0)
    ap.add_argument("--e2e-order", choices=["step", "wave"], default="wave",
                    help="e2e issue order: every lattice's sweep k before any sweep k + 1 "
                         "(step), or lattice j's sweep k in wavefront k + j (wave)")
    ap.add_argument("--e2e-copy-streams", type=int, default=1,
                    help="e2e copy mode: streams the lattices' copies are spread over")
    ap.add_argument("--e2e-mode", choices=["copy", "direct"], default="copy",
                    help="e2e host buffers: copy-engine copies on a second stream (copy) or "
                         "the import/export kernels reading and writing pinned host memory "
                         "(direct)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="leave the batched and serving forms out of the default line")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "engine":
        raise SystemExit("bench.py: at least 3 warm-up steps are required")
    world, rank, local = dist_setup()
    if args.workload == "batched" and args.impl != "reference":
        return run_batched_workload(args)
    if args.workload == "serving" and args.impl != "reference":
        return run_serving_workload(args)
    if args.workload == "philox" and args.impl != "reference":
        return run_philox_workload(args)
    if args.workload == "small" and args.impl != "reference":
        return run_small_workload(args)
    if args.workload == "cubic" and args.impl != "reference":
        return run_cubic_workload(args)
    if args.workload == "percolation" and args.impl != "reference":
        return run_percolation_workload(args)
    if args.workload == "big":  # one lattice far larger than L2
        args.L = args.big_L
        args.lattices = 1
        if args.impl == "engine":
            args.no_e2e = True  # the scan's e2e leg sizes host buffers per lattice set
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_gpu(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
