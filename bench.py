#!/usr/bin/env python
"""Benchmark: Swendsen-Wang sweeps of the pyrochlore Ising model on GB300.

One step = one full Swendsen-Wang sweep (bond activation, tile-local and
global labelling, cluster flips, E / m^2 / m^4 measurement and accumulation).
Default workload: the L = 256 Ising lattice (N = 16 * 256^3 = 268,435,456
sites) at T = 4.21394 from a Philox-random start, the workload the headline
metric is quoted on.  --workload selects the other runs (L = 8 Ising, 48
batched Ising replicas, XY L = 64 in FP32 with the plain FP64 form beside it,
24 batched Heisenberg replicas likewise, one Heisenberg L = 128 lattice) and
the generic-lattice path (the simple-cubic Ising lattice at L = 640 with
implicit bonds, at L = 512 as an explicit bond list, and at L = 512 with 80 %
of its sites occupied).  The metric is site updates per nanosecond
(sites * steps / time).

Multi-GPU: independent replicas, one lattice per rank with its own seed (the
sweep of one lattice does not shard), so scaling is weak and there is no
collective on the data path; ranks meet only at the timing barriers.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "SW site-updates/ns on 1 GB300 (% HBM roofline); batched+FP32 vs plain"
UNIT = "site-updates/ns"
FALLBACK_HBM_GBS = 6800.0
# Algorithmic bytes per site update of one sweep: one int32 label written
# and read, the spins read and written (Ising bit-packed: 1/8 byte each way;
# n-vector: n components of 4 or 8 bytes each way).
SWEEP_BYTES = {1: {0: 8.25, 1: 8.25}, 2: {0: 24.0, 1: 40.0}, 3: {0: 32.0, 1: 56.0}}
SWEEP_BYTES_PER_SITE = SWEEP_BYTES[1][1]
# The Ising sweep's 8.25 bytes split over its kernels: the local kernel
# reads the spins and writes the labels, the flip kernel reads the labels
# and writes the spins; the crossing unions, measurement and accumulation
# move nothing the model counts.
PHASE_BYTES_PER_SITE = {"local": 0.125 + 4.0, "boundary": 0.0, "flip": 4.0 + 0.125, "measure": 0.0,
                        "accumulate": 0.0}
KERNEL_NAMES = {"local": "ising_local_kernel", "boundary": "boundary_kernel", "flip": "ising_flip_kernel",
                "measure": "ising_measure_kernel", "accumulate": "accumulate_kernel"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for key in ("hbm_gbs", "hbm_GBps", "hbm"):
                if key in d:
                    return float(d[key]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


# The sources the Ising sweep's kernels are compiled from.
ISING_KERNEL_SOURCES = ("ccl.cuh", "ising.cu", "pyro_internal.cuh", "sweep_core.cuh")


def kernel_source_hash() -> str:
    """Fingerprint of the Ising kernels' source code: comments and
    whitespace are dropped, so an edit to a comment (or to another model's
    kernels) does not retire a traffic capture."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1612_08312_gb300", "csrc")
    for f in ISING_KERNEL_SOURCES:
        text = open(os.path.join(csrc, f), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(f.encode() + b"\0" + " ".join(text.split()).encode())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str, nsites: int):
    """DRAM bytes per launch of `kernel` on an nsites lattice, from the
    committed ncu summary (bytes per site of the captured case), if it was
    taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel and parts[2] == src:
            return float(parts[1]) * nsites
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(wl: dict, args, seconds: float = 12.0, max_sweeps: int = 400):
    """Time the oracle (single-threaded C) on a bounded sample of the
    workload: one L = 32 lattice of the workload's model and temperature
    (L = 8 for the L = 8 workload) from the random start."""
    import oracle
    L = 8 if args.workload == "ising_L8" else 32
    T = wl["T"]
    if "lattice" in wl:
        L = 80  # simple cubic: 512,000 sites, about the pyrochlore L = 32 sample's count
        o = graph_oracle(wl, L, 1)
    else:
        o = oracle.Oracle(L, wl["model"], 1, "random")
    o.sweep(1.0 / T, 1)
    n, t0 = 0, time.perf_counter()
    while n < max_sweeps and time.perf_counter() - t0 < seconds:
        o.sweep(1.0 / T, 1)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": o.N * n / (dt * 1e9), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle, model {wl['model']} {'simple cubic' if 'lattice' in wl else 'pyrochlore'} L={L} "
                      f"(N={o.N}) at T={T}, random start, {n} timed sweeps "
                      f"after 1 untimed ({dt:.1f} s, single thread)"}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_seed(base: int, rank: int) -> int:
    """Seed of the independent replica a rank runs (ranks never share a chain)."""
    return (base + rank * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF


def reduce_max(value: float, world: int, device=None) -> float:
    """Max over ranks of a per-rank time (the job ends when the slowest rank does)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, world, rank):
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    model, T, L = wl["model"], wl["T"], args.ref_L
    import oracle
    if "lattice" in wl:
        L = max(L, 80)
        o = graph_oracle(wl, L, 1)
    else:
        o = oracle.Oracle(L, model, 1, "random")
    for _ in range(args.warmup):
        o.sweep(1.0 / T, 1)
    t0 = time.perf_counter()
    o.sweep(1.0 / T, args.steps)
    dt = time.perf_counter() - t0
    value = o.N * args.steps / (dt * 1e9)
    sample = (f"oracle, model {model} L={L} (N={o.N}) at T={T}, random start; each step one sweep of this "
              f"bounded sample of the {args.workload} workload; single thread")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(args.steps, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": wl["dtype_ref"],
           "data": "synthetic", "config": {"workload": args.workload, "sample_L": L, "T": T},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# Workloads (sizes, temperatures and starts of the paper's kind of run;
# see workloads/__init__.py).  Batched replicas use seed + r * golden.
WORKLOADS = {
    "ising_L256": dict(model=1, L=256, T=4.21394, start="random", seed=1, precision=1, dtype="u8", dtype_ref="i8"),
    "ising_L8": dict(model=1, L=8, T=4.21394, start="up", seed=1, precision=1, dtype="u8", dtype_ref="i8"),
    "ising_batch48": dict(model=1, Ls=workloads.ISING_BATCH["L"], Ts=workloads.ISING_BATCH["T"], T=4.21394,
                          start="random", seed=1, precision=1, dtype="u8", dtype_ref="i8"),
    "xy_L64": dict(model=2, L=64, T=2.0285, start="random", seed=1, precision=0, dtype="f32", dtype_ref="f64"),
    "heis_L128": dict(model=3, L=128, T=1.31695, start="random", seed=1, precision=0, dtype="f32", dtype_ref="f64"),
    "heis_batch24": dict(model=3, Ls=workloads.HEIS_BATCH["L"], Ts=workloads.HEIS_BATCH["T"], T=1.31695,
                         start="random", seed=1, precision=0, dtype="f32", dtype_ref="f64"),
    # generic-lattice path (simple cubic, implicit bonds / explicit bond list / site-diluted)
    "sc_L640": dict(model=1, lattice="sc", L=workloads.SC_L640["L"], T=workloads.SC_L640["T"], start="random",
                    seed=1, precision=1, dtype="i8", dtype_ref="i8"),
    "sc_dil_L512": dict(model=1, lattice="sc", L=workloads.SC_DIL_L512["L"], T=workloads.SC_DIL_L512["T"],
                        p_site=workloads.SC_DIL_L512["p_site"], mask_seed=workloads.SC_DIL_L512["mask_seed"],
                        start="random", seed=1, precision=1, dtype="i8", dtype_ref="i8"),
    "sc_list_L512": dict(model=1, lattice="list", L=workloads.SC_LIST_L512["L"], T=workloads.SC_LIST_L512["T"],
                         start="random", seed=1, precision=1, dtype="i8", dtype_ref="i8"),
}


def graph_bytes_per_site(wl: dict) -> float:
    """Algorithmic bytes per site update of a generic-lattice Ising sweep:
    the int8 spin read and written (2), the union-find array's identity
    entry written, read once and the canonical label written (12); an
    explicit bond list adds its two int32 endpoints per bond (3 bonds per
    simple-cubic site: 24)."""
    return 14.0 + (24.0 if wl["lattice"] == "list" else 0.0)


def make_graph(pyro, wl: dict, L: int, seed: int):
    """The generic-lattice object of a workload (simple cubic L^3)."""
    kw = dict(sc_L=L)
    if wl["lattice"] == "list":
        bi, bj = workloads.sc_bond_list(L)
        kw = dict(nsites=L ** 3, bond_i=bi, bond_j=bj)
    if "p_site" in wl:
        kw["site_mask"] = workloads.site_mask(L ** 3, wl["p_site"], wl["mask_seed"])
    return pyro.Graph(wl["model"], seed, precision=wl["precision"], start=wl["start"], **kw)


def graph_oracle(wl: dict, L: int, seed: int):
    import oracle
    bi, bj = oracle.sc_edges(L)
    mask = workloads.site_mask(L ** 3, wl["p_site"], wl["mask_seed"]) if "p_site" in wl else None
    return oracle.GraphOracle(L ** 3, bi, bj, wl["model"], seed, wl["start"], site_mask=mask)


def time_device(stream, fn):
    """Device ms of fn() between two CUDA events on the given stream."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=60)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ising_L256", choices=list(WORKLOADS))
    ap.add_argument("--L", type=int, default=0, help="override the lattice size of a single-lattice workload")
    ap.add_argument("--tile", default="auto", help="'auto' (autotuner), 'default', or TXxTYxTZ")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--ref-L", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain FP64 arm of n-vector workloads")
    ap.add_argument("--binder-sweeps", type=int, default=8000,
                    help="sweeps of each form's Binder-ratio trace (200 bins) in the n-vector comparison")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1612_08312_gb300 as pyro

    wl = WORKLOADS[args.workload]
    model, prec = wl["model"], wl["precision"]
    peak, peak_kind = peaks()

    def barrier():
        if world > 1:
            dist.barrier()

    batched = "Ls" in wl
    graph = "lattice" in wl
    if graph:
        L = args.L or wl["L"]
        beta = 1.0 / wl["T"]
        obj = make_graph(pyro, wl, L, rank_seed(wl["seed"], rank))
        N = obj.N
        stream = torch.cuda.ExternalStream(obj.stream)
        sweep = lambda n: obj.sweep(beta, n)
        sync = obj.sync
        tile = None
    elif batched:
        reps = [(L, T) for L in wl["Ls"] for T in wl["Ts"]]
        Ls, betas = [r[0] for r in reps], [1.0 / r[1] for r in reps]
        btile = "auto" if args.tile == "auto" else ((0, 0, 0) if args.tile == "default" else
                                                    tuple(int(v) for v in args.tile.split("x")))
        obj = pyro.Replicas(Ls, betas, model, precision=prec, start=wl["start"], seed=rank_seed(wl["seed"], rank),
                            tile=btile)
        N = obj.total_sites
        stream = torch.cuda.ExternalStream(obj.stream)
        sweep = lambda n: obj.sweep(n)
        sync = obj.sync
        tile = list(obj.tile)
    else:
        L = args.L or wl["L"]
        beta = 1.0 / wl["T"]
        if args.tile == "auto":
            tile = pyro.pyro_autotune(L, model, prec, beta, 3)[0]
        elif args.tile == "default":
            tile = (0, 0, 0)
        else:
            tile = tuple(int(v) for v in args.tile.split("x"))
        obj = pyro.Lattice(L, model, rank_seed(wl["seed"], rank), precision=prec, start=wl["start"], tile=tile)
        N = obj.N
        stream = torch.cuda.ExternalStream(pyro.pyro_get_stream(obj.h))
        sweep = lambda n: obj.sweep(beta, n)
        sync = obj.sync
        tile = list(obj.tile)

    sweep(max(args.warmup, 3))
    sync()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    sync()
    l0 = obj.launches
    ms = time_device(stream, lambda: sweep(args.steps))
    sync()
    launches = obj.launches - l0
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = reduce_max(ms, world, device="cuda")
    value = N * args.steps * world / (ms * 1e6)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": wl["dtype"], "data": "synthetic",
           "config": {"workload": args.workload, "N": N, "model": model, "start": wl["start"],
                      "tile": tile, "parallelism": f"replicas{world}",
                      "l2": "inputs larger than L2" if N * 4 > 129e6 else "working set may fit in L2"},
           "gpu_launches": launches, "clocks": clk}
    if batched:
        out["config"].update({"replicas": len(reps), "L": sorted(set(Ls)), "T": wl["Ts"], "graphs": True})
    elif graph:
        out["config"].update({"L": L, "T": wl["T"], "lattice": "simple cubic", "bonds": obj.NB,
                              "bond_form": "explicit bond list" if wl["lattice"] == "list" else "implicit",
                              "site_occupation": wl.get("p_site", 1.0)})
        del out["config"]["tile"]
    else:
        out["config"].update({"L": L, "T": wl["T"]})

    sweep_bytes = graph_bytes_per_site(wl) if graph else SWEEP_BYTES[model][prec]
    if graph:
        out["roofline"] = {"bound": "hbm", "kernel": "whole sweep", "achieved": value * sweep_bytes, "peak": peak,
                           "unit": "GB/s", "frac": value * sweep_bytes / peak, "peak_kind": peak_kind,
                           "traffic": None, "alg_bytes_per_site": sweep_bytes}
    elif not batched and model == 1:
        prof = pyro.pyro_profile_phases(obj.h, beta, 5)
        dominant = max(prof, key=prof.get)
        alg_bytes = PHASE_BYTES_PER_SITE[dominant] * N
        achieved = alg_bytes / (prof[dominant] * 1e-3) / 1e9
        traffic = committed_traffic(KERNEL_NAMES[dominant], N)
        out["roofline"] = {"bound": "hbm", "kernel": KERNEL_NAMES[dominant], "achieved": achieved, "peak": peak,
                           "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                           "alg_bytes_per_site": PHASE_BYTES_PER_SITE[dominant],
                           "phase_ms": {k: round(v, 5) for k, v in prof.items()}}
    else:
        out["roofline"] = {"bound": "hbm", "kernel": "whole sweep", "achieved": value * SWEEP_BYTES[model][prec],
                           "peak": peak, "unit": "GB/s", "frac": value * SWEEP_BYTES[model][prec] / peak,
                           "peak_kind": peak_kind, "traffic": None,
                           "alg_bytes_per_site": SWEEP_BYTES[model][prec]}
    out["sweep_hbm_frac"] = value * sweep_bytes / peak

    # end to end through the C ABI with host buffers (single lattices): per
    # step the state goes host -> device, one sweep runs, the state and the
    # measurement come back device -> host
    if graph:
        # pinned host buffers (int8 spins in site order)
        host_in = torch.empty(N, dtype=torch.int8, pin_memory=True).numpy()
        host_out = torch.empty(N, dtype=torch.int8, pin_memory=True).numpy()
        obj.spins(out=host_in)
        sync()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            obj.set_spins(host_in)
            sweep(1)
            obj.spins(out=host_out)
            obj.measure()
            host_in, host_out = host_out, host_in
        e2e_s = reduce_max(time.perf_counter() - t0, world, device="cuda")
        out["e2e"] = {"value": N * args.e2e_steps * world / (e2e_s * 1e9), "unit": UNIT,
                      "h2d_bytes_per_step": N, "d2h_bytes_per_step": N + 24, "steps": args.e2e_steps}
    elif not batched:
        nbytes = pyro.pyro_state_bytes(obj.h)
        host_in = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        host_out = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        pyro.pyro_get_state(obj.h, host_in.data_ptr(), nbytes)
        sync()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            pyro.pyro_set_state(obj.h, host_in.data_ptr(), nbytes)
            sweep(1)
            pyro.pyro_get_state(obj.h, host_out.data_ptr(), nbytes)
            obj.measure()  # synchronises; E, m^2, m^4 to the host
            host_in, host_out = host_out, host_in
        e2e_s = reduce_max(time.perf_counter() - t0, world, device="cuda")
        out["e2e"] = {"value": N * args.e2e_steps * world / (e2e_s * 1e9), "unit": UNIT,
                      "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 24, "steps": args.e2e_steps}
    else:
        # a batch's state stays on the device; per step the host reads every
        # replica's measurement (one device-to-host copy)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            obj.sweep(1)
            obj.measure_all()
        e2e_s = reduce_max(time.perf_counter() - t0, world, device="cuda")
        out["e2e"] = {"value": N * args.e2e_steps * world / (e2e_s * 1e9), "unit": UNIT,
                      "h2d_bytes_per_step": 0,
                      # one copy of the replicas' contiguous 152-byte device records
                      "d2h_bytes_per_step": 152 * len(reps), "steps": args.e2e_steps}

    # n-vector workloads: the plain FP64 form (per-replica launches, no
    # graph) on the same sweeps, and the Binder ratio from both chains
    if model != 1 and not args.no_compare and rank == 0:
        out["vs_plain_fp64"] = compare_plain_fp64(pyro, wl, args, obj, batched, value, ms / args.steps)

    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(wl, args)
        print(json.dumps(out))
    obj.close()
    if world > 1:
        dist.destroy_process_group()


def compare_plain_fp64(pyro, wl, args, obj, batched, value_fast, ms_fast):
    """The plain form beside the fast one: FP64 spins, one lattice per
    replica, separate launches (no CUDA graph), the same number of sweeps;
    and the Binder ratio U = <m^4>/<m^2>^2 (Eq. 2) of one replica from
    long per-sweep traces of both forms (200 bins, jackknife errors; the
    smallest lattice of a batch, at its temperature nearest T_c), so
    that the time each form needs to reach the same error on U can be
    compared: sweeps needed scale with the squared error at a fixed sweep
    count, so time-to-equal-error ratio = (plain ms per sweep x plain error^2)
    / (fast ms per sweep x fast error^2).  The fast chain is a single FP32
    lattice with graphs: a replica of a batch runs exactly the chain of a
    single lattice with its seed."""
    import numpy as np
    from paper_1612_08312_gb300.fss import jackknife
    model = wl["model"]
    reps = [(L, T) for L in wl["Ls"] for T in wl["Ts"]] if batched else [(args.L or wl["L"], wl["T"])]
    lats = [pyro.Lattice(L, model, 7 + r, precision=pyro.FP64, start=wl["start"]) for r, (L, T) in enumerate(reps)]
    for lat in lats:
        lat.set_graphs(False)
    n = max(args.steps // 4, 10)
    for lat, (L, T) in zip(lats, reps):
        lat.sweep(1.0 / T, 2)
    for lat in lats:
        lat.sync()
    t0 = time.perf_counter()
    for _ in range(n):
        for lat, (L, T) in zip(lats, reps):
            lat.sweep(1.0 / T, 1)
    for lat in lats:
        lat.sync()
    dt = time.perf_counter() - t0
    for lat in lats:
        lat.close()
    total = sum(16 * L ** 3 for L, _ in reps)
    value_plain = total * n / (dt * 1e9)
    ms_plain = dt * 1e3 / n
    # Binder ratio from both forms at equal sweep counts, on the smallest
    # lattice at the temperature nearest the workload's critical one
    L0, T0 = min(reps, key=lambda lt: (lt[0], abs(lt[1] - wl["T"])))
    eq, nbin, per = 500, 200, args.binder_sweeps // 200
    res = {}
    for name, prec, graphs, seed in (("fp32_graph", pyro.FP32, True, 11), ("fp64_plain", pyro.FP64, False, 13)):
        lat = pyro.Lattice(L0, model, seed, precision=prec, start=wl["start"])
        lat.set_graphs(graphs)
        lat.sweep(1.0 / T0, eq)
        pyro.pyro_set_trace(lat.h, nbin * per)
        lat.sweep(1.0 / T0, nbin * per)
        tr = pyro.pyro_get_trace(lat.h, nbin * per)
        lat.close()
        b2 = tr[:, 1].reshape(nbin, per).mean(1)
        b4 = tr[:, 2].reshape(nbin, per).mean(1)
        U, err, _ = jackknife(lambda a, b: b / (a * a), b2, b4)
        res[name] = {"U": float(U), "U_err": float(err)}
    ef, ep = res["fp32_graph"]["U_err"], res["fp64_plain"]["U_err"]
    return {"value": value_plain, "unit": UNIT, "ratio": value_fast / value_plain, "sweeps": n,
            "ms_per_sweep": ms_plain,
            "form": "FP64 spins, one lattice per replica, one launch per phase (no graph)",
            "binder": {"L": L0, "T": T0, "equilibration": eq, "sweeps": nbin * per, "bins": nbin, **res,
                       "error_ratio_plain_over_fast": ep / ef if ef > 0 else None},
            "time_to_equal_error_ratio": (ms_plain * ep * ep) / (ms_fast * ef * ef) if ef > 0 else None}


if __name__ == "__main__":
    main()
