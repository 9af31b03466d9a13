#!/usr/bin/env python
"""Benchmark: Swendsen-Wang sweeps of the pyrochlore Ising model on GB300.

One step = one full Swendsen-Wang sweep (bond activation, tile-local and
global labelling, cluster flips, E / m^2 / m^4 measurement and accumulation)
of the L = 256 Ising lattice (N = 16 * 256^3 = 268,435,456 sites) at
T = 4.21394, from a Philox-random start -- the workload the headline metric
is quoted on.  The metric is site updates per nanosecond (N * steps / time).

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
# Algorithmic bytes per site of one sweep (bit-packed spins read + written,
# one int32 label written and read): the whole-sweep HBM model.
SWEEP_BYTES_PER_SITE = 8.25
# Bytes per site each phase of the Ising sweep must move in HBM.
PHASE_BYTES_PER_SITE = {
    "local": 0.125 + 2.0 + 0.125,   # spin words read; 16-bit local labels and flip words written
    "boundary": 0.0,                # only tile-crossing pairs; not credited
    "flip": 2.0 + 0.125 + 0.25,     # local labels and flip words read; spin words read and written
    "measure": 0.125,               # spin words read
    "accumulate": 0.0,
}
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


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1612_08312_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel and parts[3] == src:
            return float(parts[1]) * float(parts[2])  # bytes per site * sites of the bench lattice
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


def cpu_baseline(L: int, T: float, seconds: float = 12.0, max_sweeps: int = 40):
    """Time the oracle (single-threaded C) on a bounded sample: an L-lattice
    Ising run at temperature T from the random start."""
    import oracle
    o = oracle.Oracle(L, oracle.ISING, 1, "random")
    o.sweep(1.0 / T, 1)
    n, t0 = 0, time.perf_counter()
    while n < max_sweeps and time.perf_counter() - t0 < seconds:
        o.sweep(1.0 / T, 1)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": o.N * n / (dt * 1e9), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle, Ising L={L} (N={o.N}) at T={T}, random start, {n} timed sweeps after 1 "
                      f"untimed ({dt:.1f} s, single thread)"}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, world, rank):
    if rank != 0:
        return
    cfg = workloads.ISING_L256
    T = cfg["T"][1]
    L = args.ref_L
    import oracle
    o = oracle.Oracle(L, oracle.ISING, 1, "random")
    for _ in range(args.warmup):
        o.sweep(1.0 / T, 1)
    t0 = time.perf_counter()
    o.sweep(1.0 / T, args.steps)
    dt = time.perf_counter() - t0
    value = o.N * args.steps / (dt * 1e9)
    sample = (f"oracle, Ising L={L} (N={o.N}) at T={T}, random start; each step one sweep of this "
              f"bounded sample of the L=256 workload; single thread")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(args.steps, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
           "config": {"workload": "ising_L256", "L": 256, "T": T, "sample_L": L},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=256)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--ref-L", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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

    cfg = workloads.ISING_L256
    T = cfg["T"][1]
    beta = 1.0 / T
    L = args.L
    seed = cfg["seeds"][0] + rank  # one independent replica per rank
    lat = pyro.Lattice(L, pyro.ISING, seed, start="random")
    N = lat.N
    stream = torch.cuda.ExternalStream(pyro.pyro_get_stream(lat.h))

    lat.sweep(beta, max(args.warmup, 3))
    lat.sync()

    def barrier():
        if world > 1:
            dist.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    lat.sync()
    l0 = lat.launches
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.sweep(beta, args.steps)
    e1.record(stream)
    e1.synchronize()
    lat.sync()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    launches = lat.launches - l0
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = N * args.steps * world / (ms * 1e6)

    # per-phase device times (event-bracketed) for the roofline of the dominant kernel
    prof = pyro.pyro_profile_phases(lat.h, beta, 5)
    dominant = max(prof, key=prof.get)
    peak, peak_kind = peaks()
    alg_bytes = PHASE_BYTES_PER_SITE[dominant] * N
    achieved = alg_bytes / (prof[dominant] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": KERNEL_NAMES[dominant], "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                "traffic": committed_traffic(KERNEL_NAMES[dominant]),
                "alg_bytes_per_site": PHASE_BYTES_PER_SITE[dominant],
                "phase_ms": {k: round(v, 5) for k, v in prof.items()}}

    # end to end through the C ABI with host buffers: per step the state
    # goes host -> device, one sweep runs, the state and the measurement come
    # back device -> host
    nbytes = pyro.pyro_state_bytes(lat.h)
    host_in = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    host_out = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    pyro.pyro_get_state(lat.h, host_in.data_ptr(), nbytes)
    lat.sync()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        pyro.pyro_set_state(lat.h, host_in.data_ptr(), nbytes)
        lat.sweep(beta, 1)
        pyro.pyro_get_state(lat.h, host_out.data_ptr(), nbytes)
        lat.measure()  # synchronises; E, m^2, m^4 to the host
        host_in, host_out = host_out, host_in
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": N * args.e2e_steps * world / (e2e_s * 1e9), "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes + 24, "steps": args.e2e_steps}

    out = None
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
               "config": {"workload": "ising_L256", "L": L, "N": N, "T": T, "start": "random",
                          "tile": list(lat.tile), "parallelism": f"replicas{world}",
                          "l2": "inputs larger than L2 (labels 4N bytes)"},
               "sweep_hbm_frac": value * SWEEP_BYTES_PER_SITE / peak,
               "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(64, T)
        print(json.dumps(out))
    lat.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
