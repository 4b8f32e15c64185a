#!/usr/bin/env python
"""Spin-flip attempts per second of the replica-parallel Metropolis sweep with PT.

Workload (one "step" = one pass of the whole hot path over the batch): the
32x32 lattice x 32 Trotter slices model (32768 spins, spatial degree 4-6 plus
the 2 Trotter couplings), 256 replicas at geometric inverse temperatures
0.05..5.0, int8 spins and int16 local fields, 200 sequential Metropolis sweeps
with a parallel-tempering pass after every sweep.  Synthetic seeded inputs
(paper_1004_0024_gb300.workloads).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--rng mt19937|philox]
    python bench.py --impl reference     # the CPU oracle on the host cores
    python bench.py --workload cfg3      # 4096 spins x 65536 replicas, 500 sweeps, no PT
    python bench.py --workload paper     # the paper's 96 x 256-layer x 115-model shape, 30000 sweeps
    python bench.py --workload cfg1-trotter  # cfg1 with temperature-dependent Trotter couplings
    python bench.py --learned-passes 3   # a short learned-proposal case for profilers

The default line also carries `learned`: the ESS/s study of the learned
Trotter-column proposal against the plain sweep on the same system.

Under torchrun each rank samples its own independent instance (different
seed): the path has no data exchange between instances, so N ranks are N
replicas of the workload ("scaling": "weak"); value = all ranks' attempts /
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2
WORKLOAD_NAMES = {
    "cfg1": "32x32 lattice x 32 Trotter slices (32768 spins), 256 replicas, betas 0.05-5.0 geometric, 200 sweeps + PT each",
    "cfg3": "16x16 lattice x 16 Trotter slices (4096 spins), 65536 replicas, betas 0.1-3.0 geometric, 500 sweeps, no PT",
    "paper": "the paper's shape: 256 Trotter layers x 96 spins (8x12 lattice, 24576 spins), 115 models at betas "
             "0.1-3.0 geometric, 30000 sweeps, no PT",
    "cfg1-trotter": "32x32 lattice x 32 Trotter slices (32768 spins), 256 replicas, betas 0.05-5.0 geometric, "
                    "split couplings K_k = (1/2) ln coth(beta_k 2 / 32), 200 sweeps + PT each",
}
# The paper's figures for its own workload shape (30000 sweeps x 115 models x
# 24576 spins), derived from section 4 / Figure 13: other hardware, context only
PAPER_GTX285_ATTEMPTS = 4.3e8   # B.2, coalesced CUDA on a GTX-285
PAPER_I7_ATTEMPTS = 8.8e8       # A.4, SSE assembly, 8 threads on a Core i7-965


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rng", choices=["mt19937", "philox"], default="mt19937")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads of the default line (cfg1 Philox, cfg3, cfg1-trotter, "
                         "the paper's shape, the ragged batch)")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-proposal study (ESS/s against the plain sweep)")
    ap.add_argument("--workload", choices=["cfg1", "cfg3", "batch", "paper", "cfg1-trotter"], default="cfg1",
                    help="cfg1: the headline 32768-spin x 256-replica model; cfg3: 4096 spins x 65536 replicas; "
                         "batch: 4096 ragged instances, 100 sweeps + PT per step in one CUDA graph; "
                         "paper: the paper's 96 x 256-layer x 115-model shape; "
                         "cfg1-trotter: cfg1 with temperature-dependent Trotter couplings (ising_set_trotter)")
    ap.add_argument("--launch-flags", type=int, default=-1,
                    help="ising_set_launch flags for the handle (-1: the library's choice)")
    ap.add_argument("--sweeps", type=int, default=0,
                    help="override the sweeps per step (short cases for profilers; 0 = the workload's)")
    ap.add_argument("--learned-passes", type=int, default=0,
                    help="only run N learned passes on the 32x32x32 system (a short case for profilers)")
    return ap.parse_args()


def workload(name="cfg1"):
    from paper_1004_0024_gb300 import workloads as W
    return {"cfg1": W.config1, "cfg3": W.config3, "paper": W.config_paper,
            "cfg1-trotter": W.config1_trotter}[name]()


def attempts_per_step(c):
    return c["graph"].n * c["R"] * c["sweeps"]


# ------------------------------------------------------- multi-rank helpers
def rank_seed(base, rank):
    """Each rank samples its own instance: the workload with seed base +
    100003 * rank (independent Philox keys / MT19937 streams, no exchange)."""
    return base + 100003 * rank


def max_over_ranks(ms, world):
    """The slowest rank's time (all-reduce MAX over the default process
    group; on the CPU for gloo, on the device for NCCL)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    """Sum of a per-rank number over the default process group."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(items, rank, world):
    """Instance sharding of a batch: rank r of N takes items r, r + N, r + 2N,
    ... (instances are independent: no exchange between ranks)."""
    return list(items)[rank::world]


def whole_job_value(world, per_step, steps, max_ms):
    """All ranks' attempts over the slowest rank's time (weak scaling)."""
    return world * per_step * steps / (max_ms * 1e-3)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (200 ms period)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        smi = shutil.which("nvidia-smi")
        if not smi:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.proc = subprocess.Popen(
            [smi, f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
             "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(float(r[2]) for r in rows),
                "reasons": reasons, "samples": len(rows)}


def clocks_rejected(clocks):
    """A timed region is re-measured once when its clock samples show a
    hardware or thermal slowdown, or an SM clock well below its maximum with
    no reason active (a clock left locked); sw_power_cap alone is kept."""
    if not clocks:
        return False
    if {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"} & set(clocks.get("reasons", [])):
        return True
    return not clocks.get("reasons") and clocks["sm_mhz"] < 0.8 * clocks["sm_max_mhz"]


def any_rank(flag, world):
    """True on every rank when the flag is set on any rank (so that all ranks
    take the same number of timed passes)."""
    return sum_over_ranks(1.0 if flag else 0.0, world) > 0


# ------------------------------------------------------------- our path
def time_steps(sim, sweeps, swap_every, steps, flush, stream, dev_index, world):
    """Time `steps` runs of ising_run(sweeps, swap_every) on the handle's
    stream: CUDA events around each step, an L2 flush between steps (outside
    the events), clocks sampled during the timed region, one re-measure when
    the clocks show a slowdown or a locked clock.  Warm-up is the caller's."""
    import torch
    import torch.distributed as dist

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sim.set_profiling(True)
    timed_passes, first_clocks = 0, None
    while True:
        st0 = sim.stats()
        sampler = ClockSampler(dev_index)
        sampler.start()
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for k in range(steps):
            flush.fill_(k & 0xFF)  # L2 flush between timed steps (outside the events)
            ev[k][0].record(stream)
            sim.run(sweeps, swap_every)
            ev[k][1].record(stream)
        barrier()
        clocks = sampler.stop()
        timed_passes += 1
        if timed_passes == 1 and any_rank(clocks_rejected(clocks), world):
            first_clocks = clocks  # throttled or clock-locked: measure once more
            continue
        break
    st1 = sim.stats()
    sim.set_profiling(False)
    return {"step_ms": [a.elapsed_time(b) for a, b in ev], "clocks": clocks, "first_clocks": first_clocks,
            "timed_passes": timed_passes, "kernel_ms": st1["kernel_ms"] - st0["kernel_ms"],
            "sweep_launches": st1["timed_launches"] - st0["timed_launches"],
            "launches": st1["launches"] - st0["launches"]}


def workload_line(name, rng, steps, warmup, flush, stream, dev_index, sweeps=0):
    """One extra workload of the default line (a single GPU): its own handle,
    warm-up, timed steps, clocks and roofline."""
    from paper_1004_0024_gb300 import ising
    c = workload(name)
    if sweeps > 0:
        c = dict(c, sweeps=sweeps)
    sim = ising.Ising(c["graph"], c["betas"], seed=c["seed"], rng=rng, field_bits=c["field_bits"],
                      stream=stream.cuda_stream)
    if "K" in c:
        sim.set_trotter(c["K"])
    info = sim.info()
    t_w = time.perf_counter()
    for _ in range(warmup):
        sim.run(c["sweeps"], c["swap_every"])
    import torch
    torch.cuda.synchronize()
    warm_s = time.perf_counter() - t_w
    t = time_steps(sim, c["sweeps"], c["swap_every"], steps, flush, stream, dev_index, 1)
    sim.close()
    per_step = attempts_per_step(c)
    total_ms = sum(t["step_ms"])
    out = {"workload": WORKLOAD_NAMES[name], "rng": rng, "field_bits": c["field_bits"],
           "value": per_step * steps / (total_ms * 1e-3), "unit": "attempts/s",
           "ms_per_step": total_ms / steps, "steps": steps, "warmup": warmup, "warmup_seconds": warm_s,
           "sweeps_per_step": c["sweeps"], "attempts_per_step": per_step, "clocks": t["clocks"],
           "gpu_launches": int(t["launches"]),
           "kernel_variant": info["fast_kernel"], "levels": info["levels"],
           "roofline": roofline(c, rng, per_step * steps, t["kernel_ms"], t["sweep_launches"], t["clocks"],
                                info["fast_kernel"], name)}
    if out["roofline"] and t["sweep_launches"] > 0:
        out["roofline"]["latency_floor"] = latency_floor(
            info["levels"], c["sweeps"] * steps / t["sweep_launches"], t["kernel_ms"] / t["sweep_launches"],
            t["clocks"], info.get("persistent_ok", 1))
    if t["first_clocks"] is not None:
        out["remeasured"] = {"first_clocks": t["first_clocks"]}
    return out


# the extra workloads of the default line: (key, workload, rng, steps,
# warm-up steps, sweeps per step override)
EXTRA_WORKLOADS = [
    ("cfg1_philox", "cfg1", "philox", 5, 3, 0),
    ("cfg3_mt19937", "cfg3", "mt19937", 2, 3, 0),
    ("cfg3_philox", "cfg3", "philox", 2, 3, 0),
    ("cfg1_trotter", "cfg1-trotter", "mt19937", 5, 3, 0),
    ("paper_shape_3000_sweeps", "paper", "mt19937", 2, 3, 3000),
]


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1004_0024_gb300 import ising

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev_index = torch.cuda.current_device()
    stream = torch.cuda.current_stream()

    c = workload(args.workload)
    if args.sweeps > 0:
        c = dict(c, sweeps=args.sweeps)
    g = c["graph"]
    seed = rank_seed(c["seed"], rank)
    per_step = attempts_per_step(c)
    sweeps, swap_every = c["sweeps"], c["swap_every"]

    sim = ising.Ising(g, c["betas"], seed=seed, rng=args.rng, field_bits=c["field_bits"],
                      stream=stream.cuda_stream)
    if args.launch_flags >= 0:
        sim.set_launch(0, 0, args.launch_flags)
    if "K" in c:
        sim.set_trotter(c["K"])
    info = sim.info()
    for _ in range(args.warmup):
        sim.run(sweeps, swap_every)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    t = time_steps(sim, sweeps, swap_every, args.steps, flush, stream, dev_index, world)
    clocks, first_clocks, timed_passes = t["clocks"], t["first_clocks"], t["timed_passes"]
    step_ms = t["step_ms"]
    total_ms = sum(step_ms)
    kernel_ms, sweep_launches, launches = t["kernel_ms"], t["sweep_launches"], t["launches"]
    max_ms = max_over_ranks(total_ms, world)
    value = whole_job_value(world, per_step, args.steps, max_ms)

    e2e = None
    if not args.no_e2e and args.workload == "cfg1":
        e2e = run_e2e(args, c, seed, stream, world)

    # parity spot check of the state after the timed run (invariants at full size)
    st = sim.read_state()
    sim.close()
    assert int(st["sweeps"]) == sweeps * (args.warmup + timed_passes * args.steps)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    line = {
        "metric": "spin-flip attempts/sec vs roofline; ESS/sec learned proposal vs plain sweep",
        "value": value,
        "unit": "attempts/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": max_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int8 spins/int16 fields/uint32 RNG",
        "data": "synthetic (seeded layered lattice + matchings)",
        "config": {
            "workload": WORKLOAD_NAMES[args.workload],
            "rng": args.rng, "field_bits": c["field_bits"], "sweeps_per_step": sweeps,
            "attempts_per_step": per_step, "l2": "flushed (512 MB write) between timed steps",
            "parallelism": f"replicas-only x{world}",
            "launch": {k: info[k] for k in ("replicas_per_block", "threads_per_block", "blocks",
                                             "smem_bytes", "persistent_ok", "fast_kernel", "levels")},
        },
        "clocks": clocks,
        "gpu_launches": int(launches),
    }
    if first_clocks is not None:
        line["remeasured"] = {"first_clocks": first_clocks, "why": "slowdown or locked clock in the first timed pass"}
    line["roofline"] = roofline(c, args.rng, per_step * args.steps, kernel_ms, sweep_launches, clocks,
                                info["fast_kernel"], args.workload)
    if line["roofline"] and sweep_launches > 0:
        line["roofline"]["latency_floor"] = latency_floor(
            info["levels"], sweeps * args.steps / sweep_launches, kernel_ms / sweep_launches, clocks,
            info.get("persistent_ok", 1))
    if e2e is not None:
        line["e2e"] = e2e
    if args.workload == "paper" and c["sweeps"] == 30000:
        line["vs_baseline"] = value / PAPER_GTX285_ATTEMPTS
        line["paper_context"] = {"gtx285_b2_attempts_per_s": PAPER_GTX285_ATTEMPTS,
                                 "i7_965_8threads_a4_attempts_per_s": PAPER_I7_ATTEMPTS,
                                 "vs_i7": value / PAPER_I7_ATTEMPTS,
                                 "basis": "derived from the paper's section 4 and Figure 13 (other hardware)"}
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(c, args.rng, args.cpu_seconds)
    if world == 1 and not args.no_extra and args.workload == "cfg1" and args.sweeps == 0:
        # the other workloads, each with its own handle, clocks and roofline
        extra = {}
        for key, name, rng, steps, warm, sw in EXTRA_WORKLOADS:
            extra[key] = workload_line(name, rng, steps, warm, flush, stream, dev_index, sw)
        extra["batch"] = measure_batch(2, 3, 100, 1, 0)
        line["workloads"] = extra
    if world == 1 and not args.no_learned and args.workload == "cfg1":
        line["learned"] = learned_study()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_e2e(args, c, seed, stream, world):
    """End to end through the C ABI: pinned host inputs -> ising_create +
    ising_replicas_init (H2D inside the timed region) -> ising_run ->
    ising_read_state into pinned host buffers (D2H), per step."""
    import numpy as np
    import torch

    from paper_1004_0024_gb300 import ising

    g = c["graph"]
    R, n = c["R"], g.n

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t, t.numpy()

    keep = [pinned(x) for x in (g.row_ptr, g.col, g.J, g.h, c["betas"])]
    rp, col, J, h, betas = [k[1] for k in keep]
    out_s = torch.empty((R, n), dtype=torch.int8).pin_memory()
    out_f = torch.empty((R, n), dtype=torch.int32).pin_memory()
    out_e = torch.empty(R, dtype=torch.int64).pin_memory()
    out_t = torch.empty(R, dtype=torch.int32).pin_memory()
    out_c = torch.empty(2, dtype=torch.int64).pin_memory()
    h2d = rp.nbytes + col.nbytes + J.nbytes + h.nbytes + betas.nbytes
    d2h = out_s.numel() + 4 * out_f.numel() + 8 * R + 4 * R + 16
    import ctypes
    lib = ising._lib
    P = lambda a, t: ctypes.cast(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data, t)

    def one_step():
        hd = ising.ising_create(n, rp, col, J, h, g.n_slices)
        ising.ising_set_stream(hd, stream.cuda_stream)
        ising.ising_replicas_init(hd, R, betas, seed, args.rng, c["field_bits"])
        ising.ising_run(hd, c["sweeps"], c["swap_every"])
        ising._check(lib.ising_read_state(hd, P(out_s, ising._i8p), P(out_f, ising._i32p),
                                          P(out_e, ising._i64p), P(out_t, ising._i32p),
                                          P(out_c, ising._u64p)))
        ising.ising_destroy(hd)

    ising.ising_release_cached_memory()
    torch.cuda.synchronize()
    t_first = time.perf_counter()
    one_step()  # warm: allocations and host tables from scratch (reported, not counted)
    torch.cuda.synchronize()
    first_ms = 1e3 * (time.perf_counter() - t_first)
    steps = max(2, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one_step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    val = world * attempts_per_step(c) * steps / dt
    return {"value": val, "unit": "attempts/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps, "ms_per_step": 1e3 * dt / steps,
            "first_step_ms": first_ms,
            "host_caches": "a fresh handle per step; the MT19937 word buffers and the swap-threshold "
                           "tables of the previous step's handle (same model and ladder) are reused; "
                           "first_step_ms is a step with both caches empty; the packed kernel's word "
                           "placement (searched once per model, 0.24 s) is cached by the library across "
                           "handles and was filled by the device-timed leg"}


# ------------------------------------------------------------- roofline
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")


def avg_degree(g):
    return float(g.row_ptr[-1]) / g.n


def ops_per_attempt(g, rng):
    """Algorithmic integer operations of one attempt: the random word (MT19937
    recurrence + tempering ~17, Philox4x32-10 80 per 4 words = 20), the
    acceptance test (~6: field read, Trotter part, product, threshold read,
    two compares) and the flip's masked neighbour updates (3 per neighbour:
    address, product, add) on the average degree."""
    rng_ops = 17 if rng == "mt19937" else 20
    return rng_ops + 6 + 3 * avg_degree(g)


def int_peak_tops(clocks):
    """Integer issue peak: 152 SMs x 4 sub-partitions x 32 lanes x SM clock
    (one 32-bit integer op per lane per clock).  Uses the median SM clock
    sampled during the run, else the maximum clock."""
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    return 152 * 4 * 32 * mhz * 1e6 / 1e12, mhz


# ncu (1 pass: dram__bytes_read.sum + dram__bytes_write.sum) of the packed
# kernel with MT19937 on the 32x32x32 x 256-replica workload: 234.3 MB for a
# 10-sweep launch, 3311.4 MB for the 200-sweep launch the bench times; linear
# in the sweeps: the state once per launch and the write-back of the
# generator's word buffer per sweep
PACKED_CFG1_BYTES_PER_SWEEP = (3311.4e6 - 234.3e6) / 190
PACKED_CFG1_STATE_BYTES = 234.3e6 - 10 * PACKED_CFG1_BYTES_PER_SWEEP
PACKED_CFG1_TRAFFIC_BASIS = ("ncu 1-pass DRAM counters of this kernel build: 41.4 MB read + 3270 MB written per "
                             "200-sweep launch (and 234.3 MB for 10 sweeps), linear in the sweeps per launch; "
                             "the writes are the generator's word buffer written back from L2")


def roofline(c, rng, attempts, kernel_ms, launches, clocks, kernel, name="cfg1"):
    g = c["graph"]
    peak, mhz = int_peak_tops(clocks)
    if kernel_ms <= 0 or launches <= 0:
        return None
    if name == "cfg3" and rng == "mt19937":
        # each attempt streams its pre-generated word (4 B) from HBM; a launch
        # loads every replica's spins and int16 fields once and writes them
        # back (2 x 3 B per spin), amortised over the sweeps of the launch
        sweeps_per_launch = (attempts / (g.n * c["R"])) / launches
        bpa = 4.0 + 6.0 / sweeps_per_launch
        hbm, src = measured_peak("hbm_gbs")
        gbs = attempts * bpa / (kernel_ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "traffic": None, "peak_basis": src, "bytes_per_attempt": bpa, "sweeps_per_launch": sweeps_per_launch,
                "kernel_ms_per_launch": kernel_ms / launches, "launches": int(launches)}
    ops = attempts * ops_per_attempt(g, rng)
    achieved = ops / (kernel_ms * 1e-3) / 1e12
    # DRAM counters are reported only for the kernel build they were taken on:
    # the packed kernel with MT19937 on this workload (kernel variant 4)
    traffic, basis = None, "null: no ncu DRAM capture of this kernel build on this workload"
    if name == "cfg1" and rng == "mt19937" and kernel == 4:
        sweeps_per_launch = (attempts / (g.n * c["R"])) / launches
        traffic = PACKED_CFG1_STATE_BYTES + PACKED_CFG1_BYTES_PER_SWEEP * sweeps_per_launch
        basis = PACKED_CFG1_TRAFFIC_BASIS
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s (int32)",
            "frac": achieved / peak, "traffic": traffic,
            "traffic_basis": basis,
            "peak_basis": f"152 SM x 128 lanes x {mhz:.0f} MHz sampled SM clock (derived, not measured)",
            "kernel_ms_per_launch": kernel_ms / launches, "launches": int(launches),
            "ops_per_attempt": ops_per_attempt(g, rng)}


# one sweep level's dependent chain: the neighbour's column word (a shared
# load), ten dependent integer operations (the spin bit, its 2J, three adds of
# the field tree, the Trotter term, the sign, the threshold index, the compare,
# the flip), the threshold shuffle and the level barrier
LEVEL_CHAIN_INT_OPS = 10
_LATENCIES = None


def latency_floor(levels, sweeps_per_launch, kernel_ms_per_launch, clocks, resident=1):
    """Latency floor of a sweep launch: levels x sweeps x the cycles of one
    level's dependent chain, with the latencies measured on this GPU
    (ising_measure_latencies), at the sampled SM clock; frac = floor /
    measured kernel time.  Only for ladders whose replicas are all resident
    at once (a persistent launch); a larger ladder runs in waves of resident
    blocks and is bound by throughput, not by one replica's chain."""
    if not resident:
        return {"frac": None, "why": "replicas not all resident at once: the launch runs waves of blocks and is "
                                     "throughput-bound, so one replica's chain of levels does not bound it"}
    global _LATENCIES
    from paper_1004_0024_gb300 import ising
    if _LATENCIES is None:
        _LATENCIES = ising.ising_measure_latencies()
    lat = _LATENCIES
    cyc = lat["shared_load"] + LEVEL_CHAIN_INT_OPS * lat["int_mad"] + lat["shuffle"] + lat["barrier_8_warps"]
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    floor_ms = levels * sweeps_per_launch * cyc / (mhz * 1e3)
    return {"cycles_per_level": cyc, "levels_per_sweep": int(levels), "sweeps_per_launch": sweeps_per_launch,
            "ms_per_launch": floor_ms, "frac": floor_ms / kernel_ms_per_launch if kernel_ms_per_launch else None,
            "latencies_cycles": lat, "chain": f"shared load + {LEVEL_CHAIN_INT_OPS} dependent int ops + shuffle + "
                                              "8-warp barrier, per level (measured latencies)"}


# ------------------------------------------------------------- CPU oracle
def cpu_baseline(c, rng, seconds):
    import oracle
    if c["R"] > 512:  # a bounded sample: the first 512 replicas (no PT in this workload)
        c = dict(c, R=512, betas=c["betas"][:512])
    sim = oracle.Sim(c["graph"], c["betas"], seed=c["seed"], rng=rng)
    if "K" in c:
        sim.set_trotter(c["K"][:c["R"]])
    t0 = time.perf_counter()
    sw = 1 if c["swap_every"] else 0
    sim.run(4, sw)
    dt = time.perf_counter() - t0
    sweeps = max(4, int(seconds / max(dt / 4, 1e-6)))
    t0 = time.perf_counter()
    sim.run(sweeps, sw)
    dt = time.perf_counter() - t0
    att = c["graph"].n * c["R"] * sweeps
    return {"value": att / dt, "unit": "attempts/s", "cores": sim.threads, "kind": "oracle",
            "sample": f"same model, {c['R']} replicas, {sweeps} sweeps{' + PT after each' if sw else ''} "
                      f"({att:.3e} attempts, {dt:.1f} s)"}


def learned_study():
    """ESS/s of E and m with the learned column proposal interleaved 1:1
    with the sweep, against the plain sweep, on the same system (Philox
    streams), plus the fused network kernel against the bf16 tensor peak."""
    from paper_1004_0024_gb300 import ess, ising
    from paper_1004_0024_gb300 import workloads as W
    out = ess.study(ising, W, burn=20000, n_steps=16000, epochs=6)
    peak = measured_peak("bf16_tflops")
    net = out.pop("network")
    out["network_roofline"] = {
        "bound": "tensor", "achieved": net["tflops"], "peak": peak[0], "unit": "TFLOP/s",
        "frac": net["tflops"] / peak[0] if net["tflops"] and peak[0] else None, "peak_source": peak[1],
        "flop_per_column": net["flop_per_column"], "columns": net["columns"], "launches": net["launches"],
        "kernel": "mlp_fused_kernel (33->256->256->32, bf16 operands, FP32 accumulation in TMEM)"}
    return out


def measured_peak(key):
    try:
        with open(MEASURED) as f:
            return float(json.load(f)[key]), "measured (burst)"
    except (OSError, KeyError, ValueError):
        return {"bf16_tflops": 1900.0, "hbm_gbs": 6800.0}[key], "fallback"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    c = workload()
    sim = oracle.Sim(c["graph"], c["betas"], seed=c["seed"], rng=args.rng)
    per = 5  # sweeps per reference step (a bounded sample of the 200-sweep step)
    for _ in range(args.warmup):
        sim.run(per, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.run(per, 1)
    dt = time.perf_counter() - t0
    att = c["graph"].n * c["R"] * per * args.steps
    val = att / dt
    line = {"impl": "reference", "metric": "spin-flip attempts/sec vs roofline; ESS/sec learned proposal vs plain sweep", "value": val,
            "unit": "attempts/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int8 spins/int64 fields/uint32 RNG", "data": "synthetic",
            "config": {"workload": "32x32 lattice x 32 Trotter slices (32768 spins), 256 replicas, betas 0.05-5.0 geometric, PT each sweep",
                       "rng": args.rng, "sweeps_per_step": per},
            "cpu_baseline": {"value": val, "unit": "attempts/s", "cores": sim.threads, "kind": "oracle",
                             "sample": f"{per} sweeps + PT per step (bounded sample of the 200-sweep step)"},
            "e2e": {"value": val, "unit": "attempts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def learned_passes_only(n):
    """A short learned-pass case for profilers: 200 sweeps, one recording of
    R*S columns, one epoch, then n learned passes."""
    import torch

    from paper_1004_0024_gb300 import ising
    c = workload()
    sim = ising.Ising(c["graph"], c["betas"], seed=c["seed"], rng="philox", field_bits=c["field_bits"])
    sim.run(200, 1)
    S = c["graph"].n // c["graph"].n_slices
    net = ising.Mlp(c["graph"].n_slices, seed=1, capacity=c["R"] * S)
    net.collect(sim)
    loss = net.train(1, 4096, 1e-3)
    stats = [net.learned_pass(sim) for _ in range(n)]
    torch.cuda.synchronize()
    print(json.dumps({"learned_passes": n, "loss": loss, "accepted": [s["accepted"] for s in stats]}), flush=True)


def measure_batch(steps, warmup, sweeps, world, rank):
    """The ragged batch: 4096 instances (spin counts log-uniform in
    2^11..2^15, 8..64 replicas), autotuned, one step = ising_batch_run(sweeps,
    1) (a recorded CUDA graph of batched sweep and PT launches), Philox words.
    Under torchrun the instances are sharded over the ranks (rank r takes
    instances r, r + N, ...; numbered within its own batch): the total work is
    fixed, the value is every rank's attempts over the slowest rank's time.
    Returns the measurement on rank 0 (None elsewhere)."""
    import torch

    from paper_1004_0024_gb300 import ising
    from paper_1004_0024_gb300 import workloads as W
    t0 = time.perf_counter()
    built = [W.build_instance(d) for d in shard(W.ragged_instances(4096), rank, world)]
    inst = [(x["graph"], x["betas"], x["seed"]) for x in built]
    stream = torch.cuda.current_stream()
    b = ising.Batch(inst, rng="philox", field_bits=16, stream=stream.cuda_stream)
    b.autotune()
    setup_s = time.perf_counter() - t0
    per_step = sum(x["graph"].n * len(x["betas"]) for x in built) * sweeps
    for _ in range(warmup):
        b.run(sweeps, 1)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    first_clocks = None
    for timed_pass in range(2):
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for k in range(steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            b.run(sweeps, 1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clocks = sampler.stop()
        if timed_pass == 0 and any_rank(clocks_rejected(clocks), world):
            first_clocks = clocks  # throttled or clock-locked: measure once more
            continue
        break
    ms = max_over_ranks(sum(a.elapsed_time(e) for a, e in ev), world)
    total_per_step = sum_over_ranks(per_step, world)
    value = total_per_step * steps / (ms * 1e-3)
    resident = int(sum_over_ranks(sum(b.info(i)["resident"] for i in range(len(inst))), world))
    deg = sum(float(x["graph"].row_ptr[-1]) for x in built) / sum(x["graph"].n for x in built)
    ops = 20 + 6 + 3 * deg
    peak, mhz = int_peak_tops(clocks)
    b.close()
    if rank != 0:
        return None
    out = {"workload": f"4096 ragged instances (2^11..2^15 spins, 8..64 replicas), {sweeps} sweeps + PT each",
           "rng": "philox", "field_bits": 16, "value": value, "unit": "attempts/s", "ms_per_step": ms / steps,
           "steps": steps, "warmup": warmup, "attempts_per_step": total_per_step,
           "resident_instances": resident, "setup_seconds": setup_s, "clocks": clocks,
           "roofline": {"bound": "alu", "achieved": value / world * ops / 1e12, "peak": peak,
                        "unit": "Tops/s (int32)", "frac": value / world * ops / 1e12 / peak, "traffic": None,
                        "ops_per_attempt": ops, "per": "one GPU (the job's value divided by the ranks)",
                        "peak_basis": f"152 SM x 128 lanes x {mhz:.0f} MHz sampled SM clock (derived, not measured)",
                        "timed": "whole graph replay (every kernel of the step)"}}
    if first_clocks is not None:
        out["remeasured"] = {"first_clocks": first_clocks, "why": "slowdown or locked clock in the first timed pass"}
    return out


def run_batch(args):
    """bench.py --workload batch: the ragged batch as the line's workload."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    sweeps = args.sweeps if args.sweeps > 0 else 100
    m = measure_batch(args.steps, args.warmup, sweeps, world, rank)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {"metric": "spin-flip attempts/sec vs roofline; ESS/sec learned proposal vs plain sweep",
            "value": m["value"], "unit": "attempts/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": m["ms_per_step"], "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
            "dtype": "int8 spins/int16 fields/uint32 RNG", "data": "synthetic (seeded ragged layered models)",
            "config": {"workload": m["workload"], "rng": "philox", "attempts_per_step": m["attempts_per_step"],
                       "resident_instances": m["resident_instances"], "setup_seconds": m["setup_seconds"],
                       "l2": "flushed (512 MB write) between timed steps",
                       "parallelism": f"instances sharded x{world}" if world > 1 else "replicas-only x1"},
            "clocks": m["clocks"], "roofline": m["roofline"]}
    if "remeasured" in m:
        line["remeasured"] = m["remeasured"]
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.learned_passes > 0:
        learned_passes_only(args.learned_passes)
        return
    if args.workload == "batch" and args.impl != "reference":
        run_batch(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
