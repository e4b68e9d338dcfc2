#!/usr/bin/env python3
"""Throughput of the batched Kalman step on GB300: p2r propagate + update at
the paper's scale (100 events x 9,600 tracks, cylinder r = 30 cm).

One step = one pass of the propagate+update kernel over the whole batch,
inputs resident in HBM.  The step kernel is launched through the C ABI
(kf_p2r_propagate_update); the K timed launches are replayed from a CUDA
graph so that host launch overhead cannot starve a ~40 us kernel.  Inputs
(139 MB) and outputs (104 MB) exceed the 126 MB L2 and rotate over 4 buffer
sets, so no step reads what the previous one left in L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl kf|reference]

Under torchrun each rank processes its own batch (independent tracks: no
data-path collective); the timed region is bracketed by barriers and the
maximum time over ranks is reported (weak scaling).  --impl reference times
the FP64 CPU oracle on the host cores on bounded samples of the same
workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("tracks propagated+updated/sec on 1 GB300 (fused vs plain, ≤1e-4 rel err) "
          "and % of HBM roofline")
UNIT = "tracks/s"
NEVTS, NTRKS, RADIUS = 100, 9600, 30.0
# Algorithmic bytes per p2r track: read state 24 + cov 84 + charge 1 + hit 12
# + hit cov 24 = 145, write state 24 + cov 84 = 108.
BYTES_PER_TRACK_P2R = 253
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ("paper_2401_14221_gb300/csrc/kf_device.cuh",
                  "paper_2401_14221_gb300/csrc/kf_step.cu",
                  "paper_2401_14221_gb300/csrc/kf_step_staged.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["kf", "reference"], default="kf")
    ap.add_argument("--layout", default="auto",
                    help="auto | soa | aosoa16 | aosoa32 | aosoa64 | aosoa128")
    ap.add_argument("--step-kernel", default="auto", choices=["auto", "direct", "staged"])
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-chain", action="store_true",
                    help="skip the fused-chain vs per-layer-launch comparison")
    ap.add_argument("--chain-steps", type=int, default=10)
    ap.add_argument("--profile-only", action="store_true",
                    help="run a few launches of one layout and exit (for ncu captures)")
    ap.add_argument("--kind", choices=["p2r", "p2z"], default="p2r",
                    help="workload of --profile-only")
    ap.add_argument("--e2e-chunk", type=int, default=0,
                    help="tracks per pipeline chunk of the host-array call (0 = library default)")
    return ap.parse_args()


def workload_name():
    return f"p2r single step, {NEVTS} events x {NTRKS} tracks, r={RADIUS:g} cm, Bz=3.8 T"


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


def kernel_source_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "p2r_step_960k.json")
    try:
        with open(path) as f:
            prof = json.load(f)
        if prof.get("kernel_src_sha") == kernel_source_hash():
            return float(prof["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[4 + j] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------ reference arm

def reference_arm(args, rank, world):
    """The FP64 CPU oracle as it stands, on the host cores, on bounded samples
    of the same workload (rank 0 only)."""
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from paper_2401_14221_gb300 import workload as W

    w = W.make_p2r(NEVTS, NTRKS, seed=1)
    cores = os.cpu_count() or 1
    state, cov, hit, hc = (np.ascontiguousarray(a.T, dtype=np.float64)
                           for a in (w.state, w.cov, w.hit, w.hitcov))
    total = 4_000_000
    per_step = int(min(w.n, max(4096, total // max(1, args.steps + args.warmup))))

    def step(i):
        lo = (i * per_step) % (w.n - per_step + 1)
        sl = slice(lo, lo + per_step)
        oracle.step_batch(W.P2R, state[sl], cov[sl], w.charge[sl], hit[sl], hc[sl], w.surf, w.bz,
                          threads=cores)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    sample = f"{per_step} consecutive tracks of the {w.n}-track workload per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(), "tracks": w.n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- kf arm

def cpu_baseline(w):
    """The oracle timed on this host's cores over passes of the workload."""
    import numpy as np

    import oracle
    from paper_2401_14221_gb300 import workload as W

    cores = os.cpu_count() or 1
    state, cov, hit, hc = (np.ascontiguousarray(a.T, dtype=np.float64)
                           for a in (w.state, w.cov, w.hit, w.hitcov))
    passes, t0 = 0, time.perf_counter()
    c0 = time.process_time()
    while True:
        oracle.step_batch(W.P2R, state, cov, w.charge, hit, hc, w.surf, w.bz, threads=cores)
        passes += 1
        el = time.perf_counter() - t0
        if el > 2.0 or passes >= 20 or (time.process_time() - c0) > 20.0:
            break
    return {"value": passes * w.n / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{passes} full pass(es) over the {w.n}-track workload, "
                      f"{time.process_time() - c0:.1f} s CPU time"}


def chain_bench(args, kf, W, dev, rank):
    """Fused 15-layer chain vs the same chain as 15 single-step launches, on
    the 256-event workload (lognormal event sizes).  Both run in place, so the
    start state is restored before every timed run, outside the timed pair."""
    import torch

    from paper_2401_14221_gb300 import shard

    cw = W.make_chain(events=256, seed=shard.rank_seed(7, rank))
    dc = kf.chain_upload(cw, kf.KF_AOSOA, 32, dev)
    L = cw.L
    # per-layer launches captured once in a CUDA graph
    stream = torch.cuda.Stream()
    plain_graph = None
    try:
        dc.reset()
        with torch.cuda.stream(stream):
            dc.run_plain(stream=stream)
        torch.cuda.synchronize()
        plain_graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(plain_graph, stream=stream):
            dc.run_plain()
        torch.cuda.synchronize()
    except Exception:
        plain_graph = None

    def timed(fn, reps):
        ms = []
        for _ in range(reps):
            dc.reset()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return sorted(ms)[len(ms) // 2]

    reps = max(3, args.chain_steps)
    timed(dc.run, 2)
    fused_ms = timed(dc.run, reps)
    plain_fn = plain_graph.replay if plain_graph is not None else dc.run_plain
    timed(plain_fn, 2)
    plain_ms = timed(plain_fn, reps)
    # algorithmic bytes per track: fused reads state, cov, charge once (109 B),
    # hits + hit covariances per layer (36 B each), writes state + cov (108 B);
    # plain launches move 253 B per track per layer
    fused_b = 109 + 36 * L + 108
    plain_b = 253 * L
    return {"workload": f"{len(cw.event_sizes)} events, {cw.n} tracks (lognormal sizes, median "
                        f"5000, clipped 500-40000), {L} alternating layers",
            "tracks": cw.n, "layers": L,
            "fused_ms": fused_ms, "fused_tracks_per_s": cw.n / (fused_ms * 1e-3),
            "plain_ms": plain_ms, "plain_tracks_per_s": cw.n / (plain_ms * 1e-3),
            "speedup": plain_ms / fused_ms,
            "fused_GBps": fused_b * cw.n / (fused_ms * 1e-3) / 1e9,
            "plain_GBps": plain_b * cw.n / (plain_ms * 1e-3) / 1e9,
            "bytes_per_track": {"fused": fused_b, "plain": plain_b},
            "plain_launch": "CUDA graph" if plain_graph is not None else "eager",
            "timing": f"median of {reps} runs, CUDA events, state reset outside the timed pair"}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2401_14221_gb300 import build as kbuild
    from paper_2401_14221_gb300 import kf
    from paper_2401_14221_gb300 import shard
    from paper_2401_14221_gb300 import workload as W

    if not kbuild.up_to_date():
        kbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    layouts = {"soa": (kf.KF_SOA, 0), "aosoa16": (kf.KF_AOSOA, 16), "aosoa32": (kf.KF_AOSOA, 32),
               "aosoa64": (kf.KF_AOSOA, 64), "aosoa128": (kf.KF_AOSOA, 128)}

    if args.profile_only:
        w = (W.make_p2r(NEVTS, NTRKS, seed=1) if args.kind == "p2r"
             else W.make_p2z(NEVTS * NTRKS, seed=1))
        kind, width = layouts["aosoa16" if args.layout == "auto" else args.layout]
        kf.kf_set_step_kernel({"auto": kf.KF_STEP_AUTO, "direct": kf.KF_STEP_DIRECT,
                               "staged": kf.KF_STEP_STAGED}[args.step_kernel])
        bs = [kf.upload(w, kind, width, dev) for _ in range(2)]
        for i in range(5):
            bs[i % 2].run()
        torch.cuda.synchronize()
        print(f"profile-only: {args.kind} n={w.n} layout={args.layout}: 5 launches done")
        return 0

    w = W.make_p2r(NEVTS, NTRKS, seed=shard.rank_seed(1, rank))

    def time_launches(batches, reps):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for i in range(reps):
            batches[i % len(batches)].run()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    # Kernel x layout sweep (outside the timed region): the direct kernel on
    # SoA and AoSoA, the staged kernel on AoSoA block widths.
    modes = {"direct": kf.KF_STEP_DIRECT, "staged": kf.KF_STEP_STAGED}
    sweep = {}
    if args.layout == "auto" or args.step_kernel == "auto":
        for lname, (kind, width) in layouts.items():
            if args.layout != "auto" and lname != args.layout:
                continue
            bs = [kf.upload(w, kind, width, dev) for _ in range(2)]
            for mname, mode in modes.items():
                if kind == kf.KF_SOA and mname == "staged":
                    continue
                if args.step_kernel != "auto" and mname != args.step_kernel:
                    continue
                kf.kf_set_step_kernel(mode)
                time_launches(bs, 20)
                ms = time_launches(bs, 200)
                sweep[f"{mname}/{lname}"] = {"ms": ms, "tracks_per_s": w.n / (ms * 1e-3)}
            del bs
        best = min(sweep, key=lambda k: sweep[k]["ms"])
        chosen_kernel, chosen = best.split("/")
    else:
        chosen_kernel, chosen = args.step_kernel, args.layout
    kf.kf_set_step_kernel(modes[chosen_kernel])
    kind, width = layouts[chosen]
    sets = [kf.upload(w, kind, width, dev) for _ in range(4)]

    # Capture one launch per buffer set in a CUDA graph; replay it.
    stream = torch.cuda.Stream()
    graph = None
    try:
        with torch.cuda.stream(stream):
            for s in sets:
                s.run(stream=stream)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            for s in sets:
                s.run()
        torch.cuda.synchronize()
    except Exception as e:  # capture unsupported: eager launches
        print(f"# CUDA graph capture failed ({e}); timing eager launches", file=sys.stderr)
        graph = None

    reps_per_replay = len(sets) if graph is not None else 1

    def run_steps(k):
        if graph is not None:
            for _ in range(k // reps_per_replay):
                graph.replay()
            for i in range(k % reps_per_replay):
                sets[i].run()
        else:
            for i in range(k):
                sets[i % len(sets)].run()

    run_steps(max(args.warmup, 3))
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(dev)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local_rank)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)
    shard.barrier(world)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    run_steps(args.steps)
    t1.record()
    torch.cuda.synchronize()
    shard.barrier(world)
    clocks = sampler.stop()
    elapsed_ms = shard.max_over_ranks(t0.elapsed_time(t1), world, dev)
    ms_per_step = elapsed_ms / args.steps
    value = shard.whole_job_throughput(w.n, args.steps, world, elapsed_ms * 1e-3)

    # Roofline of the step kernel: algorithmic bytes / average launch time.
    peak, peak_src = measured_hbm_peak()
    achieved = BYTES_PER_TRACK_P2R * w.n / (ms_per_step * 1e-3) / 1e9
    traffic = profiled_traffic()

    # End to end through the host-array entry point (pinned host memory).
    e2e = None
    hb = kf.host_upload(w, kind, width, dev, chunk_tracks=args.e2e_chunk, pinned=True)
    hb.run()
    torch.cuda.synchronize()
    ke = max(3, args.e2e_steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    shard.barrier(world)
    e0.record()
    for _ in range(ke):
        hb.run()
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = shard.max_over_ranks(e0.elapsed_time(e1) / ke, world, dev)
    e2e = {"value": shard.whole_job_throughput(w.n, 1, world, e2e_ms * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": hb.h2d_bytes(), "d2h_bytes_per_step": hb.d2h_bytes(),
           "ms_per_step": e2e_ms, "host_memory": "pinned"}
    del hb

    chain = None
    if not args.no_chain:
        chain = chain_bench(args, kf, W, dev, rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(), "tracks": w.n, "layout": chosen,
                       "step_kernel": chosen_kernel,
                       "precision": "fp32 standard-form update",
                       "l2": "inputs 139 MB + outputs 104 MB per step (> 126 MB L2), "
                             "rotated over 4 buffer sets",
                       "launch": "CUDA graph of 4 launches" if graph is not None else "eager"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_src,
                         "bytes_per_track": BYTES_PER_TRACK_P2R},
            "chain": chain,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clocks,
            "sweep": sweep,
            "device_error": kf.kf_take_device_error(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
