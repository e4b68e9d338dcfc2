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
# p2z reads hit x, y and hit covariance xx, xy, yy only: 24 + 84 + 1 + 8 + 12
# read, 108 written
BYTES_PER_TRACK_P2Z = 237
# FP32 operations per track and layer of the fused chain (FFMA counted twice,
# FMUL, FADD), from the ncu thread-instruction counters of one chain launch
# on 64 events (bench.py --profile-only --kind chain; profiles/chain_instructions.json)
FLOPS_PER_TRACK_LAYER = 502
# FP32 peak from the unit counts: 152 SMs x 128 FP32 lanes x 2 flops x clock
SMS = 152
FP32_LANES = SMS * 128
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0
# what the staged step kernel is compiled from, flags included (the capture
# in profiles/ is valid while these are unchanged)
KERNEL_SOURCES = ("paper_2401_14221_gb300/csrc/kf_common.cuh",
                  "paper_2401_14221_gb300/csrc/kf_num.cuh",
                  "paper_2401_14221_gb300/csrc/kf_device.cuh",
                  "paper_2401_14221_gb300/csrc/kf_step.cuh",
                  "paper_2401_14221_gb300/csrc/kf_step.cu",
                  "paper_2401_14221_gb300/csrc/kf_step_staged.cuh",
                  "paper_2401_14221_gb300/csrc/kf_step_staged.cu",
                  "paper_2401_14221_gb300/csrc/kf_staged_p2r_f32.cu",
                  "paper_2401_14221_gb300/build.py")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["kf", "reference"], default="kf")
    ap.add_argument("--layout", default="auto",
                    help="auto | soa | aosoa16 | aosoa32 | aosoa64 | aosoa128")
    ap.add_argument("--step-kernel", default="auto",
                    choices=["auto", "direct", "staged", "staged2", "staged3"],
                    help="staged = staged2: 2 CTAs/SM x 3 stages; staged3: 3 CTAs/SM x 2 stages")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the host-array (end-to-end) timing; e2e is then null (for "
                         "launch lists of the device-resident step alone)")
    ap.add_argument("--no-chain", action="store_true",
                    help="skip the fused-chain vs per-layer-launch comparison")
    ap.add_argument("--chain-steps", type=int, default=10)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-scaling", action="store_true",
                    help="skip the context measurements of other sizes (240k / 3.84M p2r, "
                         "8,192 and 960k p2z)")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving-loop measurement")
    ap.add_argument("--serve-events", type=int, default=2048)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[3000.0, 10000.0],
                    help="Poisson arrival rates of the serving measurement, events/s")
    ap.add_argument("--profile-only", action="store_true",
                    help="run a few launches of one layout and exit (for ncu captures)")
    ap.add_argument("--kind", choices=["p2r", "p2z", "chain", "chain_adaptive", "compressed",
                                       "e2e"],
                    default="p2r",
                    help="workload of --profile-only")
    ap.add_argument("--e2e-chunk", type=int, default=0,
                    help="tracks per pipeline chunk of the host-array call (0 = library default)")
    return ap.parse_args()


def workload_name():
    return f"p2r single step, {NEVTS} events x {NTRKS} tracks, r={RADIUS:g} cm, Bz=3.8 T"


def workload_config(n):
    """The workload, the same for both arms (what is timed, not how)."""
    return {"workload": workload_name(), "tracks": n,
            "l2": "inputs larger than L2: per step 139 MB of inputs and 104 MB of outputs "
                  "against the GPU's 126 MB L2"}


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


def profiled_traffic(shape):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source and on the launch shape the bench times
    (kernel/layout, e.g. "staged3/aosoa32"); else None."""
    path = os.path.join(ROOT, "profiles", "p2r_step_960k.json")
    try:
        with open(path) as f:
            prof = json.load(f)
        entry = prof.get("shapes", {}).get(shape)
        if prof.get("kernel_src_sha") == kernel_source_hash() and entry:
            return float(entry["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


CHAIN_SOURCES = ("paper_2401_14221_gb300/csrc/kf_num.cuh",
                 "paper_2401_14221_gb300/csrc/kf_device.cuh",
                 "paper_2401_14221_gb300/csrc/kf_chain.cuh",
                 "paper_2401_14221_gb300/csrc/kf_chain.cu",
                 "paper_2401_14221_gb300/build.py")


def chain_source_hash():
    h = hashlib.sha256()
    for rel in CHAIN_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_chain_instructions():
    """Thread instructions per track-layer of the FP32 fused chain from the
    committed ncu summary, if taken on the current chain source; else None."""
    path = os.path.join(ROOT, "profiles", "chain_instructions.json")
    try:
        with open(path) as f:
            prof = json.load(f)
        if prof.get("kernel_src_sha") == chain_source_hash():
            return float(prof["instructions_per_track_layer"])
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
    # size each step's sample so the whole run takes about a minute of
    # oracle time (one calibration pass of 65,536 tracks first): per-step
    # samples large enough that thread start-up does not set the rate
    cal = min(w.n, 65536)
    t_cal = time.perf_counter()
    oracle.step_batch(W.P2R, state[:cal], cov[:cal], w.charge[:cal], hit[:cal], hc[:cal],
                      w.surf, w.bz, threads=cores)
    rate = cal / max(time.perf_counter() - t_cal, 1e-6)
    per_step = int(min(w.n, max(4096, rate * 60.0 / max(1, args.steps + args.warmup))))

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
        "data": "synthetic", "config": workload_config(w.n),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- kf arm

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        fields = dict(line.split(":", 1) for line in out.splitlines() if ":" in line)
        fields = {k.strip(): v.strip() for k, v in fields.items()}
        name = fields.get("Model name") or fields.get("BIOS Model name")
        if name:
            vendor = fields.get("Vendor ID", "")
            return f"{vendor} {name}".strip()
    except (OSError, subprocess.SubprocessError, ValueError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


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
    cpu_s = time.process_time() - c0
    # one core: a slice of the same workload
    m = min(w.n, 60000)
    sl = (slice(0, m), slice(None))
    t1 = time.perf_counter()
    oracle.step_batch(W.P2R, state[sl], cov[sl], w.charge[:m], hit[sl], hc[sl], w.surf, w.bz,
                      threads=1)
    one = m / (time.perf_counter() - t1)
    return {"value": passes * w.n / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"{passes} full pass(es) over the {w.n}-track workload, "
                      f"{cpu_s:.1f} s CPU time",
            "single_core_value": one,
            "single_core_sample": f"the first {m} tracks of the workload on one thread"}


def compressed_bench(kf, W, w, dev, kind, width, reps=100, staged=True):
    """The step on the compressed covariance store (FP32 sigmas + FP16
    correlations): 193 algorithmic bytes per p2r track instead of 253."""
    import torch

    lay = kf.make_layout(kind, width, w.n)
    sig, rho = W.compress_cov(w.cov)
    bufs = []
    for _ in range(4):
        st_in = kf.to_device(w.state, lay, dev)
        sg_in = kf.to_device(sig, lay, dev)
        rh_in = kf.to_device_rho(rho, lay, dev)
        bufs.append((st_in, sg_in, rh_in, torch.empty_like(st_in), torch.empty_like(sg_in),
                     torch.empty_like(rh_in), torch.from_numpy(w.charge).to(dev),
                     kf.to_device(w.hit, lay, dev), kf.to_device(w.hitcov, lay, dev),
                     torch.tensor([w.surf], dtype=torch.float32, device=dev),
                     torch.empty(w.n, dtype=torch.uint8, device=dev)))
    p = kf.make_params(w.bz)

    def run(b):
        kf.kf_propagate_update_compressed(kf.KF_P2R, p, lay, b[0], b[1], b[2], b[3], b[4], b[5],
                                          b[6], b[7], b[8], b[9], 0, b[10])
    run(bufs[0])
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for i in range(reps):
        run(bufs[i % 4])
    e.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(e) / reps
    return {"ms": ms, "tracks_per_s": w.n / (ms * 1e-3), "bytes_per_track": 193,
            "GBps": 193 * w.n / (ms * 1e-3) / 1e9,
            "kernel": "staged (bulk copies)" if (staged and kind == kf.KF_AOSOA)
                      else "one thread per track"}


def chain_bench(args, kf, W, dev, rank):
    """Fused 15-layer chain vs the same chain as 15 single-step launches, on
    the 256-event workload (lognormal event sizes).  Both run in place, so the
    start state is restored before every timed run, outside the timed pair."""
    import torch

    from paper_2401_14221_gb300 import shard

    cw = W.make_chain(events=256, seed=shard.rank_seed(7, rank))
    L = cw.L

    def median_run(d, reps=5):
        ms = []
        for _ in range(reps + 1):
            d.reset()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            d.run()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return sorted(ms[1:])[reps // 2]

    # Layout picked by measurement: every layout, each with the library's
    # chain autotuner (CTA size), timed on the fused chain; the fastest serves
    # the comparison below.  SoA only when n is a multiple of 4: the per-layer
    # launches of the comparison take each layer's hit arrays as 16-byte-
    # aligned slices of the stacked arrays.
    layouts = {"aosoa16": (kf.KF_AOSOA, 16), "aosoa32": (kf.KF_AOSOA, 32),
               "aosoa64": (kf.KF_AOSOA, 64), "aosoa128": (kf.KF_AOSOA, 128)}
    if cw.n % 4 == 0:
        layouts["soa"] = (kf.KF_SOA, 0)
    layout_sweep = {}
    for lname, (lk, lw) in layouts.items():
        d = kf.chain_upload(cw, lk, lw, dev)
        kf.autotune_chain(d)
        layout_sweep[lname] = median_run(d)
        del d
        torch.cuda.empty_cache()
    chosen = min(layout_sweep, key=layout_sweep.get)
    dc = kf.chain_upload(cw, *layouts[chosen], dev)
    # the library's chain autotuner picks the CTA size (served from its cache)
    tuned = kf.autotune_chain(dc)
    stream = torch.cuda.Stream()

    def capture(fn):
        # one fused launch, or the L per-layer launches, captured in a CUDA graph
        try:
            dc.reset()
            with torch.cuda.stream(stream):
                fn(stream=stream)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                fn()
            torch.cuda.synchronize()
            return g
        except Exception:
            return None

    fused_graph = capture(dc.run)
    plain_graph = capture(dc.run_plain)

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
    fused_fn = fused_graph.replay if fused_graph is not None else dc.run
    timed(fused_fn, 2)
    fused_ms = timed(fused_fn, reps)
    plain_fn = plain_graph.replay if plain_graph is not None else dc.run_plain
    timed(plain_fn, 2)
    plain_ms = timed(plain_fn, reps)
    # the fused chain under KF_ADAPTIVE (FP32, FP64 redo of ill-conditioned
    # layers), its CTA size picked by the library's tuner as for FP32
    ada_tuned = kf.autotune_chain(dc, kf.KF_ADAPTIVE)
    ada_fn = lambda: dc.run(kf.KF_ADAPTIVE)
    timed(ada_fn, 2)
    adaptive_ms = timed(ada_fn, reps)
    # context: the whole chain in double, and with the double-float update
    f64_fn = lambda: dc.run(kf.KF_FP64)
    timed(f64_fn, 1)
    fp64_ms = timed(f64_fn, max(3, reps // 3))
    df_tuned = kf.autotune_chain(dc, kf.KF_DF_UPDATE)
    df_fn = lambda: dc.run(kf.KF_DF_UPDATE)
    timed(df_fn, 1)
    df_ms = timed(df_fn, reps)
    # algorithmic bytes per track: fused reads state, cov, charge once (109 B),
    # per layer the hit and hit covariance a layer measures (a cylinder 36 B,
    # a plane x, y and their 2x2 covariance: 20 B), writes state + cov
    # (108 B); plain launches move 253 B (cylinder) or 237 B (plane) per layer
    hit_b = [36 if k == W.P2R else 20 for k in cw.kinds]
    fused_b = 109 + sum(hit_b) + 108
    plain_b = sum(253 if k == W.P2R else 237 for k in cw.kinds)
    # the chain is issue-bound: its roofline is the FP32 arithmetic peak
    fp32_peak = FP32_LANES * 2 * 2.07e9 / 1e12
    achieved = FLOPS_PER_TRACK_LAYER * cw.n * L / (fused_ms * 1e-3) / 1e12
    # and, as it is issue-bound, against the instruction-issue peak: one warp
    # instruction per scheduler per cycle, with the instructions per
    # track-layer of the committed ncu capture of the same kernel source
    issue = None
    ipl = profiled_chain_instructions()
    if ipl is not None:
        warp_instr_per_s = ipl / 32.0 * cw.n * L / (fused_ms * 1e-3)
        issue_peak = SMS * 4 * 2.07e9
        issue = {"instructions_per_track_layer": ipl, "achieved_warp_instr_per_s": warp_instr_per_s,
                 "peak": issue_peak, "frac": warp_instr_per_s / issue_peak,
                 "peak_source": "152 SMs x 4 schedulers x 1 warp instruction x 2.07 GHz",
                 "instructions_source": "profiles/chain_instructions.json (ncu, 64 events)"}
    return {"workload": f"{len(cw.event_sizes)} events, {cw.n} tracks (lognormal sizes, median "
                        f"5000, clipped 500-40000), {L} alternating layers",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak,
                         "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                         "flops_per_track_layer": FLOPS_PER_TRACK_LAYER,
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz",
                         "frac_of_hbm": fused_b * cw.n / (fused_ms * 1e-3) / 1e9
                                        / measured_hbm_peak()[0],
                         "issue": issue},
            "tracks": cw.n, "layers": L,
            "fused_ms": fused_ms, "fused_tracks_per_s": cw.n / (fused_ms * 1e-3),
            "plain_ms": plain_ms, "plain_tracks_per_s": cw.n / (plain_ms * 1e-3),
            "speedup": plain_ms / fused_ms,
            "fused_adaptive_ms": adaptive_ms,
            "fused_fp64_ms": fp64_ms,
            "fused_dfloat_update_ms": df_ms,
            # KF_ADAPTIVE and KF_FP64 meet the accuracy bounds on every track;
            # FP32 state between layers (all per-layer launches, and the
            # float-state fused variants) misses them on the ~0.3 % of tracks
            # that cross a layer at grazing incidence
            "accurate_fused_vs_plain": plain_ms / adaptive_ms,
            "fused_GBps": fused_b * cw.n / (fused_ms * 1e-3) / 1e9,
            "plain_GBps": plain_b * cw.n / (plain_ms * 1e-3) / 1e9,
            "bytes_per_track": {"fused": fused_b, "plain": plain_b},
            "fused_launch": "CUDA graph" if fused_graph is not None else "eager",
            "plain_launch": "CUDA graph" if plain_graph is not None else "eager",
            "autotune": tuned, "autotune_adaptive": ada_tuned,
            "autotune_dfloat_update": df_tuned, "layout": chosen,
            "layout_sweep_ms": layout_sweep,
            "timing": f"median of {reps} runs, CUDA events, state reset outside the timed pair"}


def serving_bench(args, kf, W, dev, rank):
    """Poisson event stream through the continuous-batching server vs a
    per-event synchronous baseline (copy in, chain, copy out, synchronise),
    both fed the same arrival times.  Events come from the 256-event chain
    workload (lognormal sizes), cycled; latency = arrival to results in host
    memory."""
    import threading

    import numpy as np
    import torch

    from paper_2401_14221_gb300 import shard

    cw = W.make_chain(events=256, seed=shard.rank_seed(11, rank))
    bounds = np.concatenate([[0], np.cumsum(cw.event_sizes)])
    E = len(cw.event_sizes)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    ev_in, ev_out = [], []
    for e in range(E):
        lo, hi = int(bounds[e]), int(bounds[e + 1])
        ev_in.append((pin(cw.state[:, lo:hi]), pin(cw.cov[:, lo:hi]), pin(cw.charge[lo:hi]),
                      pin(cw.hit[:, :, lo:hi]), pin(cw.hitcov[:, :, lo:hi])))
        n = hi - lo
        ev_out.append((torch.empty((6, n), dtype=torch.float32).pin_memory(),
                       torch.empty((21, n), dtype=torch.float32).pin_memory(),
                       torch.empty(n, dtype=torch.uint8).pin_memory()))
    total = args.serve_events
    order = np.arange(total) % E
    tracks = int(sum(cw.event_sizes[order]))
    arena = torch.empty(4 << 30, dtype=torch.uint8, device=dev)
    srv = kf.Server(cw.bz, cw.kinds, cw.pos, arena, max_events_in_flight=256)
    # warm-up: load the batched kernel's module and touch the arena
    for t in [srv.submit(*ev_in[e], *ev_out[e]) for e in range(16)]:
        srv.wait(t, 120.0)

    def serve(rate, seed, path=kf.KF_HOST_AUTO):
        # path: the host-path mode at submission (AUTO: these pinned events go
        # direct, the kernel on their host arrays; COPY: through the arena)
        arrivals = np.cumsum(np.random.default_rng(seed).exponential(1.0 / rate, total))
        kf.kf_set_host_path(path)
        srv.reset_stats()
        tickets = [None] * total
        t0 = time.perf_counter()

        def produce():
            for k in range(total):
                dt = t0 + arrivals[k] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                e = order[k]
                tickets[k] = srv.submit(*ev_in[e], *ev_out[e])

        th = threading.Thread(target=produce)
        th.start()
        th.join()
        for t in tickets:
            srv.wait(t, 120.0)
        t_end = time.perf_counter()
        kf.kf_set_host_path(kf.KF_HOST_AUTO)
        st = srv.stats()
        return arrivals, {"rate_events_per_s": rate, "tracks_per_s": tracks / (t_end - t0),
                          "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
                          "batches": st["batches"], "max_batch_events": st["max_batch_events"],
                          "scheduler_ms": {"longest_pass": st["sched_pass_max_ms"],
                                           "longest_gap_while_busy": st["sched_gap_max_ms"]},
                          "phases_ms": {ph: [st[f"{ph}_p50_ms"], st[f"{ph}_p99_ms"]]
                                        for ph in ("queue", "ready", "copyin", "compute",
                                                   "out", "gpu_copyin", "gpu_compute",
                                                   "gpu_out", "copyin_issue")}}

    runs = [serve(rate, 12 + rank + k) for k, rate in enumerate(args.serve_rates)]
    runs_copy = [serve(rate, 12 + rank + k, kf.KF_HOST_COPY)[1]
                 for k, rate in enumerate(args.serve_rates)]
    srv.close()
    del arena

    # --- per-event synchronous baseline on the same arrival times
    nmax = int(cw.event_sizes.max())
    L = cw.L
    d_state = torch.empty(6 * nmax, dtype=torch.float32, device=dev)
    d_cov = torch.empty(21 * nmax, dtype=torch.float32, device=dev)
    d_q = torch.empty(nmax, dtype=torch.int8, device=dev)
    d_hits = torch.empty(3 * nmax * L, dtype=torch.float32, device=dev)
    d_hc = torch.empty(6 * nmax * L, dtype=torch.float32, device=dev)
    d_status = torch.empty(nmax, dtype=torch.uint8, device=dev)
    layers = kf.make_layers(cw.kinds, cw.pos)
    params = kf.make_params(cw.bz)

    def sync_one(e):
        n = int(cw.event_sizes[e])
        si, ci, qi, hi_, hci = ev_in[e]
        so, co, sto = ev_out[e]
        d_state[:6 * n].copy_(si.view(-1), non_blocking=True)
        d_cov[:21 * n].copy_(ci.view(-1), non_blocking=True)
        d_q[:n].copy_(qi, non_blocking=True)
        d_hits[:3 * n * L].copy_(hi_.view(-1), non_blocking=True)
        d_hc[:6 * n * L].copy_(hci.view(-1), non_blocking=True)
        kf.kf_kalman_chain(params, kf.make_layout(kf.KF_SOA, 0, n), d_state[:6 * n],
                           d_cov[:21 * n], d_q[:n], d_hits[:3 * n * L], d_hc[:6 * n * L], layers,
                           d_status[:n])
        so.view(-1).copy_(d_state[:6 * n], non_blocking=True)
        co.view(-1).copy_(d_cov[:21 * n], non_blocking=True)
        sto.copy_(d_status[:n], non_blocking=True)
        torch.cuda.synchronize()

    for e in range(16):
        sync_one(e)
    results = []
    for (arrivals, served), served_copy in zip(runs, runs_copy):
        lat = []
        t0 = time.perf_counter()
        for k in range(total):
            arr = t0 + arrivals[k]
            dt = arr - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            sync_one(order[k])
            lat.append((time.perf_counter() - arr) * 1e3)
        t_end = time.perf_counter()
        lat = np.sort(np.array(lat))
        sync = {"tracks_per_s": tracks / (t_end - t0), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat[-1])}
        results.append({"rate_events_per_s": served["rate_events_per_s"],
                         "continuous_batching": served,
                         "continuous_batching_copy_path": served_copy,
                         "per_event_sync": sync})
    return {"workload": f"{total} events per rate (Poisson) cycled from 256 lognormal events "
                        f"(median 5000 tracks), {L}-layer chain", "tracks": tracks,
            "by_rate": results, "latency": "arrival to results in host memory; "
            "server latency counted from submit (= arrival: the producer never waits)",
            "paths": "continuous_batching: pinned events go direct (the batch kernel reads and "
                     "writes their host arrays over the CPU-GPU link); "
                     "continuous_batching_copy_path: the same events copied through the arena"}


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

    if args.profile_only and args.kind in ("chain", "chain_adaptive"):
        # the fused chain on 64 events of the chain workload (256 for the
        # adaptive one: its redo pass has work on the full workload), a few
        # launches from the same start state
        adaptive = args.kind == "chain_adaptive"
        cw = W.make_chain(events=256 if adaptive else 64, seed=7)
        dc = kf.chain_upload(cw, kf.KF_AOSOA, 32, dev)
        for _ in range(3):
            dc.reset()
            dc.run(kf.KF_ADAPTIVE if adaptive else kf.KF_FP32)
        torch.cuda.synchronize()
        print(f"profile-only: {args.kind} n={cw.n} L={cw.L}: 3 launches done")
        return 0
    if args.profile_only and args.kind == "e2e":
        # the host-array step on pinned memory (the direct path: the kernel
        # reads and writes the host arrays), a few calls
        w = W.make_p2r(NEVTS, NTRKS, seed=1)
        kind, width = layouts["aosoa32" if args.layout == "auto" else args.layout]
        hb = kf.host_upload(w, kind, width, dev, pinned=True)
        for _ in range(3):
            hb.run()
        torch.cuda.synchronize()
        print(f"profile-only: e2e n={w.n} layout={args.layout}: 3 calls done")
        return 0
    if args.profile_only and args.kind == "compressed":
        # the p2r step on the compressed covariance store, a few launches
        w = W.make_p2r(NEVTS, NTRKS, seed=1)
        kind, width = layouts["aosoa32" if args.layout == "auto" else args.layout]
        out = compressed_bench(kf, W, w, dev, kind, width, reps=5)
        print(f"profile-only: compressed n={w.n} layout={args.layout}: {out['ms']:.4f} ms")
        return 0
    if args.profile_only:
        w = (W.make_p2r(NEVTS, NTRKS, seed=1) if args.kind == "p2r"
             else W.make_p2z(NEVTS * NTRKS, seed=1))
        kind, width = layouts["aosoa16" if args.layout == "auto" else args.layout]
        kf.kf_set_step_kernel({"auto": kf.KF_STEP_AUTO, "direct": kf.KF_STEP_DIRECT,
                               "staged": kf.KF_STEP_STAGED, "staged2": kf.KF_STEP_STAGED,
                               "staged3": kf.KF_STEP_STAGED}[args.step_kernel])
        kf.kf_set_staged_ctas_per_sm(3 if args.step_kernel == "staged3" else 2)
        bs = [kf.upload(w, kind, width, dev) for _ in range(2)]
        for i in range(5):
            bs[i % 2].run()
        torch.cuda.synchronize()
        print(f"profile-only: {args.kind} n={w.n} layout={args.layout}: 5 launches done")
        return 0

    w = W.make_p2r(NEVTS, NTRKS, seed=shard.rank_seed(1, rank))

    # Launches per CUDA graph.  Inside a graph consecutive launches keep their
    # programmatic-dependent-launch overlap (the next kernel's CTAs start and
    # prefetch while the previous one drains); at a graph boundary they do
    # not, so a longer graph leaves fewer boundaries per launch (measured on
    # the staged step: 38.7 us per launch with 4 launches per graph, 37.1
    # with 16, 36.9 with 64).
    PER_GRAPH = 16

    def graph_time(batches, replays):
        # PER_GRAPH launches cycling over the batches, captured in a CUDA
        # graph and replayed; ms per launch
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            for b in batches:
                b.run(stream=st)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            for k in range(PER_GRAPH):
                batches[k % len(batches)].run()
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(replays):
            g.replay()
        b_.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b_) / (replays * PER_GRAPH)

    # Kernel x layout sweep (outside the timed region): the direct kernel and
    # the staged kernel (2 or 3 CTAs per SM) on SoA and the AoSoA widths.
    # direct: one thread per track, 128-thread CTAs; staged2 / staged3: the
    # persistent bulk-copy kernel with 2 CTAs x 3 stages or 3 CTAs x 2 stages
    modes = {"direct": kf.KF_STEP_DIRECT, "staged": kf.KF_STEP_STAGED,
             "staged2": kf.KF_STEP_STAGED, "staged3": kf.KF_STEP_STAGED}
    swept = ("direct", "staged2", "staged3")
    sweep = {}
    if args.layout == "auto" or args.step_kernel == "auto":
        for lname, (kind, width) in layouts.items():
            if args.layout != "auto" and lname != args.layout:
                continue
            bs = [kf.upload(w, kind, width, dev) for _ in range(2)]
            for mname in swept:
                mode = modes[mname]
                if args.step_kernel != "auto" and mname != args.step_kernel:
                    continue
                kf.kf_set_step_kernel(mode)
                # staged: 2 CTAs per SM x 3 stages; staged3: 3 x 2 stages
                kf.kf_set_staged_ctas_per_sm(3 if mname == "staged3" else 2)
                ms = graph_time(bs, 100)
                sweep[f"{mname}/{lname}"] = {"ms": ms, "tracks_per_s": w.n / (ms * 1e-3)}
            del bs
        best = min(sweep, key=lambda k: sweep[k]["ms"])
        chosen_kernel, chosen = best.split("/")
    else:
        chosen_kernel, chosen = args.step_kernel, args.layout
    kf.kf_set_step_kernel(modes[chosen_kernel])
    kf.kf_set_staged_ctas_per_sm(3 if chosen_kernel == "staged3" else 2)
    kind, width = layouts[chosen]
    sets = [kf.upload(w, kind, width, dev) for _ in range(4)]
    tuned = None
    if args.step_kernel == "auto":
        # the library's autotuner on the chosen layout, for the record: the
        # timed launches keep the sweep's choice (graph-timed, as they are),
        # so that the headline's launch shape is the measured best one
        kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
        tuned = kf.autotune_step(sets[0])
        kf.kf_set_step_kernel(modes[chosen_kernel])
        kf.kf_set_staged_ctas_per_sm(3 if chosen_kernel == "staged3" else 2)

    # Every timed launch is a graph replay: a CUDA graph of exactly k launches
    # cycling over the buffer sets (captured once per k, outside the timed
    # region), so that the timed region has one graph boundary however many
    # steps are asked for.  Beyond MAX_GRAPH launches, graphs of PER_GRAPH
    # launches are replayed, plus one graph of the remainder.
    MAX_GRAPH = 1024
    stream = torch.cuda.Stream()
    graphs = {}
    graph_ok = True
    with torch.cuda.stream(stream):
        for s in sets:
            s.run(stream=stream)
    torch.cuda.synchronize()

    def graph_of(k):
        if k not in graphs:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                for i in range(k):
                    sets[i % len(sets)].run()
            torch.cuda.synchronize()
            graphs[k] = g
        return graphs[k]

    def plan(k):
        # the graphs that make up k launches, captured before any timing
        if k <= 0:
            return []
        if k <= MAX_GRAPH:
            return [graph_of(k)]
        reps, rest = divmod(k, PER_GRAPH)
        return [graph_of(PER_GRAPH)] * reps + ([graph_of(rest)] if rest else [])

    try:
        # capture, then replay every graph once: a graph's first launch also
        # uploads it to the device, which must not land in the timed region
        for g in set(plan(args.steps) + plan(max(args.warmup, 3))):
            g.replay()
        torch.cuda.synchronize()
    except Exception as e:  # capture unsupported: eager launches
        print(f"# CUDA graph capture failed ({e}); timing eager launches", file=sys.stderr)
        graph_ok = False

    def run_steps(k):
        if graph_ok:
            for g in plan(k):
                g.replay()
        else:
            for i in range(k):
                sets[i % len(sets)].run()

    # Clock sampling starts first; the warm-up steps then run right before the
    # timed ones, so that the GPU is not idle (clocks settling) when timing
    # starts.
    props = torch.cuda.get_device_properties(dev)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local_rank)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)
    run_steps(max(args.warmup, 3))
    torch.cuda.synchronize()
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

    # The p2z single step on 8,192 tracks (the small configuration): latency
    # of one launch, graph-replayed back to back; and p2z at the p2r batch
    # size (237 algorithmic bytes per track: hit z and three hit-covariance
    # entries are not read)
    p2z_small_us, p2z_small_isolated_us, p2z_small_call_us, p2z_big = None, None, None, None
    p2z_small_prepared_us = None
    if not args.no_scaling:
        w_small = W.make_p2z(8192, seed=shard.rank_seed(1, rank))
        small = [kf.upload(w_small, kind, width, dev) for _ in range(2)]
        p2z_small_us = graph_time(small, 500) * 1e3
        # and as the latency of one launch on an otherwise idle GPU (median
        # of 50): on the device, events around a launch that was queued behind
        # a short sleep kernel, so that the host's call overhead is not in
        # it; and of the whole call, the events recorded before the host
        # makes it
        lat, call, prep = [], [], []
        prepared = [b_.prepare() for b_ in small]
        for k in range(55):
            torch.cuda.synchronize()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda._sleep(400000)
            a_.record()
            small[k % 2].run()
            b_.record()
            torch.cuda.synchronize()
            c_, d_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c_.record()
            small[k % 2].run()
            d_.record()
            torch.cuda.synchronize()
            e_, f_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e_.record()
            prepared[k % 2]()
            f_.record()
            torch.cuda.synchronize()
            if k >= 5:
                lat.append(a_.elapsed_time(b_) * 1e3)
                call.append(c_.elapsed_time(d_) * 1e3)
                prep.append(e_.elapsed_time(f_) * 1e3)
        p2z_small_isolated_us = float(np.median(lat))
        p2z_small_call_us = float(np.median(call))
        p2z_small_prepared_us = float(np.median(prep))
        del small
        w_z = W.make_p2z(w.n, seed=shard.rank_seed(2, rank))
        bz_ = [kf.upload(w_z, kind, width, dev) for _ in range(4)]
        ms_z = graph_time(bz_, 200)
        p2z_big = {"tracks": w_z.n, "ms": ms_z, "tracks_per_s": w_z.n / (ms_z * 1e-3),
                   "GBps": BYTES_PER_TRACK_P2Z * w_z.n / (ms_z * 1e-3) / 1e9,
                   "bytes_per_track": BYTES_PER_TRACK_P2Z}
        del bz_, w_z

    # Spread: ten timed repeats of the same timed region (the same K graph-
    # replayed launches), so that its mean and sd describe the headline.
    reps = []
    for _ in range(10):
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record()
        run_steps(args.steps)
        r1.record()
        torch.cuda.synchronize()
        reps.append(r0.elapsed_time(r1) / args.steps)
    reps_sorted = sorted(reps)
    spread = {"repeats": 10, "steps_each": args.steps,
              "ms_per_step_mean": sum(reps) / 10,
              "ms_per_step_sd": (sum((x - sum(reps) / 10) ** 2 for x in reps) / 9) ** 0.5,
              "ms_per_step_p50": 0.5 * (reps_sorted[4] + reps_sorted[5])}

    peak, peak_src = measured_hbm_peak()
    # Batch-size scaling of the same kernel (context: a fixed per-launch cost
    # of ramp, tail and launch gap weighs less on larger batches).  The
    # 960,000-track arrays are cut to a quarter (four buffer sets rotate, 244 MB
    # in all, more than L2 holds) or tiled to 4x (two sets rotate).
    scaling = []
    if not args.no_scaling:
        import dataclasses

        import numpy as np
        for mult, reps in ((0.25, 400), (4, 100)):
            m = int(w.n * mult)
            tile = (lambda a: np.tile(a, (1, 4))[:, :m]) if mult > 1 else (lambda a: a[:, :m])
            wm = dataclasses.replace(w, n=m, state=tile(w.state), cov=tile(w.cov),
                                     charge=np.tile(w.charge, 4)[:m], hit=tile(w.hit),
                                     hitcov=tile(w.hitcov))
            bm = [kf.upload(wm, kind, width, dev) for _ in range(4 if mult < 1 else 2)]
            # each size with the launch shape the library's autotuner picks
            # for it (the headline's shape suits 960,000 tracks)
            kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
            shape = kf.autotune_step(bm[0])
            ms_m = graph_time(bm, reps)
            kf.kf_set_step_kernel(modes[chosen_kernel])
            kf.kf_set_staged_ctas_per_sm(3 if chosen_kernel == "staged3" else 2)
            scaling.append({"tracks": m, "ms": ms_m, "tracks_per_s": m / (ms_m * 1e-3),
                            "GBps": BYTES_PER_TRACK_P2R * m / (ms_m * 1e-3) / 1e9,
                            "frac": BYTES_PER_TRACK_P2R * m / (ms_m * 1e-3) / 1e9 / peak,
                            "shape": shape})
            del bm

    # Roofline of the step kernel: algorithmic bytes / average launch time.
    achieved = BYTES_PER_TRACK_P2R * w.n / (ms_per_step * 1e-3) / 1e9
    traffic = profiled_traffic(f"{chosen_kernel}/{chosen}")

    # End to end through the host-array entry point: HOST arrays in and out,
    # the transfers inside the timed region.  Two batches alternate, so that
    # no step finds its inputs in L2 (each batch's inputs are 139 MB).
    def time_host(pinned, path):
        kf.kf_set_host_path(path)
        try:
            hbs = [kf.host_upload(w, kind, width, dev, chunk_tracks=args.e2e_chunk, pinned=pinned)
                   for _ in range(2)]
            for hb in hbs:
                hb.run()
            torch.cuda.synchronize()
            ke = max(3, args.e2e_steps)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            shard.barrier(world)
            e0.record()
            for k in range(ke):
                hbs[k % 2].run()
            e1.record()
            torch.cuda.synchronize()
            ms = shard.max_over_ranks(e0.elapsed_time(e1) / ke, world, dev)
            return ms, hbs[0].h2d_bytes(), hbs[0].d2h_bytes()
        finally:
            kf.kf_set_host_path(kf.KF_HOST_AUTO)

    e2e = None
    if not args.no_e2e:
        # pinned memory, the default path (direct: the kernel reads and writes
        # the host arrays over the CPU-GPU link)
        e2e_ms, h2d, d2h = time_host(True, kf.KF_HOST_AUTO)
        e2e = {"value": shard.whole_job_throughput(w.n, 1, world, e2e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": e2e_ms, "host_memory": "pinned", "path": "direct",
               "transfer": "the step kernel loads the inputs from and stores the results to "
                           "the pinned host arrays over the CPU-GPU link inside the timed "
                           "region (no copy engine); copy_path_value: the same with chunked "
                           "cudaMemcpyAsync copies"}
        # context: the copy-engine pipeline on the same pinned arrays, and both
        # paths from pageable memory
        ms_copy = time_host(True, kf.KF_HOST_COPY)[0]
        e2e["copy_path_value"] = w.n / (ms_copy * 1e-3)
        try:
            e2e["pageable_value"] = w.n / (time_host(False, kf.KF_HOST_AUTO)[0] * 1e-3)
        except kf.KfError:
            e2e["pageable_value"] = None
        e2e["pageable_copy_path_value"] = w.n / (time_host(False, kf.KF_HOST_COPY)[0] * 1e-3)


    # Update variants and the compressed covariance store on the same batch
    # (context for the precision study; errors are measured by the tests).
    variants = {}
    if not args.no_variants:
        # each variant with the library's default launch shape for it
        kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
        kf.autotune_clear()
        for vname, prec in (("fp32", kf.KF_FP32), ("fp64_update", kf.KF_FP64_UPDATE),
                            ("dfloat_update", kf.KF_DF_UPDATE),
                            ("joseph", kf.KF_JOSEPH), ("fp64", kf.KF_FP64),
                            ("adaptive", kf.KF_ADAPTIVE)):
            sets[0].run(prec)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for i in range(100):
                sets[i % len(sets)].run(prec)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / 100
            variants[vname] = {"ms": ms, "tracks_per_s": w.n / (ms * 1e-3),
                               "GBps": BYTES_PER_TRACK_P2R * w.n / (ms * 1e-3) / 1e9}
        # the compressed store: its staged kernel (the default for AoSoA), and
        # its one-thread-per-track kernel
        mode_now = modes[chosen_kernel]
        kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
        variants["compressed_fp32"] = compressed_bench(kf, W, w, dev, kind, width)
        kf.kf_set_step_kernel(kf.KF_STEP_DIRECT)
        variants["compressed_fp32_direct"] = compressed_bench(kf, W, w, dev, kind, width,
                                                              staged=False)
        kf.kf_set_step_kernel(mode_now)

    chain = None
    if not args.no_chain:
        chain = chain_bench(args, kf, W, dev, rank)

    serving = None
    if not args.no_serving:
        serving = serving_bench(args, kf, W, dev, rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

    if p2z_big is not None:
        p2z_big["frac"] = p2z_big["GBps"] / peak
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(w.n),
            "setup": {"layout": chosen,
                      "step_kernel": chosen_kernel,
                      "precision": "fp32 standard-form update",
                      "buffers": "4 buffer sets rotated, so no step reads what the previous "
                                 "one left in L2",
                      "launch": ((f"one CUDA graph of the {args.steps} timed launches cycling "
                                  "over the 4 sets" if args.steps <= MAX_GRAPH else
                                  f"CUDA graphs of {PER_GRAPH} launches and one of the "
                                  "remainder, cycling over the 4 sets")
                                 if graph_ok else "eager")},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_src,
                         "frac_of_nominal_7900": achieved / NOMINAL_HBM_GBS,
                         "bytes_per_track": BYTES_PER_TRACK_P2R},
            "variants": variants,
            "chain": chain,
            "serving": serving,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clocks,
            "spread": spread,
            "batch_scaling": scaling,
            "p2z_8192_us_per_launch": p2z_small_us,
            "p2z_8192_isolated_latency_us": p2z_small_isolated_us,
            "p2z_8192_call_latency_us": p2z_small_call_us,
            "p2z_8192_prepared_call_latency_us": p2z_small_prepared_us,
            "p2z_960k": p2z_big,
            "sweep": sweep,
            "autotune": tuned,
            "device_error": kf.kf_take_device_error(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
