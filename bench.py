"""Benchmark: events/s and ell-sweeps/s of the event-chain sweep on one GB300.

Workload (the 10^6-bead melt): 1000 chains x N=1000 on a 100^3 lattice,
spacing 1.05 sigma (phi ~ 0.45), b_max = 1.2 sigma, ell = 20 sigma,
isotropic directions, FP32 screen + FP64 confirmation, swap moves calibrated
to 0.1 attempts per bead per sweep; lanes per EC, tile side, cell side and
ECs per tile picked by the library's autotuner (outside the timed region).
One step = one sweep: domain assignment + cell list + one EC launch.

The batched form (256 replicas of uneven N, bead count and phi, one CUDA
graph per sweep, autotuned) is timed in the same run and reported under
`batched`, against the same replicas advanced one at a time through the
single-melt API and against the batched plain FP64 kernel.

`value` is events/s of the FP32-screened form (inputs resident in HBM, L2
flushed between steps, device time from CUDA events).  The plain FP64 kernel
on the same state is reported beside it.  `e2e` goes through the public API
with host buffers (positions in, one sweep, positions out).

`--impl reference` times the oracle (plain serial FP64 C, the checker of the
CUDA path) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1502_06447_gb300.configs import C2, C3, C5, C5_LAUNCH, C5_LAUNCH_FP64  # noqa: E402

WORKLOADS = {"c5": (C5, (25, 25, 25)), "c3": (C3, (20, 20, 20)), "c2": (C2, (16, 16, 16))}
C5_DEFAULT = C5
ELL = C5.ell
TILES = (25, 25, 25)
SWAP_RATE = 0.1
METRIC = "events/s (EC sweep, 1e6-bead melt, FP32 screen + FP64 confirm)"
UNIT = "events/s"
C0 = 1.2  # stencil cell side of the bytes-per-event definition (= b_max)
# revision of the block-lockstep kernel; DRAM counters in profiles/ are used
# only when they were taken on the same revision
KERNEL_REV = 6


def launch_settings(args):
    """Timed launch settings {screened: ..., fp64: ...}: the pinned ones for
    the 1e6-bead melt, 8 / 16 lanes with one EC per tile elsewhere, each
    field overridable from the command line."""
    base = {True: dict(C5_LAUNCH), False: dict(C5_LAUNCH_FP64)}
    for k in (True, False):
        if C5.name != "c5_swap_1m":
            base[k].update(tiles=TILES, ecs_per_tile=1, cell_side=1.05)
        if args.tiles:
            base[k]["tiles"] = (args.tiles,) * 3
        if args.ecs_per_tile:
            base[k]["ecs_per_tile"] = args.ecs_per_tile
    if args.lanes:
        base[True]["lanes"] = args.lanes
    if args.lanes64:
        base[False]["lanes"] = args.lanes64
    if args.block_tiles >= 0:
        base[True]["block_tiles"] = args.block_tiles
    base[False]["block_tiles"] = 0
    return base


LAUNCH = None
# push-off sweeps run the plain FP64 kernel with one tile per warp: at these
# sizes (a few hundred tiles, often only a few with overlapping beads) a
# sweep is as long as its slowest tile, and 32 lanes step a tile fastest
# (5,340 beads: 0.96 s at 32 lanes, 1.30 s at 16, 1.90 s at 8; the same
# sweeps and positions)
PO_LANES = 32
# untimed sweeps that melt the lattice start before tuning and timing
MELT_SWEEPS = 20


def bytes_per_event(phi, confirmed_per_event, fp32f=True):
    """Algorithmic bytes per event: a 27-cell stencil of side c0 = b_max
    holds nbar = rho 27 c0^3 beads; FP64 reads 24 B each, the FP32 screen
    16 B each plus 24 B per FP64-confirmed bead; 216 B of cell offsets,
    96 (FP32) or 72 (FP64) B of pivot and bond partners, 24 B written."""
    rho = 6.0 * phi / math.pi
    nbar = rho * 27.0 * C0 ** 3
    if fp32f:
        return 16.0 * nbar + 24.0 * confirmed_per_event + 216.0 + 96.0
    return 24.0 * nbar + 216.0 + 72.0 + 24.0


def reduce_over_ranks(sums, maxes, device):
    """Whole-job aggregates of a replicas run: `sums` added over the ranks
    (events), `maxes` maxed (times).  Returns two lists of floats."""
    import torch
    import torch.distributed as dist
    ts = torch.tensor([float(x) for x in sums], dtype=torch.float64, device=device)
    tm = torch.tensor([float(x) for x in maxes], dtype=torch.float64, device=device)
    dist.all_reduce(ts, op=dist.ReduceOp.SUM)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    return ts.tolist(), tm.tolist()


def rank_seed(base, rank):
    """Each rank advances its own replica: the Philox key's seed word is
    offset by the rank."""
    return int(base) + int(rank)


def setting_key(kernel, st):
    """The key a DRAM profile is filed under: kernel revision and the whole
    launch setting."""
    return (f"{kernel} rev {KERNEL_REV} lanes {st['lanes']} tiles {'x'.join(map(str, st['tiles']))} "
            f"cell {st['cell_side']} ecs {st['ecs_per_tile']} block_tiles {st['block_tiles']} "
            f"tight {st['tight_factor']}")


def measured_traffic(kernel, st):
    """DRAM bytes per launch of `kernel` on this workload from the committed
    ncu summary, or None unless the summary was taken on this kernel
    revision in exactly this launch setting."""
    import re
    p = os.path.join(ROOT, "profiles", "launches_bench_1e6_melt.md")
    try:
        txt = open(p).read()
    except OSError:
        return None
    k = re.search(r"^setting = (.+)$", txt, re.M)
    b = re.search(r"^dram_bytes_per_launch = ([0-9.eE+]+)$", txt, re.M)
    if not (k and b and k.group(1).strip() == setting_key(kernel, st) and C5.name == "c5_swap_1m"):
        return None
    return float(b.group(1))


def measured_counters(kernel, st):
    """Per-event instruction counts of `kernel` from the committed ncu
    summary (warp instructions, FP64-pipe warp instructions, FP64-pipe
    cycles per FP64 instruction), or None unless it was taken on this
    kernel revision in exactly this launch setting."""
    import re
    p = os.path.join(ROOT, "profiles", "ec_lock_counters_1e6_melt.md")
    try:
        txt = open(p).read()
    except OSError:
        return None
    k = re.search(r"^setting = (.+)$", txt, re.M)
    if not (k and k.group(1).strip() == setting_key(kernel, st) and C5.name == "c5_swap_1m"):
        return None
    out = {}
    for name in ("warp_instr_per_event", "fp64_warp_instr_per_event", "fp64_cycles_per_instr"):
        m = re.search(rf"^{name} = ([0-9.eE+]+)$", txt, re.M)
        if not m:
            return None
        out[name] = float(m.group(1))
    return out


def ceilings(cnt, ec_events_per_s, sm_mhz):
    """Two ceilings of the EC kernel besides HBM: instruction issue (four
    warp instructions per cycle per SM, one per sub-partition) and the SM's
    FP64 pipe (busy fp64_cycles_per_instr SM cycles per FP64 warp
    instruction, the measured ratio of FP64-pipe active cycles to FP64
    instructions: 16 on GB300, i.e. 64 FP64 flops per 16 cycles per SM,
    1.26 TFLOP/s at 2.07 GHz), each divided by the kernel's measured
    per-event counts."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    hz = sm_mhz * 1e6
    issue = 4.0 * sms * hz / cnt["warp_instr_per_event"]
    fp64 = sms * hz / (cnt["fp64_warp_instr_per_event"] * cnt["fp64_cycles_per_instr"])
    return {"issue": {"events_per_s": issue, "frac": ec_events_per_s / issue,
                      "warp_instr_per_event": cnt["warp_instr_per_event"]},
            "fp64_pipe": {"events_per_s": fp64, "frac": ec_events_per_s / fp64,
                          "fp64_warp_instr_per_event": cnt["fp64_warp_instr_per_event"],
                          "fp64_cycles_per_instr": cnt["fp64_cycles_per_instr"]},
            "sms": sms, "sm_mhz": sm_mhz,
            "note": "events/s of the EC launches against each ceiling; the kernel is latency "
                    "bound (dependent FP64 chains, barriers, shared-memory round trips) and "
                    "reaches neither"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index=0):
        self.rows = []
        self.proc = None
        self.index = index

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for k, nm in enumerate(names):
                    if r[4 + k].lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_gpu(args, rank, world):
    import numpy as np
    import torch

    from paper_1502_06447_gb300 import build as b
    from paper_1502_06447_gb300 import ecmc

    if rank == 0 or True:
        b.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    seed = rank_seed(C5.seed, rank)  # replicas: independent seeds

    def configure(ctx, precision, st):
        ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=precision,
                      tiles=st["tiles"], lanes=st["lanes"], ecs_per_tile=st["ecs_per_tile"],
                      cell_side=st["cell_side"], schedule=args.schedule,
                      block_tiles=st["block_tiles"], tight_factor=st["tight_factor"])

    def make(precision):
        ctx = ecmc.Context.create_lattice(C5.dims, C5.spacing, C5.N, sigma=C5.sigma,
                                          b_max=C5.b_max, jitter=C5.jitter, seed=seed)
        ctx.set_stream(stream.cuda_stream)
        st = dict(LAUNCH[precision == ecmc.PREC_FP32F])
        configure(ctx, precision, st)
        # melt the lattice start first: its contacts per sweep fall by a third
        # over the first ~20 sweeps, so tuner trials, the swap calibration
        # and the timed sweeps on the lattice itself would not describe the
        # melt (and its tiles overflow the tight staging capacities)
        ctx.run(ELL, seed=seed, n_sweeps=MELT_SWEEPS)
        tune = ctx.autotune(ELL, seed=seed, trial_sweeps=3) if args.tune else None
        if tune and args.time_tuned:
            st = {"lanes": tune["lanes"], "tiles": tuple(tune["tiles"]),
                  "cell_side": tune["cell_side"], "ecs_per_tile": tune["ecs_per_tile"],
                  "block_tiles": tune["block_tiles"], "tight_factor": tune["tight_factor"]}
        # the timed setting (the pinned one unless --time-tuned); the tuner
        # restored the state, so this is the run that would have followed
        configure(ctx, precision, st)
        # swap calibration under the final setting: one sweep without swaps,
        # then p_swap for 0.1 attempts / bead / sweep
        ctx.run(ELL, seed=seed, n_sweeps=1)
        ctx.swap(SWAP_RATE)
        return ctx, tune, st

    ctx, tune, setting = make(ecmc.PREC_FP32F)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        ctx.run(ELL, seed=seed, n_sweeps=1)
        # re-calibrated on the latest sweep: the contacts per sweep fall while
        # the lattice start melts
        ctx.swap(SWAP_RATE)
    ctx.g1_reset()
    o0 = ctx.observables()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()  # L2 flush between steps (256 MB > 129 MB L2)
            ev[k][0].record(stream)
            ctx.run(ELL, seed=seed, n_sweeps=1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    step_ms = [a.elapsed_time(b_) for a, b_ in ev]
    o1 = ctx.observables()
    events = o1["events_total"] - o0["events_total"]
    ecs = o1["ecs"] - o0["ecs"]
    dev_s = sum(step_ms) / 1e3
    ec_s = o1["ec_kernel_seconds"] - o0["ec_kernel_seconds"]
    confirmed = o1["confirmed"] - o0["confirmed"]
    exhaustive = o1["exhaustive"] - o0["exhaustive"]
    assert o1["overlaps"] == 0 and o1["tether_violations"] == 0
    tried = o1["swap_tried"] - o0["swap_tried"]
    physics = {
        "re2_mean_before": o0["re2_mean"], "re2_mean_after": o1["re2_mean"],
        "g1_over_timed_steps": o1["g1"], "g1_per_device_second": o1["g1"] / dev_s,
        "g1_note": "the launch setting trades events/s against relaxation: more ECs per tile "
                   "(tiles fixed for longer) and smaller tiles (fewer motile beads) raise "
                   "events/s but lower g1 per device-second; measured from one melted start, "
                   "25^3 tiles at 8 ECs per tile reach about 22 % less g1 per device-second "
                   "than at 2, and 22^3 tiles at 2 ECs per tile 15 % more",
        "pressure_contact": o1["pressure_contact"],
        "pressure_lift": {
            "value": 1 + (o1["lift_sum"] - o0["lift_sum"]) / (o1["disp_sum"] - o0["disp_sum"]),
            "valid": False,
            "why": "the lift-distance estimator is exact for serial (undecomposed) ECs only; "
                   "in the domain mode reflections at joint beads and tile walls use up "
                   "displacement without lifting, so it reads low; pressure_contact (contact "
                   "values of the final state) is the estimate"},
        "swap_attempts_per_bead_sweep": tried / C5.n / args.steps,
        "swap_acceptance": (o1["swap"] - o0["swap"]) / tried if tried else None,
        "swap_note": "with tethers of 1.2 sigma an exchange of two touching beads almost always "
                     "over-stretches a bond, so swaps are proposed and timed but change no "
                     "topology here",
        "overlaps": o1["overlaps"], "tether_violations": o1["tether_violations"]}
    extra = args.extra and rank == 0
    structure = structure_run(ctx, stream) if args.extra else None
    init = init_run() if args.extra else None
    precision, prec_state = precision_run(args, stream) if extra else (None, None)
    springs = springs_run(stream, max(3, args.steps // 2)) if extra else None
    systems = ({name: springs_run(stream, max(3, args.steps // 2), name)
                for name in args.systems.split(",") if name and name != "I"}
               if extra and args.systems else None)
    reptation = reptation_run(stream) if extra else None
    fig3 = fig3_run(stream) if extra else None

    # plain FP64 kernel on the same workload (fresh lattice, same calibration)
    ctx64, tune64, setting64 = make(ecmc.PREC_FP64)
    ctx64.run(ELL, seed=seed, n_sweeps=1)
    p0 = ctx64.observables()
    n64 = max(1, args.steps // 2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx64.run(ELL, seed=seed, n_sweeps=n64)
    e1.record(stream)
    torch.cuda.synchronize()
    p1 = ctx64.observables()
    fp64_eps = (p1["events_total"] - p0["events_total"]) / (e0.elapsed_time(e1) / 1e3)
    ctx64.close()

    # e2e through the public API with host buffers
    r_host, img_host = ctx.get_positions()
    r_pin = torch.from_numpy(r_host).pin_memory()
    i_pin = torch.from_numpy(img_host).pin_memory()
    n_e2e = max(1, args.steps)  # as many sweeps as the timed region (sweep times vary)
    q0 = ctx.observables()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    host = (r_pin.numpy(), i_pin.numpy())
    for _ in range(n_e2e):
        ctx.set_positions(*host)  # checked on the device: no overlap, every bond <= b_max
        ctx.run(ELL, seed=seed, n_sweeps=1)
        ctx.get_positions(out=host)
    e2e_s = time.perf_counter() - t0
    q1 = ctx.observables()
    e2e_events = q1["events_total"] - q0["events_total"]

    # aggregate over ranks (replicas; max time, summed events)
    tot_events, max_dev, max_wall = float(events), dev_s, wall
    e2e_tot, e2e_max = float(e2e_events), e2e_s
    if world > 1:
        (tot_events, e2e_tot), (max_dev, max_wall, e2e_max) = reduce_over_ranks(
            [events, e2e_events], [dev_s, wall, e2e_s], dev)
    # the batched form is a single-GPU measurement: rank 0 alone runs it
    batched = run_batch(args, stream) if args.batch and rank == 0 else None
    if rank != 0:
        return None
    hbm, peak_src = load_peaks()
    phi = C5.phi
    bpe = bytes_per_event(phi, confirmed / max(events, 1))
    achieved = events * bpe / ec_s / 1e9
    kname = (f"ec_lock_kernel<{setting['lanes']}, 0>" if args.schedule == 0 and setting["lanes"] in (4, 8, 16)
             else f"ec_kernel<{setting['lanes']}, 1, 0>")
    traffic = measured_traffic(kname, setting)
    counters = measured_counters(kname, setting)
    csum = clk.summary()
    clk_mhz = csum["sm_mhz"] or csum["sm_max_mhz"] or 2070.0
    n_beads = C5.n
    value = tot_events / max_dev
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * max_dev / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": C5.name, "beads": n_beads, "chains": C5.n_chains, "N": C5.N,
                   "lattice": list(C5.dims), "spacing": C5.spacing, "phi": round(phi, 4),
                   "b_max": C5.b_max, "ell": ELL,
                   "tiles": list(setting["tiles"]), "directions": "iso",
                   "precision": "fp32 screen + fp64 confirm", "swap_attempts_per_bead_sweep":
                   SWAP_RATE, "lanes_per_ec": setting["lanes"],
                   "ecs_per_tile": setting["ecs_per_tile"], "cell_side": setting["cell_side"],
                   "block_tiles": setting["block_tiles"], "tight_factor": setting["tight_factor"],
                   "tuning": ("the autotuner's pick of this run" if args.time_tuned and tune else
                              "pinned launch setting (the autotuner's pick on a GB300, "
                              "configs.C5_LAUNCH); this run's pick under tuning.fp32f"),
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "ell_sweeps_per_s": (ecs / n_beads) / dev_s,
        "ecs_per_s": ecs / dev_s,
        "fp64_events_per_s": fp64_eps,
        "fp32f_over_fp64": value / fp64_eps / world,
        "confirmed_per_event": confirmed / max(events, 1),
        "exhaustive_per_event": exhaustive / max(events, 1),
        "events_per_ec": events / max(ecs, 1),
        "wall_s": max_wall,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "ceilings": (ceilings(counters, events / ec_s, clk_mhz) if counters else None),
                     "kernel": kname,
                     "bytes_per_event": bpe,
                     "kernel_share_of_step": ec_s / dev_s, "peak_source": peak_src},
        "e2e": {"value": e2e_tot / e2e_max, "unit": UNIT, "steps": n_e2e,
                "ms_per_step": 1e3 * e2e_max / n_e2e, "events": e2e_tot,
                "h2d_bytes_per_step": int(r_host.nbytes + img_host.nbytes),
                "d2h_bytes_per_step": int(r_host.nbytes + img_host.nbytes)},
        # per sweep: 5 cell-list kernels + the EC launch (two passes for the
        # block-lockstep kernel: tight capacities, then deferred tiles)
        "gpu_launches": (7 if kname.startswith("ec_lock") else 6) * args.steps,
        "physics": physics,
        "structure": structure,
        "init": init,
        "clocks": csum,
        "tuning": {"fp32f": tune, "fp64": tune64, "fp64_timed_setting": setting64},
    }
    if batched is not None:
        line["batched"] = batched
    if precision is not None:
        line["precision"] = precision
    if springs is not None:
        line["springs"] = springs
    if systems:
        line["springs_systems"] = systems
    if reptation is not None:
        line["reptation"] = reptation
    if fig3 is not None:
        line["init_fig3"] = fig3
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_run(steps=2)
        line["cpu_baseline"]["all_cores"] = cpu_allcore_run(sweeps=1)
        if prec_state is not None:
            line["precision"].update(precision_vs_oracle(prec_state))
    return line


def run_batch(args, stream):
    """256 replicas (N in {10..160}, 2k-64k beads, phi in [0.35, 0.50],
    ell = 5): aggregate throughput of the graph-captured batched sweep, the
    same replicas one at a time through the single-melt API, and the batched
    plain FP64 kernel.  Device time from the library's CUDA events on its
    stream; the batch state (~0.5 GB) exceeds L2, so no flush."""
    import torch

    from paper_1502_06447_gb300 import ecmc
    from paper_1502_06447_gb300.configs import replica_specs
    ms = replica_specs()
    specs = [dict(dims=m.dims, spacing=m.spacing, N=m.N) for m in ms]
    ell, seed, jitter = ms[0].ell, ms[0].seed, ms[0].jitter
    beads = sum(m.n for m in ms)
    ksteps = max(3, args.steps // 2)
    res = {"workload": f"{len(ms)} replicas, N in {{10..160}}, {min(m.n for m in ms)}-"
                       f"{max(m.n for m in ms)} beads each, phi in [0.35, 0.50], ell = {ell}",
           "replicas": len(ms), "beads": beads, "steps": ksteps,
           "l2": "state larger than L2 (no flush)"}
    for name, prec, lanes in (("fp32f", ecmc.PREC_FP32F, 8), ("fp64", ecmc.PREC_FP64, 16)):
        b = ecmc.Batch(specs, jitter=jitter, seed=seed)
        b.configure(dir_mode=ecmc.DIR_ISO, precision=prec, lanes=lanes)
        b.run(ell, seed=seed, n_sweeps=3, graph=False)  # melt the lattice start first
        tune = b.autotune(ell, seed=seed, trial_sweeps=3)
        b.run(ell, seed=seed, n_sweeps=max(1, args.warmup), graph=True)
        s0 = b.stats()
        b.run(ell, seed=seed, n_sweeps=ksteps, graph=True)
        s1 = b.stats()
        dt = s1["device_seconds"] - s0["device_seconds"]
        ev = s1["events_total"] - s0["events_total"]
        ecs = s1["ecs"] - s0["ecs"]
        res[name] = {"events_per_s": ev / dt, "ecs_per_s": ecs / dt,
                     "ell_sweeps_per_s": ecs / beads / dt, "ms_per_sweep": 1e3 * dt / ksteps,
                     "tuning": tune}
        if name == "fp32f":
            tiles = [b.info(r)[0] for r in range(len(ms))]
        b.close()
    res["fp32f_over_fp64"] = res["fp32f"]["events_per_s"] / res["fp64"]["events_per_s"]
    # the same replicas one at a time (one launch sequence and one host
    # round trip per replica per sweep), same tuned setting
    t = res["fp32f"]["tuning"]
    ctxs = []
    for m, d in zip(ms, tiles):
        c = ecmc.Context.create_lattice(m.dims, m.spacing, m.N, jitter=jitter, seed=seed)
        c.set_stream(stream.cuda_stream)
        c.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP32F,
                    tiles=d, lanes=t["lanes"], cell_side=t["cell_side"],
                    ecs_per_tile=t["ecs_per_tile"])
        c.run(ell, seed=seed, n_sweeps=3 + max(1, args.warmup))  # as melted as the batch
        ctxs.append(c)
    nseq = max(1, ksteps // 3)
    o0 = [c.observables()["events_total"] for c in ctxs]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(nseq):
        for c in ctxs:
            c.run(ell, seed=seed, n_sweeps=1)
    e1.record(stream)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3
    ev = sum(c.observables()["events_total"] - a for c, a in zip(ctxs, o0))
    for c in ctxs:
        c.close()
    res["sequential"] = {"events_per_s": ev / dt, "ms_per_sweep": 1e3 * dt / nseq,
                         "steps": nseq}
    res["batched_over_sequential"] = res["fp32f"]["events_per_s"] / res["sequential"]["events_per_s"]
    return res


def precision_run(args, stream, sweeps=5):
    """The precision form on the 512k-bead melt at phi = 0.50 (2000 chains x
    N = 256 on an 80^3 lattice, spacing 1.0156, ell = 10, 16^3 tiles): the
    FP32-screened kernel and the plain FP64 kernel from the same lattice and
    seed, `sweeps` sweeps each with per-EC digests.  Reports whether every
    EC's event digest is the same in both, the largest position difference
    between them, and both kernels' events/s (CUDA events on the launching
    stream).  The sweep-1 state of the screened run is kept for the oracle
    check of the CPU leg."""
    import numpy as np
    import torch

    from paper_1502_06447_gb300 import ecmc
    m = C3
    nt = m.D[0] * m.D[1] * m.D[2]
    out = {}
    for name, prec, lanes in (("fp32f", ecmc.PREC_FP32F, 8), ("fp64", ecmc.PREC_FP64, 16)):
        ctx = ecmc.Context.create_lattice(m.dims, m.spacing, m.N, sigma=m.sigma, b_max=m.b_max,
                                          jitter=m.jitter, seed=m.seed)
        ctx.set_stream(stream.cuda_stream)
        ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=prec, tiles=m.D,
                      lanes=lanes, record=1)
        ctx.run(m.ell, seed=m.seed, n_sweeps=1)
        d1, _, _ = ctx.records(nt)
        r1, i1 = ctx.get_positions()
        o0 = ctx.observables()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.run(m.ell, seed=m.seed, n_sweeps=sweeps - 1)
        b.record(stream)
        torch.cuda.synchronize()
        dk, _, _ = ctx.records(nt * (sweeps - 1))
        rk, ik = ctx.get_positions()
        o1 = ctx.observables()
        ev = o1["events_total"] - o0["events_total"]
        out[name] = {"digests": np.concatenate([d1, dk]), "r1": r1, "i1": i1, "rk": rk,
                     "events": o1["events_total"], "overlaps": o1["overlaps"],
                     "tether_violations": o1["tether_violations"],
                     "events_per_s": ev / (a.elapsed_time(b) / 1e3),
                     "confirmed_per_event": (o1["confirmed"] - o0["confirmed"]) / max(ev, 1)}
        ctx.close()
    f, g = out["fp32f"], out["fp64"]
    L = np.array(m.L)
    d = f["rk"] - g["rk"]
    d -= L * np.round(d / L)
    res = {"workload": m.name, "beads": m.n, "phi": round(m.phi, 4), "ell": m.ell,
           "tiles": list(m.D), "sweeps": sweeps, "ecs": int(len(f["digests"])),
           "events": int(f["events"]),
           "events_identical": bool(len(f["digests"]) == len(g["digests"]) and
                                    (f["digests"] == g["digests"]).all()),
           "max_dr_vs_fp64": float(np.abs(d).max()),
           "overlaps": int(f["overlaps"]), "tether_violations": int(f["tether_violations"]),
           "fp32f_events_per_s": f["events_per_s"], "fp64_events_per_s": g["events_per_s"],
           "fp32f_over_fp64": f["events_per_s"] / g["events_per_s"],
           "confirmed_per_event": f["confirmed_per_event"],
           "note": "FP32 screen (block-lockstep kernel, 8 lanes) vs plain FP64 kernel (16 lanes), "
                   "same lattice and seed; digests are 64-bit FNV-1a over every event of an EC"}
    state = {"r1": f["r1"], "i1": f["i1"], "d1": f["digests"][:nt]}
    return res, state


def precision_vs_oracle(state):
    """CPU-leg check of the precision form: the oracle runs the first sweep
    of the same 512k-bead melt; its per-EC digests and final positions are
    compared with the screened GPU run's sweep 1 (outside any timed region)."""
    import numpy as np

    import oracle
    m = C3
    o = oracle.System(oracle.lattice(m.dims, m.spacing, m.jitter, m.seed), m.L, m.N,
                      mode=oracle.MODE_DOMAIN, dir_mode=oracle.DIR_ISO, D=m.D, seed=m.seed)
    t0 = time.perf_counter()
    res = o.run_domain(1, m.ell, digests=True)
    dt = time.perf_counter() - t0
    L = np.array(m.L)
    d = state["r1"] - o.r
    d -= L * np.round(d / L)
    return {"oracle_sweeps": 1, "oracle_s": dt,
            "events_identical_vs_oracle": bool((res["digest"] == state["d1"]).all()),
            "images_identical_vs_oracle": bool((state["i1"] == o.img).all()),
            "max_dr_vs_oracle": float(np.abs(d).max())}


# the paper's System I (Sec. IV.A): M = 400 bead-spring chains of N = 120 at
# packing fraction 0.390 in a 40^3 box, k = 30 kT/sigma^2, built as the paper
# builds its melts (phantom chains, c = 1.9, pushed off with tethers)
SPRINGS = dict(L=40.0, n_chains=400, N=120, c=1.9, seed=61, po_seed=0xEC1F0F, k=30.0, ell=10.0,
               tiles=(9, 9, 9), ecs_per_tile=4, max_sweeps=40000)
# the paper's Systems I-III (M chains of N beads in a 40^3 box, k = 30):
# eta = 0.390, 0.490, 0.490
SYSTEMS = {"I": dict(n_chains=400, N=120), "II": dict(n_chains=500, N=120),
           "III": dict(n_chains=250, N=240)}


def springs_run(stream, steps, system="I"):
    """Bead-spring melt of the paper's System I (or II, III) size through
    the public API: phantom chains and slow push-off with the springs acting
    (outside the timed region), then EC sweeps with harmonic bonds,
    FP32-screened and plain FP64, each timed with CUDA events on the
    launching stream."""
    import torch

    from paper_1502_06447_gb300 import ecmc
    c = dict(SPRINGS, **SYSTEMS[system])
    L = (c["L"],) * 3
    eta = c["n_chains"] * c["N"] * math.pi / 6.0 / c["L"] ** 3
    res = {"workload": f"System {system} size: {c['n_chains']} chains x N = {c['N']}, "
                       f"eta = {eta:.3f}, 40^3 box, k = 30 kT/sigma^2",
           "beads": c["n_chains"] * c["N"], "ell": c["ell"], "tiles": list(c["tiles"]),
           "ecs_per_tile": c["ecs_per_tile"], "steps": steps}
    ctx = ecmc.Context.create_phantom(L, c["n_chains"], c["N"], bond=1.0, c=c["c"], seed=c["seed"])
    ctx.set_stream(stream.cuda_stream)
    # the push-off with the springs acting (the paper builds its spring melts
    # this way)
    ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP64,
                  tiles=c["tiles"], lanes=PO_LANES, k_spring=c["k"])
    t0 = time.perf_counter()
    res["pushoff_sweeps"] = ctx.pushoff(f0=0.5, stages=5, ell=2.0, seed=c["po_seed"],
                                        max_sweeps=c["max_sweeps"])
    res["pushoff_s"] = time.perf_counter() - t0
    r0, i0 = ctx.get_positions()
    for name, prec, lanes in (("fp32f", ecmc.PREC_FP32F, 8), ("fp64", ecmc.PREC_FP64, 16)):
        ctx.set_positions(r0, i0)
        ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=prec,
                      tiles=c["tiles"], lanes=lanes, ecs_per_tile=c["ecs_per_tile"], k_spring=c["k"])
        ctx.run(c["ell"], seed=c["seed"], n_sweeps=3)
        o0 = ctx.observables()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.run(c["ell"], seed=c["seed"], n_sweeps=steps)
        b.record(stream)
        torch.cuda.synchronize()
        o1 = ctx.observables()
        dt = a.elapsed_time(b) / 1e3
        ev = o1["events_total"] - o0["events_total"]
        res[name] = {"events_per_s": ev / dt, "ecs_per_s": (o1["ecs"] - o0["ecs"]) / dt,
                     "ms_per_sweep": 1e3 * dt / steps, "bond_mean": o1["bond_mean"],
                     "bond_max": o1["bond_max"], "overlaps": o1["overlaps"],
                     "spring_events_share": (o1["te_lift"] + o1["te_reflect"]
                                             - o0["te_lift"] - o0["te_reflect"]) / max(ev, 1)}
    res["fp32f_over_fp64"] = res["fp32f"]["events_per_s"] / res["fp64"]["events_per_s"]
    res["note"] = ("<b> is the mean bond length of the final state; the paper quotes <b> ~ 1.1 sigma "
                   "for k = 30; the free-bond law of the oracle pin gives 1.168 sigma")
    ctx.close()
    return res


# the paper's reptation melt (Sec. IV.B, Fig. 6): M = 20 chains of N = 500
# with tethers of 1.4 sigma at packing fraction 0.298, from phantom chains
# and the slow push-off; g1 of the middle beads over log-spaced lags
REPTATION = dict(M=20, N=500, eta=0.298, b_max=1.4, seed=71, po_seed=72, run_seed=73, ell=10.0,
                 tiles=(6, 6, 6), ecs_per_tile=2, P=4, K=8, sweeps=8192, max_s=25.0)


def reptation_run(stream):
    """Push-off (wall time), then sweeps of the FP32-screened kernel with the
    device-side g1 table until `sweeps` sweeps or about `max_s` seconds;
    reports the table and the slope of log g1 against log lag over the
    longest decade of lags that have at least 8 origins."""
    import numpy as np
    import torch

    from paper_1502_06447_gb300 import ecmc
    c = REPTATION
    L = (c["M"] * c["N"] * math.pi / (6.0 * c["eta"])) ** (1.0 / 3.0)
    ctx = ecmc.Context.create_phantom((L, L, L), c["M"], c["N"], bond=1.0, c=1.9, seed=c["seed"],
                                      b_max=c["b_max"])
    ctx.set_stream(stream.cuda_stream)
    ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP64,
                  tiles=c["tiles"], lanes=PO_LANES)
    t0 = time.perf_counter()
    po_sweeps = ctx.pushoff(f0=0.5, stages=5, ell=2.0, seed=c["po_seed"], max_sweeps=20000)
    po_s = time.perf_counter() - t0
    ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP32F,
                  tiles=c["tiles"], lanes=8, ecs_per_tile=c["ecs_per_tile"])
    ctx.g1_track(c["P"], c["K"])
    o0 = ctx.observables()
    done, chunk = 0, 256
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    t1 = time.perf_counter()
    while done < c["sweeps"] and time.perf_counter() - t1 < c["max_s"]:
        ctx.run(c["ell"], seed=c["run_seed"], n_sweeps=chunk)
        done += chunk
        torch.cuda.synchronize()
    b.record(stream)
    torch.cuda.synchronize()
    dt = a.elapsed_time(b) / 1e3
    o1 = ctx.observables()
    lags, g1, cnt = ctx.g1_table()
    ok = (cnt >= 8) & (g1 > 0)
    fit = None
    if ok.sum() >= 3:
        x, y = np.log(lags[ok]), np.log(g1[ok])
        sel = x >= x.max() - math.log(10.0)
        if sel.sum() >= 2:
            fit = float(np.polyfit(x[sel], y[sel], 1)[0])
    ctx.close()
    return {"workload": "reptation melt: 20 chains x N = 500, eta = 0.298, tethers b_max = 1.4, "
                        "phantom chains + push-off",
            "box": L, "pushoff_sweeps": po_sweeps, "pushoff_s": po_s, "sweeps": done,
            "events_per_s": (o1["events_total"] - o0["events_total"]) / dt,
            "ms_per_sweep": 1e3 * dt / max(done, 1),
            "g1_table": {"lag_sweeps": [int(v) for v in lags[cnt > 0]],
                         "g1": [float(v) for v in g1[cnt > 0]],
                         "origins": [int(v) for v in cnt[cnt > 0]]},
            "g1_exponent_last_decade": fit,
            "paper": "g1 ~ t^0.3 in the reptation regime (Fig. 6), reached there after much longer "
                     "runs; this run covers the time the budget allows",
            "overlaps": o1["overlaps"], "tether_violations": o1["tether_violations"]}


def structure_run(ctx, stream):
    """The chain-structure pass (ecmc_structure) on the melt's final state:
    its device time with and without R^2(n) (CUDA events on the library's
    stream, after one untimed call) and what it measures.  g2 is over the
    timed sweeps (the reference is taken before them)."""
    import torch

    def timed(r2n, reps=5):
        ctx.structure(dR=2.0, nbins=64, r2n=r2n)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            out = ctx.structure(dR=2.0, nbins=64, r2n=r2n)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps, out
    ms0, _ = timed(False)
    ms1, (got, rn, hist) = timed(True)
    nch, N = got["n_chains"], got["N"]
    pairs = nch * N * (N - 1) / 2
    T = got["rg2_sum"] / nch
    return {"ms": ms1, "ms_without_r2n": ms0, "chains": nch, "N": N,
            "r2n_fp64_gflops": 9.0 * pairs / ((ms1 - ms0) * 1e-3) / 1e9 if ms1 > ms0 else None,
            "rg2_mean": T, "re2_mean": got["re2_sum"] / nch,
            "lam_fractions": [x / got["rg2_sum"] for x in got["lam_sum"]],
            "kappa2_mean": got["kappa2_sum"] / nch,
            "bc_over_trI2": got["bc_sum"] / nch / (4.0 * T * T),
            "g2_over_timed_steps": got["g2_sum"] / nch,
            "r2n_over_n": {str(n): float(rn[n] / n) for n in (1, 10, 100, N - 1) if n < N},
            "note": "lam_fractions = <-I1+I2+I3>, <I1-I2+I3>, <I1+I2-I3> over <Tr I> (inertia "
                    "tensor eigenvalues in descending order); ideal chains give 0.0646, 0.175, "
                    "0.754 and bc_over_trI2 = 2/3"}


# initial configuration measured beside the EC sweeps: phantom chains of 20
# beads (c = 1.9) at packing fraction 0.35, pushed off in 5 stages from half
# the diameter (ECs of length 2, 3^3 tiles), as the paper builds its melts
INIT = dict(L=20.0, n_chains=267, N=20, c=1.9, seed=51, po_seed=0xEC0F0F, f0=0.5, stages=5,
            ell=2.0, tiles=(4, 4, 4), max_sweeps=6000)


def init_run():
    """Phantom chains and the slow push-off through the public API (each
    call synchronises; wall time)."""
    from paper_1502_06447_gb300 import ecmc

    c = INIT
    L = (c["L"],) * 3
    t0 = time.perf_counter()
    ctx = ecmc.Context.create_phantom(L, c["n_chains"], c["N"], bond=1.0, c=c["c"], seed=c["seed"])
    t1 = time.perf_counter()
    ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP64,
                  tiles=c["tiles"], lanes=PO_LANES)
    t2 = time.perf_counter()
    sweeps = ctx.pushoff(f0=c["f0"], stages=c["stages"], ell=c["ell"], seed=c["po_seed"],
                         max_sweeps=c["max_sweeps"])
    t3 = time.perf_counter()
    got, rn, _ = ctx.structure(r2n=True)
    o = ctx.observables()
    n = c["n_chains"] * c["N"]
    return {"beads": n, "eta": n * math.pi / 6 / c["L"] ** 3, "phantom_ms": 1e3 * (t1 - t0),
            "pushoff_ms": 1e3 * (t3 - t2), "pushoff_sweeps": sweeps,
            "overlaps": o["overlaps"], "tether_violations": o["tether_violations"],
            "r2n_over_n": {str(k): float(rn[k] / k) for k in (1, 5, 19)},
            "setting": "267 chains x 20 beads, c = 1.9, 20^3 box, 4^3 tiles, f0 = 0.5, 5 stages, "
                       "ECs of length 2, plain FP64 kernel, 32 lanes per tile"}


ORC_PARTS = 8  # one-core oracle samples run the tiles t % 8 == 0 of each sweep


def oracle_c5(r, img=None, p_swap=0.0, parts=ORC_PARTS, rem=0):
    """The oracle on the 10^6-bead melt in the timed launch's tiling (the
    pinned tiles and ECs per tile), running the tiles t % parts == rem of
    each sweep (tiles are independent within a sweep: a part does exactly
    the serial sweep's work on those tiles)."""
    import oracle
    st = launch_settings_default()
    return oracle.System(r, C5.L, C5.N, mode=oracle.MODE_DOMAIN, dir_mode=oracle.DIR_ISO,
                         D=tuple(st["tiles"]), seed=C5.seed, img=img, p_swap=p_swap,
                         ecs_per_tile=st["ecs_per_tile"], tile_mod=parts, tile_rem=rem)


def launch_settings_default():
    """The timed screened setting of this workload without command-line
    overrides (the pinned one for the 1e6-bead melt)."""
    st = dict(C5_LAUNCH)
    if C5.name != "c5_swap_1m":
        st.update(tiles=TILES, ecs_per_tile=1, cell_side=1.05)
    return st


def oracle_rate(steps, warmup):
    """Events/s of the oracle as it stands (serial FP64 C, one core) on
    bounded samples of the timed workload: from the lattice start, warm-up
    sweeps with swaps off (the last one calibrates p_swap for 0.1 attempts
    per bead per sweep from its contacts, as ecmc_swap does), then `steps`
    timed sweeps with swaps, each running 1/8 of the tiles (a new random
    shift every sweep).  Returns (events/s, events, seconds, p_swap)."""
    r = oracle_lattice_c5()
    o = oracle_c5(r)
    sweep = 0
    res = None
    for _ in range(max(int(warmup), 1)):
        res = o.run_domain(1, ELL, sweep0=sweep)
        sweep += 1
    contacts = res["stats"]["hs_lift"] + res["stats"]["swap"]
    p = min(1.0, SWAP_RATE * (C5.n / ORC_PARTS) / contacts) if contacts else 0.0
    o = oracle_c5(o.r, img=o.img, p_swap=p)
    t0 = time.perf_counter()
    ev = 0
    for _ in range(int(steps)):
        res = o.run_domain(1, ELL, sweep0=sweep)
        ev += res["stats"]["events"]
        sweep += 1
    dt = time.perf_counter() - t0
    return ev / dt, ev, dt, p


def oracle_lattice_c5():
    import oracle
    return oracle.lattice(C5.dims, C5.spacing, C5.jitter, C5.seed)


def _oracle_part(k, parts, sweeps):
    """One process of the all-core oracle timing: tiles t % parts == k of
    `sweeps` sweeps of the 1e6-bead melt (timed tiling, swaps off); returns
    (events, seconds)."""
    o = oracle_c5(oracle_lattice_c5(), parts=parts, rem=k)
    t0 = time.perf_counter()
    res = o.run_domain(sweeps, ELL)
    return res["stats"]["events"], time.perf_counter() - t0


def cpu_allcore_run(sweeps=1):
    """The oracle on every host core: the tiles of a sweep split over one
    process per core (tiles are independent within a sweep, so the parts do
    exactly the serial sweep's work); events/s = all events / the slowest
    part's run time (process start-up and state building excluded)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    parts = os.cpu_count() or 1
    with cf.ProcessPoolExecutor(max_workers=parts, mp_context=mp.get_context("spawn")) as ex:
        out = list(ex.map(_oracle_part, range(parts), [parts] * parts, [sweeps] * parts))
    ev = sum(e for e, _ in out)
    dt = max(t for _, t in out)
    return {"value": ev / dt, "unit": UNIT, "cores": parts, "kind": "oracle",
            "sample": f"{sweeps} sweep(s) of the 1e6-bead melt in the timed tiling without swaps, "
                      f"its tiles split over {parts} processes ({ev} events, slowest part "
                      f"{dt:.1f} s)"}


# the paper's Fig. 3 initial configuration (Sec. II.B): M = 500 phantom
# chains of N = 121 (c = 1.9, bonds of sigma) at packing fraction 0.495 in a
# 40^3 box, pushed off with ECs of length 2 sigma
FIG3 = dict(L=40.0, n_chains=500, N=121, c=1.9, seed=81, po_seed=0xEC3F03, f0=0.5, stages=10,
            ell=2.0, tiles=(9, 9, 9), max_sweeps=40000, k=30.0)


def fig3_run(stream):
    """Phantom chains and slow push-off of the Fig. 3 melt through the
    public API, with the paper's bead springs (k = 30 kT/sigma^2): R^2(n)/n
    of the phantom chains and after the push-off (the paper's figure), the
    sweeps and wall time, the mean bond, and the overlaps left if a stage
    does not finish within max_sweeps (ECMC_ESTUCK)."""
    from paper_1502_06447_gb300 import ecmc
    c = FIG3
    L = (c["L"],) * 3
    ctx = ecmc.Context.create_phantom(L, c["n_chains"], c["N"], bond=1.0, c=c["c"], seed=c["seed"])
    ctx.set_stream(stream.cuda_stream)
    n = c["n_chains"] * c["N"]
    _, rn0, _ = ctx.structure(r2n=True)
    ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP64,
                  tiles=c["tiles"], lanes=PO_LANES, k_spring=c["k"])
    t0 = time.perf_counter()
    res = {"workload": "Fig. 3 melt: 500 phantom chains x N = 121, eta = 0.495, 40^3 box, "
                       "bead springs k = 30, push-off in 10 stages from half the diameter, "
                       "ECs of length 2",
           "beads": n, "eta": n * math.pi / 6 / c["L"] ** 3}
    try:
        res["pushoff_sweeps"] = ctx.pushoff(f0=c["f0"], stages=c["stages"], ell=c["ell"],
                                            seed=c["po_seed"], max_sweeps=c["max_sweeps"])
        res["finished"] = True
    except ecmc.EcmcError as e:
        res["finished"] = False
        res["stuck"] = str(e)
    res["pushoff_s"] = time.perf_counter() - t0
    _, rn1, _ = ctx.structure(r2n=True)
    pick = (1, 5, 10, 30, 60, 120)
    res["r2n_over_n_phantom"] = {str(k): float(rn0[k] / k) for k in pick}
    res["r2n_over_n_pushed_off"] = {str(k): float(rn1[k] / k) for k in pick}
    o = ctx.observables()
    res["overlaps_left"] = o["overlaps"]
    res["bond_mean"] = o["bond_mean"]
    res["paper"] = "a couple of minutes of wall time for these parameters (Sec. II.B)"
    ctx.close()
    return res


def cpu_baseline_run(steps=2):
    """The oracle as it stands (serial FP64 C, one core) on a bounded sample
    of the timed workload (oracle_rate: one warm-up sweep, `steps` timed
    sweeps of 1/8 of the tiles each), then the structure pass and the
    init leg's push-off."""
    import oracle
    v, ev, dt, p = oracle_rate(steps, 1)
    o = oracle.System(oracle_lattice_c5(), C5.L, C5.N, mode=oracle.MODE_DOMAIN,
                      dir_mode=oracle.DIR_ISO, D=TILES, seed=C5.seed)
    t1 = time.perf_counter()
    o.chain_struct(dR=2.0, nbins=64)
    ds = time.perf_counter() - t1
    c = INIT
    L = (c["L"],) * 3
    t2 = time.perf_counter()
    rp, ip = oracle.phantom_chains(L, c["n_chains"], c["N"], bond=1.0, c=c["c"], seed=c["seed"])
    po = oracle.System(rp, L, c["N"], sigma=1.0, b_max=1.2, mode=oracle.MODE_DOMAIN,
                       dir_mode=oracle.DIR_ISO, D=c["tiles"], seed=c["po_seed"], img=ip)
    rc, po_sweeps, _ = po.pushoff(c["f0"], c["stages"], c["ell"], c["max_sweeps"])
    dp = time.perf_counter() - t2
    return {"value": v, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{steps} sweep(s) of 1/{ORC_PARTS} of the 1e6-bead melt's tiles in the "
                      f"timed tiling, swaps at p_swap = {p:.4g} ({ev} events, {dt:.1f} s)",
            "structure_ms": 1e3 * ds,
            "structure_sample": "one chain-structure pass (gyration tensors, R^2(n), W(R)) "
                                "over the same melt",
            "init_ms": 1e3 * dp, "init_sweeps": po_sweeps, "init_rc": rc,
            "init_sample": "the phantom chains and push-off of the JSON line's init setting"}


def run_reference(args, rank):
    """The reference arm: the oracle as it stands, on one host core, on
    bounded samples of the timed workload (oracle_rate)."""
    if rank != 0:
        return None
    import oracle
    oracle.build()
    v, ev, dt, p = oracle_rate(args.steps, args.warmup)
    st = launch_settings_default()
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": C5.name, "tiles": list(st["tiles"]), "ell": ELL,
                       "ecs_per_tile": st["ecs_per_tile"], "p_swap": p,
                       "sample": f"each step 1/{ORC_PARTS} of the tiles of a sweep, one core"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} sweep(s) of 1/{ORC_PARTS} of the "
                                       f"1e6-bead melt's tiles ({ev} events)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lanes", type=int, default=0,
                    help="lanes per EC, screened kernel (0: the pinned setting)")
    ap.add_argument("--lanes64", type=int, default=0,
                    help="lanes per EC, plain FP64 kernel (0: the pinned setting)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--workload", default="c5", choices=sorted(WORKLOADS),
                    help="c5: the 1e6-bead melt (default); c2/c3: smaller melts")
    ap.add_argument("--tiles", type=int, default=0, help="tiles per axis (0: workload default)")
    ap.add_argument("--ecs-per-tile", type=int, default=0, help="0: the pinned setting")
    ap.add_argument("--schedule", type=int, default=0,
                    help="screened kernel: 0 block lockstep, 1 warp lockstep")
    ap.add_argument("--block-tiles", type=int, default=-1,
                    help="block lockstep: tiles per block (-1: the pinned setting, 0: occupancy)")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="skip the autotuner (the timed setting is the pinned one anyway)")
    ap.add_argument("--time-tuned", action="store_true",
                    help="time the autotuner's pick of this run instead of the pinned setting")
    ap.add_argument("--no-batch", dest="batch", action="store_false",
                    help="skip the batched-replicas measurement")
    ap.add_argument("--systems", default="",
                    help="also run the paper's Systems II, III (comma list, e.g. II,III)")
    ap.add_argument("--no-extra", dest="extra", action="store_false",
                    help="skip the legs beside the headline melt (structure, initial "
                         "configurations, precision form, springs, reptation)")
    args = ap.parse_args()
    global C5, ELL, TILES, LAUNCH
    C5, TILES = WORKLOADS[args.workload]
    if args.tiles:
        TILES = (args.tiles,) * 3
    LAUNCH = launch_settings(args)
    ELL = C5.ell
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        line = run_reference(args, rank)
        if line:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    if world > 1 or rank != 0:
        args.cpu_baseline = args.cpu_baseline and rank == 0 and world == 1
    line = run_gpu(args, rank, world)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
