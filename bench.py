"""Throughput benchmark of the TVLBM sweep: MLUPS and fraction of the HBM roofline.

Default workload (one GPU): 1024 x 1024 periodic D2Q16, FP32 populations, tau = 0.7,
T = 1 + 0.05 Gaussian bump (sigma 64 cells), seeded random Fourier flow (|k| <= 8, 0.02).
One bench step = the workload's full run of 1000 time steps (each time step is one fused
stream+collide sweep over the grid).  Inputs are resident in HBM when a timed step starts; the
L2 is flushed (a 512 MiB write) between timed steps, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c1|c1_4096|c0|c2|c2_bf16|c3|c4|fv] [--form tiled|flow|plain]
                  [--no-cpu-baseline] [--no-extras]

Prints one JSON line.  With the default workload the line also carries sub-records of the other
configurations (4096^2 FP32, the 4096x512 channel in FP16 and BF16 deviations, the 256-domain
batch), each timed on its own with its oracle check.  --impl reference times the FP64 CPU oracle
on this machine's host cores on the same workload (each step a bounded sample of the time steps).  Under torchrun
(N > 1) every rank advances its own replica of the workload (no data exchange) and the line
reports the aggregate.
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
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

WORKLOADS = {
    # storage: the shipped (chosen) form; plain_storage: the plain form's storage
    "c1": dict(desc="D2Q16 1024x1024 periodic FP32 populations tau=0.7, Gaussian T bump + random Fourier flow, "
                    "1000 time steps", nx=1024, ny=1024, velset="D2Q16", storage="fp32_dev", plain_storage="fp32",
               tau=0.7, walls=None, tsteps=1000),
    "c1_4096": dict(desc="D2Q16 4096x4096 periodic FP32 populations tau=0.7 (C1 recipe, sigma 256), 100 time steps",
                    nx=4096, ny=4096, velset="D2Q16", storage="fp32_dev", plain_storage="fp32", tau=0.7, walls=None,
                    tsteps=100),
    "c0": dict(desc="D2Q16 64x64 periodic FP64 tau=0.8 shear wave, 200 time steps",
               nx=64, ny=64, velset="D2Q16", storage="fp64", plain_storage="fp64", tau=0.8, walls=None, tsteps=200,
               note="1 MB of state, resident in L2: its time per step is FP64 arithmetic on 4096 cells (GB300's "
                    "FP64 rate is a small fraction of its FP32 rate) and launch latency, so its HBM roofline "
                    "fraction is not meaningful"),
    "c2": dict(desc="D2Q36 4096x512 thermal Couette FP16-deviation storage tau=0.9, walls T=1.0/1.1, u_top=0.1, "
                    "1000 time steps", nx=4096, ny=512, velset="D2Q36", storage="fp16_dev", plain_storage="fp16_dev",
               tau=0.9, walls=(0.0, 1.0, 0.1, 1.1), tsteps=1000, reference="rows", refresh=100, ref_kind="mean"),
    "c2_bf16": dict(desc="D2Q36 4096x512 thermal Couette BF16-deviation storage tau=0.9, walls T=1.0/1.1, "
                         "u_top=0.1, 1000 time steps", nx=4096, ny=512, velset="D2Q36", storage="bf16_dev",
                    plain_storage="bf16_dev", tau=0.9, walls=(0.0, 1.0, 0.1, 1.1), tsteps=1000, reference="rows",
                    refresh=40, ref_kind="mean"),
}

# configurations measured beside the default line (their own sub-records in the JSON line)
EXTRA = ("c1_4096", "c2", "c2_bf16", "c3", "c0")

BATCH = dict(desc="256 independent periodic D2Q16 domains, sides drawn from {128,256,512,768,1024}, tau~U[0.55,1.5], "
                   "Mach~U[0.05,0.3], seeded fields, FP32 populations; the bench step's 20 time steps as one "
                   "persistent dataflow launch or 20 launches over all tiles (autotuned with the tile shape), "
                   "CUDA-graph replay",
             count=256, seed=3, velset="D2Q16", storage="fp32_dev", tsteps=20)

CLOSURE = dict(desc="learned closure: D2Q16 256x256 periodic coarse run with the 54-128-128-12 GELU network "
                    "(BF16 tcgen05 kernels, FP32 accumulate), trained on 1024x1024 runs (tau=0.8) downsampled 4x "
                    "from C3-style seeded fields (random Fourier flow |k| <= 32, Mach U[0.05,0.3]); 32 coarse steps "
                    "(= 128 fine steps) per bench step; MLUPS counted as fine-grid cell updates represented", nf=1024, m=4, coarse_steps=32)

METRIC = "MLUPS (million lattice-cell updates per second) of the fused TVLBM sweep"
UNIT = "MLUPS"


def fields_for(name, w, nx=None):
    nx, ny = nx or w["nx"], w["ny"]
    if name.startswith("c1"):
        return workloads.gaussian_bump_random_flow(nx, ny, seed=1, sigma=64.0 * nx / 1024)
    if name == "c0":
        return workloads.shear_wave(nx, ny, eps=0.01)
    return workloads.couette_linear(nx, ny, 1.0, 1.1)


def field_errors(got, want):
    """Max relative errors of (rho, u, T), each against the field's own max |value| (u: both
    components against max |u_ref|)."""
    e_rho = float(np.max(np.abs(got[0] - want[0])) / np.max(np.abs(want[0])))
    umax = max(np.max(np.abs(want[1])), np.max(np.abs(want[2])))
    e_u = float(max(np.max(np.abs(got[1] - want[1])), np.max(np.abs(got[2] - want[2]))) / umax)
    e_T = float(np.max(np.abs(got[3] - want[3])) / np.max(np.abs(want[3])))
    return {"max_rel_err_rho": e_rho, "max_rel_err_u": e_u, "max_rel_err_T": e_T}


def max_over_ranks(x, world, device):
    """The largest of the ranks' values of x (x itself on one rank)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(world, cells, tsteps, steps, seconds):
    """Whole-job MLUPS: every rank advances its own replica of `cells` cells by tsteps x steps
    time steps; `seconds` is the slowest rank's time."""
    return world * cells * tsteps * steps / seconds / 1e6


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


class Clocks:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[3 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_bf16():
    """Dense BF16 tensor peak in TFLOP/s: the measured burst figure, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def csrc_hash(files):
    """sha256 of the named kernel source files (in order), or None if one is missing."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1004_5059_gb300", "csrc")
    try:
        for fn in files:
            h.update(open(os.path.join(csrc, fn), "rb").read())
    except (OSError, TypeError):
        return None
    return h.hexdigest()


def profile_entry(workload, form, tile=None):
    """The committed ncu record of the sweep kernel of `workload` in `form` (profiles/traffic.json:
    one record, or a list of them for several tile shapes), if it was taken on the current kernel
    sources with the same tile shape (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    entries = d.get("%s/%s" % (workload, form))
    if not entries:
        return None
    for e in entries if isinstance(entries, list) else [entries]:
        # the sources the kernel is built from, as recorded with the counters
        if e.get("csrc_sha256") != csrc_hash(e.get("csrc_files")):
            continue
        if tile is not None and e.get("tile") is not None and list(e["tile"]) != list(tile):
            continue
        return e
    return None


def kernel_traffic(workload, form, tile=None):
    """DRAM bytes per sweep launch from the committed ncu summary (profile_entry), else None."""
    e = profile_entry(workload, form, tile)
    return e.get("dram_bytes_per_launch") if e else None


# SM instruction issue of one GB300: 152 SMs x 4 schedulers x 1 warp instruction per cycle x
# 32 threads at the 2070 MHz maximum SM clock, in thread instructions per second
ISSUE_PEAK = 152 * 4 * 32 * 2.07e9


def kernel_instructions(workload, form, tile=None):
    """Thread instructions per cell update of the sweep kernel from the committed ncu summary
    (profile_entry), else None."""
    e = profile_entry(workload, form, tile)
    return e.get("thread_instructions_per_cell") if e else None


def issue_roofline(workload, form, tile, cells, s_per_tstep):
    """The sweep against the SM instruction-issue rate: recorded instructions per cell x cells
    per second of the whole time step (other kernels of the step counted as sweep time, so a
    lower bound), or None without a record."""
    ipc = kernel_instructions(workload, form, tile)
    if ipc is None:
        return None
    achieved = ipc * cells / s_per_tstep
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": ISSUE_PEAK / 1e12,
            "unit": "T thread-instructions/s", "frac": achieved / ISSUE_PEAK, "instructions_per_cell": ipc}


def traffic_per_time_step(workload, form, tile=None):
    """kernel_traffic divided by the time steps one launch advances (a dataflow launch runs many)."""
    e = profile_entry(workload, form, tile)
    if not e or e.get("dram_bytes_per_launch") is None:
        return None
    return e["dram_bytes_per_launch"] / e.get("time_steps_per_launch", 1)


def run_ours(args, w, rank, world, local_rank, sub=None):
    """The workload's bench line.  sub: the name of a configuration measured beside the default
    line -- then only its timed sweep, roofline fraction and oracle check (no e2e, plain form or
    process-group set-up), as a compact record."""
    import torch
    import paper_1004_5059_gb300 as tv

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1 and sub is None:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    nx, ny, tsteps = w["nx"], w["ny"], w["tsteps"]
    cells = nx * ny
    fields = fields_for(sub or args.workload, w)
    stream = torch.cuda.current_stream(dev)

    def make(form, storage=None):
        s = tv.Simulation(nx, ny, w["velset"], tau=w["tau"], dt=1.0, walls=w["walls"],
                          storage=storage or w["storage"], form=form, stream=stream)
        if w.get("reference") == "rows" and (storage or w["storage"]).endswith("_dev"):
            # per-row deviation reference at the channel's start: at rest, T linear across it
            s.set_reference_rows(np.zeros(ny), np.zeros(ny), fields[3][:, 0])
        elif w.get("reference") and (storage or w["storage"]).endswith("_dev"):
            s.set_reference(*w["reference"])
        s.init_moments(*fields)
        if w.get("refresh") and (storage or w["storage"]).endswith("_dev"):
            s.set_reference_refresh(w["refresh"], kind=w.get("ref_kind"))
        return s

    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1 and sub is None:
            import torch.distributed as dist
            dist.barrier()

    def timed(sim, K, W):
        for _ in range(W):
            sim.step(tsteps)
        torch.cuda.synchronize()
        evs = []
        barrier()
        torch.cuda.synchronize()
        for _ in range(K):
            flush.zero_()  # evict the L2 between timed steps (outside the events)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.step(tsteps)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        barrier()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        return ms

    # form and tile shape: the requested ones, else the fastest (form, tile) pair the autotuner
    # finds among the tiled form, the strip form (no tile shape) and, on periodic domains,
    # the multi-step dataflow form
    if args.form == "auto":
        forms = ["tiled", "strip"] if w["walls"] else ["tiled", "strip", "flow"]
    else:
        forms = [args.form]
    probe, chosen, tuning, trials, predicted = None, None, None, {}, None
    for form in forms:
        try:
            sim = make(form)
        except tv.TvlbmError:
            continue
        if form == "strip" and len(forms) > 1:
            from paper_1004_5059_gb300 import autotune
            t = autotune.time_config(sim, 0, min(tsteps, 100), 3)
            trials["strip"] = round(t * 1e6, 2)
            if tuning is not None and t >= tuning["s_per_step"]:
                sim.close()
                continue
            tuning = {"best": 0, "s_per_step": t}
        elif form not in ("plain", "strip"):
            if args.tile >= 0:
                sim.set_tile(args.tile)
            else:
                from paper_1004_5059_gb300 import autotune
                log = autotune_log_path(args)
                if log and predicted is None:  # the log's model, before this run adds to it
                    predicted = autotune.predict(autotune.read_log(log), w["nx"], w["ny"], sim.velset, sim.storage,
                                                 form)
                tr = autotune.autotune(sim, steps=min(tsteps, 100), repeats=3, log_path=log, form=form)
                for t in tr["trials"]:
                    trials["%s %s" % (form, tuple(t["tile"]))] = round(t["s_per_step"] * 1e6, 2)
                best_t = min(t["s_per_step"] for t in tr["trials"])
                if tuning is not None and best_t >= tuning["s_per_step"]:
                    sim.close()
                    continue
                tuning = {"best": tr["best"], "s_per_step": best_t}
        if probe is not None:
            probe.close()
        probe, chosen = sim, form
        if tuning is None:
            break
    if probe is None:
        raise RuntimeError("no sweep form available for workload %s" % args.workload)
    probe.init_moments(*fields)
    if sub is not None:
        return sub_record(sub, w, probe, chosen, tuning, trials, timed, fields, tv)
    clocks = Clocks(local_rank)
    clocks.start()
    ms_total = timed(probe, args.steps, args.warmup)
    clk = clocks.stop()
    bytes_per_cell = probe.bytes_per_cell()
    ms_max = max_over_ranks(ms_total, world, dev)
    launches_per_tstep = 2 if w["walls"] else 1
    # seconds per time step of the sweep: one launch per time step (wall kernels of wall runs
    # counted in), or, for the dataflow form, one launch per bench step of tsteps time steps
    avg_launch_s = ms_total / 1e3 / (args.steps * tsteps)
    value = aggregate_mlups(world, cells, tsteps, args.steps, ms_max / 1e3)

    # plain form beside the chosen one (the metric reports both)
    plain, sp = None, None
    if chosen != "plain" or w["plain_storage"] != w["storage"]:
        sp = make("plain", w["plain_storage"])
        kp = max(1, args.steps // 2)
        msp = timed(sp, kp, 1)
        plain_launch_s = msp / 1e3 / (kp * tsteps)
        plain = {"value": cells * tsteps * kp / (msp / 1e3) / 1e6, "unit": UNIT, "form": "plain",
                 "storage": w["plain_storage"], "bytes_per_cell": sp.bytes_per_cell(), "roofline_frac": None}

    # end to end through the C ABI with host buffers: init from pinned host fields (H2D),
    # run the time steps, read the moments back (D2H), every step
    pinned_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in fields]
    pinned_out = [torch.empty((ny, nx), dtype=torch.float64).pin_memory() for _ in range(4)]
    host_in = [p.numpy() for p in pinned_in]
    host_out = [p.numpy() for p in pinned_out]
    e2e_steps = max(1, min(args.steps, 5))
    probe.init_moments(*host_in)
    probe.step(tsteps)
    tv.tvlbm_moments(probe.ctx, nx, ny, out=host_out)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        probe.init_moments(*host_in)
        probe.step(tsteps)
        tv.tvlbm_moments(probe.ctx, nx, ny, out=host_out)
    torch.cuda.synchronize()
    e2e_value = aggregate_mlups(world, cells, tsteps, e2e_steps,
                                max_over_ranks(time.perf_counter() - t0, world, dev))

    peak, peak_kind = measured_peak_hbm()
    achieved = bytes_per_cell * cells / avg_launch_s / 1e9
    if plain is not None:
        plain["roofline_frac"] = plain["bytes_per_cell"] * cells / plain_launch_s / 1e9 / peak
    line_tile = form_tile(tv, probe, chosen, tuning["best"] if tuning else max(args.tile, 0))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp16_dev": "f32 (f16 storage)", "bf16_dev": "f32 (bf16 storage)",
                  "fp32_dev": "f32"}[w["storage"]],
        "data": "synthetic (seeded fields shaped like the paper's test problems)",
        "config": {"workload": w["desc"], "nx": nx, "ny": ny, "velset": w["velset"], "storage": w["storage"],
                   "tau": w["tau"], "time_steps_per_bench_step": tsteps, "form": chosen,
                   "deviation_reference": ("per row: the start's equilibria (u = 0, T linear between the walls), "
                                           "reset every %d steps inside the timed region to the rows' %s" % (
                                               w.get("refresh", 0),
                                               "mean populations" if w.get("ref_kind") == "mean"
                                               else "mean-state equilibria")
                                           if w.get("reference") == "rows" else w.get("reference")),
                   "tile": line_tile,
                   "autotune_us_per_time_step": trials or None,
                   "autotune_log_prediction": predicted,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "L2 flushed (512 MiB write) between timed steps; state %.0f MB" % (
                       bytes_per_cell * cells / 1e6)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "bytes_per_cell": bytes_per_cell,
                     "traffic": kernel_traffic(args.workload, chosen, line_tile),
                     "traffic_per_time_step": traffic_per_time_step(args.workload, chosen, line_tile),
                     "algorithmic_bytes_per_time_step": bytes_per_cell * cells,
                     "issue": issue_roofline(args.workload, chosen, line_tile, cells, avg_launch_s)},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * 8 * cells,
                "d2h_bytes_per_step": 4 * 8 * cells},
        # sweeps (+ wall kernel per step) and, with a refreshed per-row reference, the five kernels
        # of each refresh (row averages, two table kernels, shifts, re-encoding)
        "gpu_launches": args.steps * ((1 if chosen == "flow" else tsteps * launches_per_tstep) +
                                      (5 * (tsteps // w["refresh"]) if w.get("refresh") else 0)),
        "clocks": clk,
    }
    if plain is not None:
        line["plain_form"] = plain
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sims = {"chosen": probe}
        if sp is not None:
            sims["plain"] = sp
        line["cpu_baseline"], acc = cpu_baseline(args.workload, w, fields, sims)
        line["accuracy_vs_oracle"] = acc
        if plain is not None and acc:
            plain["max_rel_err_vs_oracle"] = acc["plain"]
            plain["time_steps_checked"] = acc["time_steps"]
    if sp is not None:
        sp.close()
    if rank == 0 and world == 1 and not args.no_extras and args.workload == "c1":
        line["extra_keys"] = list(EXTRA)
        probe.close()
        probe = None
        for name in EXTRA:
            line[name] = (run_batch(args, rank, world, local_rank, sub=True) if name == "c3" else
                          run_ours(args, WORKLOADS[name], rank, world, local_rank, sub=name))
    if probe is not None:
        probe.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line if rank == 0 else None


def form_tile(tv, sim, form, cfg):
    """The sweep's work shape: (tile width, tile height, rows per thread) of the tiled and
    dataflow forms; (128 columns, 1 row, 1 row) for the strip form, whose CTAs walk 128-column
    strips a row at a time; None for the plain form."""
    if form == "plain":
        return None
    if form == "strip":
        return [128, 1, 1]
    return list(tv.tvlbm_tile_shape(sim.ctx, cfg))


def autotune_log_path(args):
    """Where the autotuner appends its trials (None: not logged)."""
    if args.autotune_log == "none":
        return None
    if args.autotune_log:
        return args.autotune_log
    from paper_1004_5059_gb300 import autotune
    return autotune.default_log_path()


def _oracle_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(name, w, fields, sims=None, target_s=10.0):
    """The FP64 oracle, as it stands, on this machine's host cores over a bounded sample of the
    workload's time steps (whole grid), with all threads and with one; then the oracle continued
    to the workload's full run (untimed) and every GPU form in `sims` run as far from the same
    start, compared field by field.  A channel (x-invariant flow) is checked on an 8-column strip
    of the oracle, every GPU column against it."""
    import oracle
    cores = _oracle_threads()
    o = oracle.Oracle(w["nx"], w["ny"], w["velset"], tau=w["tau"], dt=1.0, walls=w["walls"], threads=cores)
    o.init_moments(*fields)
    t0 = time.perf_counter()
    o.run(1)
    one = time.perf_counter() - t0
    n = int(max(1, min(w["tsteps"] - 1, target_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    o.run(n)
    dt = time.perf_counter() - t0
    out = {"value": w["nx"] * w["ny"] * n / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "%d of the workload's %d time steps on the full %dx%d grid (after 1 untimed step)" % (
               n, w["tsteps"], w["nx"], w["ny"])}
    if cores > 1:
        o1 = oracle.Oracle(w["nx"], w["ny"], w["velset"], tau=w["tau"], dt=1.0, walls=w["walls"], threads=1)
        o1.init_moments(*fields)
        t0 = time.perf_counter()
        o1.run(1)
        one1 = time.perf_counter() - t0
        n1 = int(max(1, min(w["tsteps"], 0.4 * target_s / max(one1, 1e-6))))
        t0 = time.perf_counter()
        o1.run(n1)
        dt1 = time.perf_counter() - t0
        out["one_thread"] = {"value": w["nx"] * w["ny"] * n1 / dt1 / 1e6, "unit": UNIT, "cores": 1,
                             "sample": "%d time steps on the full grid (after 1 untimed step)" % n1}
        del o1
    if not sims:
        return out, None
    if w["walls"]:
        o = oracle.Oracle(8, w["ny"], w["velset"], tau=w["tau"], dt=1.0, walls=w["walls"], threads=cores)
        o.init_moments(*[a[:, :8] for a in fields])
        o.run(w["tsteps"])
    else:
        o.run(w["tsteps"] - 1 - n)
    want = o.moments()
    if w["walls"]:
        want = [np.broadcast_to(a[:, :1], (w["ny"], w["nx"])) for a in want]
    acc = {"time_steps": w["tsteps"]}
    for label, sim in sims.items():
        sim.init_moments(*fields)
        if w.get("refresh") and w["storage"].endswith("_dev"):
            sim.set_reference_refresh(w["refresh"], kind=w.get("ref_kind"))  # restarts the refresh count
        sim.step(w["tsteps"])
        acc[label] = field_errors(sim.moments(), want)
    return out, acc


def sub_record(name, w, sim, form, tuning, trials, timed, fields, tv, K=3, W=2):
    """Compact record of a configuration measured beside the default line: K timed bench steps
    after W, MLUPS and the HBM roofline fraction, and the GPU against the oracle (a channel: after
    the full run on an 8-column strip; a periodic grid: after its whole run if small, else a few
    time steps, on the full grid)."""
    import oracle
    nx, ny, tsteps = w["nx"], w["ny"], w["tsteps"]
    ms = timed(sim, K, W)
    s_per_tstep = ms / 1e3 / (K * tsteps)
    bpc = sim.bytes_per_cell()
    peak, peak_kind = measured_peak_hbm()
    achieved = bpc * nx * ny / s_per_tstep / 1e9
    rec = {"workload": w["desc"], "value": nx * ny / s_per_tstep / 1e6, "unit": UNIT, "ms_per_step": ms / K,
           "steps": K, "warmup": W, "form": form, "storage": w["storage"],
           "tile": form_tile(tv, sim, form, tuning["best"]) if tuning else None,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "peak_kind": peak_kind, "bytes_per_cell": bpc,
                        "traffic": kernel_traffic(name, form, form_tile(tv, sim, form, tuning["best"])
                                                  if tuning else None),
                        "issue": issue_roofline(name, form, form_tile(tv, sim, form, tuning["best"])
                                                if tuning else None, nx * ny, s_per_tstep)}}
    if w.get("refresh"):
        rec["deviation_reference"] = "per row, %s kind, refreshed every %d time steps inside the timed region" % (
            w.get("ref_kind", "equilibrium"), w["refresh"])
    if w.get("note"):
        rec["note"] = w["note"]
    cores = _oracle_threads()
    if w["walls"]:
        o = oracle.Oracle(8, ny, w["velset"], tau=w["tau"], dt=1.0, walls=w["walls"], threads=cores)
        o.init_moments(*[a[:, :8] for a in fields])
        t0 = time.perf_counter()
        o.run(tsteps)
        dt = time.perf_counter() - t0
        checked = tsteps
        want = [np.broadcast_to(a[:, :1], (ny, nx)) for a in o.moments()]
        rec["cpu_baseline"] = {"value": 8 * ny * tsteps / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": "the full run of an 8x%d strip of the channel (the flow is x-invariant)" % ny}
    else:
        o = oracle.Oracle(nx, ny, w["velset"], tau=w["tau"], dt=1.0, walls=w["walls"], threads=cores)
        o.init_moments(*fields)
        checked = tsteps if nx * ny * tsteps <= 1 << 22 else 3  # a small grid: its whole run
        t0 = time.perf_counter()
        o.run(checked)
        dt = time.perf_counter() - t0
        want = o.moments()
        rec["cpu_baseline"] = {"value": nx * ny * checked / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": "%d time steps on the full grid" % checked}
    sim.init_moments(*fields)
    if w.get("refresh"):
        sim.set_reference_refresh(w["refresh"], kind=w.get("ref_kind"))  # restarts the refresh count
    sim.step(checked)
    rec["accuracy_vs_oracle"] = dict(time_steps=checked, **field_errors(sim.moments(), want))
    if trials:
        rec["autotune_us_per_time_step"] = trials
    sim.close()
    return rec


def run_reference(args, w, rank, world):
    """The FP64 CPU oracle timed on the host cores: each bench step runs a bounded sample of
    `sample_steps` of the workload's time steps on the full grid."""
    if rank != 0:
        return None
    import oracle
    cores = _oracle_threads()
    fields = fields_for(args.workload, w)
    o = oracle.Oracle(w["nx"], w["ny"], w["velset"], tau=w["tau"], dt=1.0, walls=w["walls"], threads=cores)
    o.init_moments(*fields)
    t0 = time.perf_counter()
    o.run(1)
    one = time.perf_counter() - t0
    # size each step so that warmup + steps stay within ~3 minutes
    per_step_budget = 180.0 / max(1, args.steps + args.warmup)
    sample = int(max(1, min(w["tsteps"], per_step_budget / max(one, 1e-6))))
    for _ in range(args.warmup):
        o.run(sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.run(sample)
    dt = time.perf_counter() - t0
    value = w["nx"] * w["ny"] * sample * args.steps / dt / 1e6
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "nx": w["nx"], "ny": w["ny"], "velset": w["velset"],
                   "storage": "fp64 (oracle)", "tau": w["tau"], "time_steps_per_bench_step": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d of the workload's %d time steps per bench step, full grid" % (sample, w["tsteps"])},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def batch_fields(spec):
    """Seeded initial fields of one batched domain: T bump + random Fourier flow scaled to the
    domain's Mach number (c_s = 1)."""
    n = spec["n"]
    return workloads.gaussian_bump_random_flow(n, n, seed=spec["seed"], amp_u=spec["mach"], sigma=n / 16.0)


def run_batch(args, rank, world, local_rank, sub=False):
    """The batched workload's bench line; sub: a compact record measured beside the default line
    (3 timed bench steps after 2, the roofline fraction, the smallest domains against the oracle)."""
    import torch
    import paper_1004_5059_gb300 as tv
    from paper_1004_5059_gb300 import autotune

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1 and not sub:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    specs = workloads.batched_domains(BATCH["count"], seed=BATCH["seed"])
    n = [s["n"] for s in specs]
    stream = torch.cuda.current_stream(dev)
    b = tv.Batch(n, n, [s["tau"] for s in specs], BATCH["velset"], storage=BATCH["storage"], stream=stream)
    fields = [batch_fields(s) for s in specs]
    for d, f in enumerate(fields):
        b.init_moments(d, *f)
    tsteps = BATCH["tsteps"]
    # autotune form and tile shape on the batch itself (untimed), then restart from the initial
    # state: the tiled form (one launch per time step) and the dataflow form (the bench step's
    # time steps in one persistent launch, replayed from a captured graph)
    trials = {}
    for form in ("tiled", "flow"):
        for cfg in range(b.tile_count()):
            b.set_form("tiled")
            b.set_tile(cfg)
            try:
                b.set_form(form)
            except tv.TvlbmError:
                continue
            b.step(tsteps)
            b.step(tsteps)
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            b.step(tsteps)
            e.record(stream)
            e.synchronize()
            trials[(form, cfg)] = a.elapsed_time(e) / tsteps
    best_form, best = min(trials, key=trials.get)
    b.set_form("tiled")
    b.set_tile(best)
    b.set_form(best_form)
    for d, f in enumerate(fields):
        b.init_moments(d, *f)
    cells = b.cells()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    K, W = (3, 2) if sub else (args.steps, args.warmup)
    for _ in range(W):
        b.step(tsteps)
    torch.cuda.synchronize()
    if world > 1 and not sub:
        import torch.distributed as dist
        dist.barrier()
    clocks = Clocks(local_rank)
    clocks.start()
    evs = []
    for _ in range(K):
        flush.zero_()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        b.step(tsteps)
        e.record(stream)
        evs.append((a, e))
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(e) for a, e in evs)
    peak, peak_kind = measured_peak_hbm()
    if sub:
        achieved = b.bytes_per_cell() * cells / (ms / 1e3 / (K * tsteps)) / 1e9
        rec = {"workload": BATCH["desc"], "value": cells * tsteps * K / (ms / 1e3) / 1e6, "unit": UNIT,
               "ms_per_step": ms / K, "steps": K, "warmup": W, "storage": BATCH["storage"], "domains": b.count,
               "cells": cells, "form": best_form, "tile": list(b.tile_shape(best)),
               "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "peak_kind": peak_kind, "bytes_per_cell": b.bytes_per_cell(),
                            "traffic": None}}
        # the 8 smallest domains after the bench step's time steps, against the oracle
        import oracle
        order = sorted(range(b.count), key=lambda d: specs[d]["n"])[:8]
        for d in order:
            b.init_moments(d, *fields[d])
        b.step(tsteps)
        worst = {"max_rel_err_rho": 0.0, "max_rel_err_u": 0.0, "max_rel_err_T": 0.0}
        for d in order:
            o = oracle.Oracle(specs[d]["n"], specs[d]["n"], BATCH["velset"], tau=specs[d]["tau"],
                              threads=_oracle_threads())
            o.init_moments(*fields[d])
            o.run(tsteps)
            e = field_errors(b.moments(d), o.moments())
            worst = {k: max(worst[k], e[k]) for k in worst}
        rec["accuracy_vs_oracle"] = dict(time_steps=tsteps, domains=len(order), **worst)
        b.close()
        rec["cpu_baseline"] = batch_cpu_baseline(target_s=4.0)
        return rec
    ms_max = max_over_ranks(ms, world, dev)
    value = aggregate_mlups(world, cells, tsteps, args.steps, ms_max / 1e3)
    achieved = b.bytes_per_cell() * cells / (ms / 1e3 / (args.steps * tsteps)) / 1e9
    # end to end: host fields of every domain in (pinned), time steps, every domain's moments out
    pinned = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in f] for f in fields]
    e2e_steps = 2
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for d, f in enumerate(pinned):
            b.init_moments(d, *f)
        b.step(tsteps)
        for d in range(b.count):
            b.moments(d)
    torch.cuda.synchronize()
    e2e = aggregate_mlups(world, cells, tsteps, e2e_steps, max_over_ranks(time.perf_counter() - t0, world, dev))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded fields)",
        "config": {"workload": BATCH["desc"], "domains": b.count, "cells": cells, "velset": BATCH["velset"],
                   "storage": BATCH["storage"], "time_steps_per_bench_step": tsteps,
                   "form": best_form, "tile": list(b.tile_shape(best)), "autotune_ms_per_time_step": {
                       "%s %s" % (f, b.tile_shape(k)): round(v, 4) for (f, k), v in trials.items()},
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "L2 flushed between timed steps; state %.1f GB" % (b.bytes_per_cell() * cells / 1e9)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "bytes_per_cell": b.bytes_per_cell(), "traffic": None},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 32 * cells, "d2h_bytes_per_step": 32 * cells},
        "gpu_launches": args.steps * (1 if best_form == "flow" else tsteps),
        "clocks": clk,
    }
    b.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline()
    return line if rank == 0 else None


def batch_cpu_baseline(target_s=10.0):
    """The oracle on a bounded sample of the batched workload: time steps of the smallest domains
    (all of them advanced together) repeated until about target_s seconds of host work."""
    import oracle
    specs = sorted(workloads.batched_domains(BATCH["count"], seed=BATCH["seed"]), key=lambda s: s["n"])[:8]
    cores = _oracle_threads()
    sims = []
    for s in specs:
        o = oracle.Oracle(s["n"], s["n"], BATCH["velset"], tau=s["tau"], threads=cores)
        o.init_moments(*batch_fields(s))
        sims.append(o)
    cells = sum(s["n"] ** 2 for s in specs)
    for o in sims:
        o.run(1)
    done, t0 = 0, time.perf_counter()
    while True:
        for o in sims:
            o.run(1)
        done += 1
        dt = time.perf_counter() - t0
        if dt >= target_s:
            break
    return {"value": cells * done / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d time steps of the %d smallest domains (%d cells) of the same batch" % (done, len(specs), cells)}


def run_batch_reference(args, rank):
    """The oracle on the batched workload: each bench step one time step of a bounded sample of
    the domains (the smallest ones first), timed on the host cores."""
    if rank != 0:
        return None
    import oracle
    specs = sorted(workloads.batched_domains(BATCH["count"], seed=BATCH["seed"]), key=lambda s: s["n"])[:8]
    cores = _oracle_threads()
    sims = []
    for s in specs:
        o = oracle.Oracle(s["n"], s["n"], BATCH["velset"], tau=s["tau"], threads=cores)
        o.init_moments(*batch_fields(s))
        sims.append(o)
    cells = sum(s["n"] ** 2 for s in specs)
    for _ in range(args.warmup):
        for o in sims:
            o.run(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for o in sims:
            o.run(1)
    dt = time.perf_counter() - t0
    value = cells * args.steps / dt / 1e6
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": BATCH["desc"], "sample": "one time step of the %d smallest domains" % len(specs)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one time step of the %d smallest domains per bench step" % len(specs)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


FV = dict(desc="the paper's finite-volume scheme (Eq. FVLB + Prandtl term, tau_g = 2 tau): D2Q16 1024x1024 "
               "periodic FP32, tau = 0.5, dt = 0.02, C1 fields; 200 explicit steps per bench step",
          nx=1024, ny=1024, tau=0.5, tau_g=1.0, dt=0.02, tsteps=200)


def run_fv(args, rank, world, local_rank):
    """Throughput of the finite-volume scheme: one fused kernel per step (collision term of each
    block in shared memory, then the update), with the two-kernel form timed beside it."""
    import torch
    import paper_1004_5059_gb300 as tv
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    nx, ny, tsteps = FV["nx"], FV["ny"], FV["tsteps"]
    fields = workloads.gaussian_bump_random_flow(nx, ny, seed=1)
    stream = torch.cuda.current_stream(dev)
    sim = tv.Simulation(nx, ny, "D2Q16", tau=FV["tau"], dt=FV["dt"], storage="fp32", stream=stream)
    sim.set_scheme("fvlb", FV["tau_g"])
    sim.init_moments(*fields)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def timed(fused, steps, warmup):
        sim.set_fv_fused(fused)
        for _ in range(warmup):
            sim.step(tsteps)
        torch.cuda.synchronize()
        evs = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.step(tsteps)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs)

    for _ in range(args.warmup):
        sim.step(tsteps)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = Clocks(local_rank)
    clocks.start()
    ms = timed(True, args.steps, 0)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms, world, dev)
    cells = nx * ny
    value = aggregate_mlups(world, cells, tsteps, args.steps, ms_max / 1e3)
    # algorithmic bytes per cell update of the fused kernel: read Q and write Q values (the halo
    # ring's re-reads come from L2); the two-kernel form: the collision term reads Q and writes Q,
    # the update reads 2 Q distinct values (f and the collision term; the 3 x 3 neighbours from
    # cache) and writes Q
    bpc, bpc_split = 2 * 16 * 4, 5 * 16 * 4
    peak, peak_kind = measured_peak_hbm()
    achieved = bpc * cells / (ms / 1e3 / (args.steps * tsteps)) / 1e9
    split_steps = max(1, min(args.steps, 3))
    ms_split = timed(False, split_steps, 1)
    sec_split = ms_split / 1e3 / (split_steps * tsteps)
    two_kernel = {"value": cells / sec_split / 1e6, "unit": UNIT, "bytes_per_cell": bpc_split,
                  "roofline_frac": bpc_split * cells / sec_split / 1e9 / peak, "bench_steps": split_steps}
    sim.set_fv_fused(True)
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in fields]
    out = [torch.empty((ny, nx), dtype=torch.float64).pin_memory().numpy() for _ in range(4)]
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(2):
        sim.init_moments(*pinned)
        sim.step(tsteps)
        tv.tvlbm_moments(sim.ctx, nx, ny, out=out)
    e2e = aggregate_mlups(world, cells, tsteps, 2, max_over_ranks(time.perf_counter() - te, world, dev))
    line = {"metric": METRIC + " (finite-volume scheme)", "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (C1 fields)",
            "config": {"workload": FV["desc"], "nx": nx, "ny": ny, "time_steps_per_bench_step": tsteps,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "L2 flushed (512 MiB write) between timed steps"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "bytes_per_cell": bpc, "traffic": None},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 32 * cells, "d2h_bytes_per_step": 32 * cells},
            "two_kernel_form": two_kernel,
            "gpu_launches": args.steps * tsteps, "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        from oracle import fvlb
        cores = _oracle_threads()
        o = fvlb.FVLB(256, 256, "D2Q16", tau=FV["tau"], tau_g=FV["tau_g"], dt=FV["dt"])
        o.init_moments(*workloads.gaussian_bump_random_flow(256, 256, seed=1, sigma=16.0))
        t0 = time.perf_counter()
        o.step(5)
        dt_ = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 256 * 256 * 5 / dt_ / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "5 finite-volume steps of a 256x256 grid (numpy, one core)"}
    sim.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line if rank == 0 else None


def run_fv_reference(args, rank):
    if rank != 0:
        return None
    from oracle import fvlb
    o = fvlb.FVLB(256, 256, "D2Q16", tau=FV["tau"], tau_g=FV["tau_g"], dt=FV["dt"])
    o.init_moments(*workloads.gaussian_bump_random_flow(256, 256, seed=1, sigma=16.0))
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt_ = time.perf_counter() - t0
    value = 256 * 256 * args.steps / dt_ / 1e6
    return {"impl": "reference", "metric": METRIC + " (finite-volume scheme)", "value": value, "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt_ * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": FV["desc"], "sample": "one step of a 256x256 grid per bench step (oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "one finite-volume step of a 256x256 grid per bench step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


MESH = dict(desc="volumetric scheme on a mesh non-uniform in y: D2Q16 1024x1024 thermal Couette channel (walls "
                 "u = 0, T = 1 and u = 0.1, T = 1.1), tanh faces (beta = 2.3, cells 0.09 to 2.3) over a height of "
                 "1024, FP32 deviation storage, tau = 0.9, dt = 1, 100 steps per bench step",
            nx=1024, ny=1024, beta=2.3, tau=0.9, dt=1.0, tsteps=100, walls=(0.0, 1.0, 0.1, 1.1),
            sample_nx=64, sample_ny=64, sample_steps=60)


def run_mesh(args, rank, world, local_rank):
    """Throughput of the volumetric step on the tanh mesh (plain form: per-row gather tables and
    the wall fill), with unit cells timed beside it on the same grid, and the errors against the
    oracle on a 64x64 channel of the same mesh law."""
    import torch
    import paper_1004_5059_gb300 as tv
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    nx, ny, tsteps, walls = MESH["nx"], MESH["ny"], MESH["tsteps"], MESH["walls"]
    stream = torch.cuda.current_stream(dev)
    sim = tv.Simulation(nx, ny, "D2Q16", tau=MESH["tau"], dt=MESH["dt"], storage="fp32_dev", walls=walls,
                        stream=stream)
    sim.set_y_faces(workloads.tanh_faces(ny, float(ny), MESH["beta"]))
    fields = workloads.couette_linear(nx, ny, walls[1], walls[3])
    sim.init_moments(*fields)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def timed(steps, warmup):
        for _ in range(warmup):
            sim.step(tsteps)
        torch.cuda.synchronize()
        evs = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.step(tsteps)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs)

    timed(0, args.warmup)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = Clocks(local_rank)
    clocks.start()
    ms = timed(args.steps, 0)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms, world, dev)
    cells = nx * ny
    value = aggregate_mlups(world, cells, tsteps, args.steps, ms_max / 1e3)
    bpc = 2 * 16 * 4  # read and write Q FP32 values per cell update (the wall fill and the extra
    peak, peak_kind = measured_peak_hbm()  # gather rows of the thin cells come from L2)
    achieved = bpc * cells / (ms / 1e3 / (args.steps * tsteps)) / 1e9
    # unit cells on the same grid, same form (the uniform scheme's plain sweep and wall kernel)
    sim.set_y_faces(None)
    sim.set_form("plain")
    sim.init_moments(*fields)
    ms_u = timed(max(1, min(args.steps, 3)), 1)
    unit = {"value": cells * tsteps * max(1, min(args.steps, 3)) / (ms_u / 1e3) / 1e6, "unit": UNIT,
            "form": "plain", "note": "unit cells, the uniform scheme's plain sweep and wall kernel"}
    sim.set_y_faces(workloads.tanh_faces(ny, float(ny), MESH["beta"]))
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in fields]
    out = [torch.empty((ny, nx), dtype=torch.float64).pin_memory().numpy() for _ in range(4)]
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(2):
        sim.init_moments(*pinned)
        sim.step(tsteps)
        tv.tvlbm_moments(sim.ctx, nx, ny, out=out)
    e2e = aggregate_mlups(world, cells, tsteps, 2, max_over_ranks(time.perf_counter() - te, world, dev))
    sim.close()
    line = {"metric": METRIC + " (volumetric scheme, non-uniform y mesh)", "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (channel fields)",
            "config": {"workload": MESH["desc"], "nx": nx, "ny": ny, "time_steps_per_bench_step": tsteps,
                       "form": "plain", "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "L2 flushed (512 MiB write) between timed steps"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "bytes_per_cell": bpc, "traffic": None},
            "unit_cells": unit,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 32 * cells, "d2h_bytes_per_step": 32 * cells},
            "gpu_launches": args.steps * tsteps * 2, "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle.mesh import MeshOracle
        snx, sny, sst = MESH["sample_nx"], MESH["sample_ny"], MESH["sample_steps"]
        sf = workloads.tanh_faces(sny, float(sny), MESH["beta"])
        sw = workloads.couette_linear(snx, sny, walls[1], walls[3])
        o = MeshOracle(snx, sf, "D2Q16", tau=MESH["tau"], dt=MESH["dt"], walls=walls)
        o.init_moments(*sw)
        t0 = time.perf_counter()
        o.step(sst)
        dt_ = time.perf_counter() - t0
        g = tv.Simulation(snx, sny, "D2Q16", tau=MESH["tau"], dt=MESH["dt"], storage="fp32_dev", walls=walls)
        g.set_y_faces(sf)
        g.init_moments(*sw)
        g.step(sst)
        got, want = g.moments(), o.moments()
        g.close()
        du = np.max(np.abs(got[1] - want[1]) + np.abs(got[2] - want[2])) / np.max(np.hypot(want[1], want[2]))
        line["accuracy_vs_oracle"] = {
            "sample": "%dx%d channel, same mesh law and walls, %d steps" % (snx, sny, sst),
            "max_rel_err_rho": float(np.max(np.abs(got[0] - want[0])) / np.max(np.abs(want[0]))),
            "max_rel_err_u": float(du),
            "max_rel_err_T": float(np.max(np.abs(got[3] - want[3])) / np.max(np.abs(want[3])))}
        line["cpu_baseline"] = {"value": snx * sny * sst / dt_ / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "%d steps of the %dx%d channel (numpy gather, C collision, one core)"
                                          % (sst, snx, sny)}
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line if rank == 0 else None


def run_mesh_reference(args, rank):
    if rank != 0:
        return None
    from oracle.mesh import MeshOracle
    snx, sny = MESH["sample_nx"], MESH["sample_ny"]
    walls = MESH["walls"]
    o = MeshOracle(snx, workloads.tanh_faces(sny, float(sny), MESH["beta"]), "D2Q16", tau=MESH["tau"], dt=MESH["dt"], walls=walls)
    o.init_moments(*workloads.couette_linear(snx, sny, walls[1], walls[3]))
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt_ = time.perf_counter() - t0
    value = snx * sny * args.steps / dt_ / 1e6
    return {"impl": "reference", "metric": METRIC + " (volumetric scheme, non-uniform y mesh)", "value": value,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt_ * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": MESH["desc"], "sample": "one step of a %dx%d channel per bench step (oracle)"
                       % (snx, sny)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "one step of a %dx%d channel per bench step" % (snx, sny)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _closure_setup():
    from paper_1004_5059_gb300 import closure as C
    cfg = C.ClosureConfig(nf=CLOSURE["nf"], m=CLOSURE["m"])
    return C, cfg


def run_closure(args, rank, world, local_rank):
    """Learned coarse run (network trained here first, untimed) against the plain fine run it
    replaces: fine-equivalent MLUPS, the network's tensor throughput, and the errors of the
    plain and learned coarse runs against the block-averaged fine run on held-out seeds."""
    import torch
    import paper_1004_5059_gb300 as tv

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    C, cfg = _closure_setup()
    nsteps = CLOSURE["coarse_steps"]
    t0 = time.perf_counter()
    solver = C.TargetSolver(cfg.nc, cfg.lam, cfg.active)
    norm = C.statistics(cfg, cfg.train_seeds[0], solver)
    X, Y = C.generate(cfg, cfg.train_seeds, norm, solver)
    t1 = time.perf_counter()
    net, hist = C.train(cfg, X, Y, log_every=max(1, cfg.iters // 4))
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    del X, Y
    errors = {str(seed): C.evaluate(cfg, net, norm, seed, nsteps) for seed in cfg.test_seeds}
    # the accuracy bar: the plain fine run's own RMS error against a 2x finer run, both
    # block-averaged to the coarse grid; the learned run meets it when no field's error exceeds it
    bar = {str(seed): C.fine_grid_accuracy(cfg, seed, nsteps) for seed in cfg.test_seeds}
    for sd, e in errors.items():
        e["fine_grid_accuracy_bar"] = bar[sd]
        e["bar_met"] = all(e["learned_coarse"][k] <= bar[sd]["rms"][k] for k in bar[sd]["rms"])
    # beyond the bench horizon (the training data cover coarse steps warm .. warm + snapshots)
    horizon = C.trajectory(cfg, net, norm, cfg.test_seeds[0], checkpoints=(32, 64, 128))

    stream = torch.cuda.current_stream(dev)
    seed = cfg.test_seeds[0]
    fine = C._fine_sim(cfg, seed)
    fine.step(cfg.m * cfg.warm)
    learned, start = C._coarse_sim(cfg), C._coarse_sim(cfg)
    tv.downsample(fine, start)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def timed(fn, K, W, reset=None):
        """K timed calls of fn after W untimed ones; reset() runs before each, outside the events."""
        for _ in range(W):
            if reset:
                reset()
            fn()
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        evs = []
        for _ in range(K):
            if reset:
                reset()
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs)

    # every bench step: the 32 learned coarse steps from the block-averaged start
    clocks = Clocks(local_rank)
    clocks.start()
    ms = timed(lambda: tv.step_closure(learned, net, norm.mu, norm.inv_sigma, norm.out_scale, nsteps),
               args.steps, args.warmup, reset=lambda: tv.copy_state(start, learned))
    clk = clocks.stop()
    ms_max = max_over_ranks(ms, world, dev)
    fine_cells = cfg.nf * cfg.nf
    value = aggregate_mlups(world, fine_cells, cfg.m * nsteps, args.steps, ms_max / 1e3)
    # the plain fine run over the same physical time (what the learned run replaces)
    kf = max(1, args.steps // 2)
    ms_fine = timed(lambda: fine.step(cfg.m * nsteps), kf, 1)
    fine_value = fine_cells * cfg.m * nsteps * kf / (ms_fine / 1e3) / 1e6
    # the network alone on the whole coarse grid: the tensor-core kernels' throughput
    cells = cfg.nc * cfg.nc
    xb = torch.zeros((cells, 64), dtype=torch.bfloat16, device=dev)
    yb = torch.zeros((cells, 16), dtype=torch.float32, device=dev)
    tv.closure_features(start, norm.mu, norm.inv_sigma, xb)
    reps = 20
    ms_net = timed(lambda: [net.forward(xb, yb) for _ in range(reps)], 3, 2) / (3 * reps)
    flops = 2.0 * cells * (64 * 128 + 128 * 128 + 128 * 16)
    peak, peak_kind = measured_peak_bf16()
    achieved = flops / (ms_net / 1e3) / 1e12
    # end to end: host fields in (pinned), the learned steps, host moments out
    prims = start.moments()
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in prims]
    out = [torch.empty((cfg.nc, cfg.nc), dtype=torch.float64).pin_memory().numpy() for _ in range(4)]
    e2e_steps = 3
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        learned.init_moments(*pinned)
        tv.step_closure(learned, net, norm.mu, norm.inv_sigma, norm.out_scale, nsteps)
        tv.tvlbm_moments(learned.ctx, cfg.nc, cfg.nc, out=out)
    torch.cuda.synchronize()
    e2e = aggregate_mlups(world, fine_cells, cfg.m * nsteps, e2e_steps, max_over_ranks(time.perf_counter() - te, world, dev))
    line = {
        "metric": METRIC + " (fine-grid cell updates represented by the learned coarse run)", "value": value,
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (bf16 network operands)",
        "data": "synthetic (seeded C3-style fields)",
        "config": {"workload": CLOSURE["desc"], "fine": [cfg.nf, cfg.nf], "coarse": [cfg.nc, cfg.nc], "factor": cfg.m,
                   "tau_fine": cfg.tau_f, "tau_coarse_plain": cfg.tau_c, "coarse_steps_per_bench_step": nsteps,
                   "train_seeds": list(cfg.train_seeds), "test_seeds": list(cfg.test_seeds),
                   "samples": len(cfg.train_seeds) * cfg.snapshots * cells, "iters": cfg.iters, "batch": cfg.batch,
                   "loss_history": hist, "data_seconds": round(t1 - t0, 2), "train_seconds": round(t2 - t1, 2),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "L2 flushed (512 MiB write) between timed steps"},
        "errors_vs_block_averaged_fine_run": errors,
        "rms_errors_longer_horizon": horizon,
        "plain_fine": {"value": fine_value, "unit": UNIT, "form": "flow", "storage": "fp32_dev",
                       "note": "the 1024x1024 run over the same physical time"},
        "speedup_vs_plain_fine": value / fine_value,
        "roofline": {"bound": "tensor", "kernel": "network forward (3 tcgen05 GEMMs + epilogues) on 65536 rows",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "flops_per_launch": flops, "traffic": None},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 4 * 8 * cells, "d2h_bytes_per_step": 4 * 8 * cells},
        # per learned step: streaming with moments, the network (inputs built in it), the collision
        "gpu_launches": args.steps * nsteps * 3,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = closure_cpu_baseline(cfg, net, norm, start)
    for s_ in (fine, learned, start):
        s_.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line if rank == 0 else None


def closure_cpu_baseline(cfg, net, norm, coarse, target_s=12.0):
    """The oracle's learned coarse step (FP64, the trained parameters) on the host cores."""
    import oracle
    from oracle import closure as cl
    cores = _oracle_threads()
    theta = net.get_params().astype(np.float64)
    p = cl.unpack(theta)
    p = {k: cl.bf16_round(v) if k.startswith("W") else v for k, v in p.items()}
    o = oracle.Oracle(cfg.nc, cfg.nc, "D2Q16", tau=cfg.tau_c, threads=cores)
    o.set_populations(coarse.populations_f64())
    t0 = time.perf_counter()
    cl.closure_step(o, p, norm.mu, norm.inv_sigma, norm.out_scale)
    one = time.perf_counter() - t0
    n = int(max(1, min(8, target_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    for _ in range(n):
        cl.closure_step(o, p, norm.mu, norm.inv_sigma, norm.out_scale)
    dt = time.perf_counter() - t0
    return {"value": cfg.nf * cfg.nf * cfg.m * n / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d learned coarse steps of the 256x256 grid (fine-equivalent cell updates)" % n}


def run_closure_reference(args, rank):
    """The oracle's learned coarse step with a seeded (untrained) network, timed on the host."""
    if rank != 0:
        return None
    import oracle
    from oracle import closure as cl
    C, cfg = _closure_setup()
    cores = _oracle_threads()
    o = oracle.Oracle(cfg.nc, cfg.nc, "D2Q16", tau=cfg.tau_c, threads=cores)
    f = workloads.gaussian_bump_random_flow(cfg.nc, cfg.nc, seed=cfg.test_seeds[0], sigma=cfg.nc / 16.0)
    o.init_moments(*f)
    p = cl.init_params(cfg.init_seed, scale=0.5)
    mu, isg, sc = np.array([1.0, 0, 0, 1.0, 0, 0]), np.array([30.0, 20, 20, 30, 500, 500]), np.full(12, 1e-4)
    for _ in range(args.warmup):
        cl.closure_step(o, p, mu, isg, sc)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cl.closure_step(o, p, mu, isg, sc)
    dt = time.perf_counter() - t0
    value = cfg.nf * cfg.nf * cfg.m * args.steps / dt / 1e6
    return {"impl": "reference", "metric": METRIC + " (fine-grid cell updates represented by the learned coarse run)",
            "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": CLOSURE["desc"], "sample": "one learned coarse step per bench step (oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one learned coarse step of the 256x256 grid per bench step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c1", choices=sorted(WORKLOADS) + ["c3", "c4", "fv", "mesh"])
    ap.add_argument("--form", default=None, choices=["tiled", "flow", "plain", "strip"],
                    help="sweep form (default: the fastest of tiled, strip and, on periodic domains, flow)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the configurations measured beside it")
    ap.add_argument("--autotune-log", default=None,
                    help="file the autotuner appends its trials to (default: $TVLBM_AUTOTUNE_LOG, else the user's "
                         "cache directory; 'none': no log)")
    ap.add_argument("--tile", type=int, default=-1, help="tile configuration of the tiled form (-1: autotune)")
    args = ap.parse_args()
    rank, world, local_rank = dist_env()
    if args.workload == "fv":
        line = run_fv(args, rank, world, local_rank) if args.impl == "ours" else run_fv_reference(args, rank)
        if rank == 0 and line is not None:
            print(json.dumps(line))
        return
    if args.workload == "mesh":
        line = run_mesh(args, rank, world, local_rank) if args.impl == "ours" else run_mesh_reference(args, rank)
        if rank == 0 and line is not None:
            print(json.dumps(line))
        return
    if args.workload == "c4":
        line = run_closure(args, rank, world, local_rank) if args.impl == "ours" else run_closure_reference(args, rank)
        if rank == 0 and line is not None:
            print(json.dumps(line))
        return
    if args.workload == "c3":
        line = run_batch(args, rank, world, local_rank) if args.impl == "ours" else run_batch_reference(args, rank)
        if rank == 0 and line is not None:
            print(json.dumps(line))
        return
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        line = run_reference(args, w, rank, world)
    else:
        if args.form is None:
            import paper_1004_5059_gb300 as tv
            import torch
            torch.cuda.set_device(local_rank)
            s = tv.Simulation(16, 16, w["velset"], storage=w["storage"])
            try:
                s.set_form("tiled")
                args.form = "auto"
            except tv.TvlbmError:
                args.form = "plain"
            s.close()
        line = run_ours(args, w, rank, world, local_rank)
    if rank == 0 and line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
