"""Tile-shape autotuner for the tiled sweep.

For one context it times every tile configuration the library offers (tvlbm_tile_count /
tvlbm_tile_shape / tvlbm_set_tile) with CUDA events on the context's stream, keeps the fastest,
and appends one JSON record per trial to a log -- (grid, velocity set, storage, tile shape,
configuration, seconds per time step) -- which is the training data for a shape -> config
model.  Timing runs advance the simulation, so tune on a scratch context (or reinitialise).
"""
from __future__ import annotations

import json
import os
import time

import paper_1004_5059_gb300 as tv


def tile_shapes(sim) -> list[tuple[int, int, int]]:
    return [tv.tvlbm_tile_shape(sim.ctx, cfg) for cfg in range(tv.tvlbm_tile_count(sim.ctx))]


def time_config(sim, cfg: int, steps: int, repeats: int) -> float:
    """Median seconds per time step of configuration cfg (one untimed warm-up run first)."""
    import torch
    sim.set_tile(cfg)
    sim.step(steps)
    times = []
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(sim.stream)
        sim.step(steps)
        b.record(sim.stream)
        b.synchronize()
        times.append(a.elapsed_time(b) / 1e3 / steps)
    times.sort()
    return times[len(times) // 2]


def autotune(sim, steps: int = 64, repeats: int = 3, log_path: str | None = None) -> dict:
    """Select the fastest tile configuration for `sim` (left selected) and return the trials."""
    shapes = tile_shapes(sim)
    trials = []
    for cfg, shape in enumerate(shapes):
        try:
            t = time_config(sim, cfg, steps, repeats)
        except tv.TvlbmError:  # not usable in the current form (dataflow: tiles must cover the domain)
            continue
        trials.append({"config": cfg, "tile": list(shape), "s_per_step": t})
    best = min(trials, key=lambda r: r["s_per_step"])
    sim.set_tile(best["config"])
    result = {"nx": sim.nx, "ny": sim.ny, "velset": sim.velset, "storage": sim.storage, "best": best["config"],
              "trials": trials}
    if log_path:
        os.makedirs(os.path.dirname(os.path.abspath(log_path)), exist_ok=True)
        with open(log_path, "a") as fh:
            for r in trials:
                fh.write(json.dumps({"time": time.time(), "nx": sim.nx, "ny": sim.ny, "velset": sim.velset,
                                     "storage": sim.storage, **r}) + "\n")
    return result
