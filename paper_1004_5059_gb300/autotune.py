"""Tile-shape autotuner for the tiled sweep.

For one context it times every tile configuration the library offers (tvlbm_tile_count /
tvlbm_tile_shape / tvlbm_set_tile) with CUDA events on the context's stream, keeps the fastest,
and appends one JSON record per trial to a log -- (grid, velocity set, storage, form, tile
shape, configuration, seconds per time step).  `predict` is the shape -> configuration model
trained on that log: for a grid that was never tuned it returns the configuration that won on
the nearest logged grid of the same velocity set, storage and form.  Timing runs advance the
simulation, so tune on a scratch context (or reinitialise).
"""
from __future__ import annotations

import json
import math
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


def default_log_path() -> str:
    """$TVLBM_AUTOTUNE_LOG, else autotune.jsonl in the user's cache directory."""
    path = os.environ.get("TVLBM_AUTOTUNE_LOG")
    if path:
        return path
    cache = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(cache, "tvlbm_gb300", "autotune.jsonl")


def autotune(sim, steps: int = 64, repeats: int = 3, log_path: str | None = None, form: str | None = None) -> dict:
    """Select the fastest tile configuration for `sim` (left selected) and return the trials;
    with `log_path`, append them to that log (`form` labels the records)."""
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
                                     "storage": sim.storage, "form": form, **r}) + "\n")
    return result


def read_log(log_path: str) -> list[dict]:
    """The log's records (lines that do not parse are skipped)."""
    out = []
    try:
        with open(log_path) as fh:
            for line in fh:
                try:
                    out.append(json.loads(line))
                except ValueError:
                    continue
    except FileNotFoundError:
        pass
    return out


def predict(records: list[dict], nx: int, ny: int, velset: int, storage: int, form: str | None = None) -> dict | None:
    """Configuration for an nx x ny grid from logged trials: per logged grid (same velocity set,
    storage and form) the configuration with the lowest median time per time step; of those
    grids, the one nearest in (log2 cells, log2 aspect ratio).  None when nothing matches.
    Returns {"config", "tile", "from": [nx, ny], "distance"}."""
    per_grid: dict[tuple[int, int], dict[int, list]] = {}
    for r in records:
        if r.get("velset") != velset or r.get("storage") != storage or r.get("form") != form:
            continue
        try:
            key, cfg, t = (int(r["nx"]), int(r["ny"])), int(r["config"]), float(r["s_per_step"])
        except (KeyError, TypeError, ValueError):
            continue
        per_grid.setdefault(key, {}).setdefault(cfg, [r.get("tile"), []])[1].append(t)
    best = None
    for (gx, gy), cfgs in per_grid.items():
        d = math.hypot(math.log2(gx * gy) - math.log2(nx * ny), math.log2(gx / gy) - math.log2(nx / ny))
        cfg, (tile, ts) = min(cfgs.items(), key=lambda kv: sorted(kv[1][1])[len(kv[1][1]) // 2])
        if best is None or d < best["distance"]:
            best = {"config": cfg, "tile": tile, "from": [gx, gy], "distance": d}
    return best
