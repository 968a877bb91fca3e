"""Autotuner for the launch configuration of the decoder and the reference
kernel, with an on-disk cache.

The tunables are, for the persistent tensor-core decoder, the tile
pipelines (warpgroups) per CTA and the resident CTAs per SM, and for the
reference integrator the lanes per shading point.  Each candidate is timed
with CUDA events on the caller's workload through the C ABI; the winner is
stored in a JSON cache keyed by GPU name, SM count, precision, material
count and workload size bucket, and applied with fabric_set_launch_config.
"""
from __future__ import annotations

import json
import math
import os

import torch

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "fabric_gb300_autotune.json")
# (tile pipelines per CTA, CTAs per SM, warpgroups per tile pipeline)
DECODER_CANDIDATES = [(1, 1, 1), (1, 2, 1), (1, 3, 1), (1, 4, 1), (2, 1, 1), (2, 2, 1), (4, 1, 1),
                      (1, 2, 2), (1, 3, 2), (1, 4, 2), (2, 1, 2), (2, 2, 2)]


def _key(fab, kind: str, precision: str, n_mat: int, n: int, extra: str = "") -> str:
    name = torch.cuda.get_device_name(fab.device)
    bucket = 1 << max(0, int(math.log2(max(n, 1))))
    return f"{name}|sm{fab.sm_count}|{kind}|{precision}|mat{n_mat}|n{bucket}|{extra}"


def _load(path):
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return {}


def _store(path, cache):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _current(fab):
    return getattr(fab, "launch_config", (0, 0, 0))


def tune_decoder(fab, g, precision: str = "fp16", candidates=None, reps: int = 50,
                 cache_path: str = DEFAULT_CACHE, force: bool = False) -> dict:
    """Pick (tile pipelines per CTA, CTAs per SM, warpgroups per pipeline) of
    the decoder for G-buffer `g` (neural state already prepared for
    `precision`)."""
    candidates = candidates or DECODER_CANDIDATES
    cache = _load(cache_path)
    key = _key(fab, "decoder", precision, fab.n_mat, g.n)
    lanes = _current(fab)[2]
    if not force and key in cache and "tile_warpgroups" in cache[key]:
        e = cache[key]
        fab.set_launch_config(e["ctas_per_sm"], e["warpgroups"], lanes, e["tile_warpgroups"])
        return e
    out = torch.empty((g.n, 3), dtype=torch.float32, device=fab.device)
    timings = {}
    for wg, c, h in candidates:
        fab.set_launch_config(c, wg, lanes, h)
        timings[(wg, c, h)] = _time(lambda: fab.shade_neural_prepared(g, precision, out_rgb=out), reps)
    wg, c, h = min(timings, key=timings.get)
    fab.set_launch_config(c, wg, lanes, h)
    cache[key] = {"warpgroups": wg, "ctas_per_sm": c, "tile_warpgroups": h, "ms": timings[(wg, c, h)],
                  "timings": {f"wg{k[0]}_cta{k[1]}_h{k[2]}": v for k, v in timings.items()}}
    _store(cache_path, cache)
    return cache[key]


def tune_plan(fab, plan, precision: str = "fp16", candidates=None, reps: int = 20,
              cache_path: str = DEFAULT_CACHE, force: bool = False) -> dict:
    """Pick the decoder's launch shape for a batched plan (its segments'
    tile count decides how the persistent CTAs share the work), with the
    neural state already prepared for `precision`."""
    candidates = candidates or DECODER_CANDIDATES
    cache = _load(cache_path)
    key = _key(fab, "plan", precision, fab.n_mat, plan.points, f"segs{plan.n_segs}")
    lanes = _current(fab)[2]
    if not force and key in cache and "tile_warpgroups" in cache[key]:
        e = cache[key]
        fab.set_launch_config(e["ctas_per_sm"], e["warpgroups"], lanes, e["tile_warpgroups"])
        return e
    timings = {}
    for wg, c, h in candidates:
        fab.set_launch_config(c, wg, lanes, h)
        timings[(wg, c, h)] = _time(lambda: plan.shade(precision), reps)
    wg, c, h = min(timings, key=timings.get)
    fab.set_launch_config(c, wg, lanes, h)
    cache[key] = {"warpgroups": wg, "ctas_per_sm": c, "tile_warpgroups": h, "ms": timings[(wg, c, h)],
                  "timings": {f"wg{k[0]}_cta{k[1]}_h{k[2]}": v for k, v in timings.items()}}
    _store(cache_path, cache)
    return cache[key]


def tune_reference(fab, g, spp_x: int, spp_y: int, candidates=(1, 2, 4, 8, 16, 32), reps: int = 3,
                   cache_path: str = DEFAULT_CACHE, force: bool = False) -> dict:
    """Pick the reference kernel's lanes per point for `g` at spp_x x spp_y."""
    cache = _load(cache_path)
    key = _key(fab, "reference", "fp32", fab.n_mat, g.n, f"spp{spp_x}x{spp_y}")
    ctas, wg, _ = _current(fab)
    h = getattr(fab, "tile_warpgroups", 0)
    if not force and key in cache:
        fab.set_launch_config(ctas, wg, cache[key]["lanes"], h)
        return cache[key]
    out = torch.empty((g.n, 3), dtype=torch.float32, device=fab.device)
    timings = {}
    for lanes in candidates:
        fab.set_launch_config(ctas, wg, lanes, h)
        timings[lanes] = _time(lambda: fab.shade_reference(g, spp_x, spp_y, 1, out_rgb=out), reps)
    best = min(timings, key=timings.get)
    fab.set_launch_config(ctas, wg, best, h)
    cache[key] = {"lanes": best, "ms": timings[best], "timings": {str(k): v for k, v in timings.items()}}
    _store(cache_path, cache)
    return cache[key]
