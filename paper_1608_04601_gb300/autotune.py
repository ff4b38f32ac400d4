"""Autotuner of the sweep's launch shape and the sort period.

Searches the sweep tile (threads per CTA x particles per thread), persistent CTAs per SM and
the stable-sort period K over a small grid, timing whole steps with CUDA events (L2 flushed
before each timed step, as in the benchmark), and caches the fastest choice per (workload,
precision, GPU) in a JSON file next to this module. The search itself only calls the library's
public API.
"""
from __future__ import annotations

import hashlib
import json
import os

from . import pic

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune_cache.json")

TILES = [(256, 4), (256, 2), (128, 4), (256, 8), (128, 8)]
CTAS = [0, 1]


def sort_periods(steps_per_period: int, choices=(1, 2, 4, 8, 16, 32, 64)) -> list:
    """Sort periods that divide the rf period (so one-period CUDA graphs stay periodic)."""
    return [k for k in choices if steps_per_period % k == 0]


def _key(gases, discharges, precision: str) -> str:
    import torch
    h = hashlib.sha256()
    for g in gases:
        h.update(f"{g.name}|{g.mass_kg}|{g.n_pts}|{g.de_eV}".encode())
    for d, gi in discharges:
        h.update(repr((gi, d.gas, d.gap_m, d.p_Pa, d.V_rf_V, d.n_cells, d.steps_per_period, d.n_e0, d.n_i0,
                       d.gamma_see)).encode())
    h.update(precision.encode())
    h.update(torch.cuda.get_device_name().encode())
    return h.hexdigest()[:20]


def time_config(gases, discharges, precision: str, block: int, ppt: int, ctas: int, sort_every: int,
                steps: int = 12, warmup: int = 4) -> float:
    """Mean device milliseconds per full step, L2 flushed before every step."""
    import torch
    stream = torch.cuda.Stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        sim = pic.Simulation(gases, discharges, precision=precision, sort_every=sort_every, block=block, ppt=ppt,
                             ctas_per_sm=ctas, stream="torch")
        sim.step(warmup)
        total = 0.0
        for k in range(steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.step(1)
            b.record(stream)
            b.synchronize()
            total += a.elapsed_time(b)
        sim.sync()
        sim.close()
    return total / steps


def autotune(gases, discharges, precision: str = "fp32", tiles=None, ctas=None, sorts=None, use_cache: bool = True,
             log=None) -> dict:
    """Returns {"block", "ppt", "ctas_per_sm", "sort_every", "ms_per_step"} of the fastest configuration."""
    if not isinstance(gases, (list, tuple)):
        gases = [gases]
    if not isinstance(discharges, (list, tuple)):
        discharges = [discharges]
    discharges = [d if isinstance(d, tuple) else (d, 0) for d in discharges]
    key = _key(gases, discharges, precision)
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except ValueError:
            cache = {}
        if key in cache:
            return cache[key]
    spp = discharges[0][0].steps_per_period
    best = None
    results = []
    for block, ppt in (tiles or TILES):
        for c in (ctas or CTAS):
            for k in (sorts or sort_periods(spp)):
                # warm-up through the first sort, then two whole sort periods
                ms = time_config(gases, discharges, precision, block, ppt, c, k, steps=max(12, 2 * k),
                                 warmup=max(4, k))
                results.append({"block": block, "ppt": ppt, "ctas_per_sm": c, "sort_every": k, "ms_per_step": ms})
                if log:
                    log(results[-1])
                if best is None or ms < best["ms_per_step"]:
                    best = results[-1]
    best = dict(best)
    best["searched"] = len(results)
    cache[key] = best
    try:
        json.dump(cache, open(CACHE, "w"), indent=1)
    except OSError:
        pass
    return best
