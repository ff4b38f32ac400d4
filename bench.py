#!/usr/bin/env python3
"""Benchmark of the PIC/MCC step on one GB300 (or N independent GPUs under torchrun).

Workload: Ar-like gas, 10 Pa, 2.5 cm gap, 300 V at 13.56 MHz, 512 cells, 2000 steps per rf
period, 1e6 electrons + 1e6 ions loaded uniform/Maxwellian (synthetic cross sections). One
benchmark step = one full PIC/MCC time step (sweep: gather, Verlet, MCC, walls, compaction,
deposit; births appended; Poisson; moments; the periodic cell sort when due).

The particle store (40 MB) would fit in L2, so L2 is flushed (a 256 MB write) before every
timed step, outside the timed region; each step is timed with CUDA events on the library's
stream (the torch stream handed to it). Prints one JSON line.
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

METRIC = "particle-steps/s/GPU FP32 vs FP64 path; rf periods to steady state warm vs cold"
UNIT = "particle-steps/s"
BYTES_PER_PS = {"fp32": 40, "fp64": 72}   # algorithmic HBM bytes per particle-step (read + write)


def workload(name: str = "c2"):
    """c2: the 1e6 + 1e6 Ar-like discharge the metric is quoted on; c3: the 2e7 + 2e7 He-like 500 V
    discharge; c3s: the same physics at 4e6 + 4e6 (160 MB per record buffer, beyond L2, small enough
    for a profiler capture)."""
    from paper_1608_04601_gb300.workloads import c2, c3
    if name == "c3":
        return c3()
    if name == "c3s":
        return c3().scaled(name="C3 physics at 4e6+4e6 (he-like 80Pa 5cm 500V N2048 gamma0.1)", n_e0=4_000_000,
                           n_i0=4_000_000)
    return c2()


def gas_for(d):
    from paper_1608_04601_gb300 import xsections as X
    return X.by_name(d.gas, eps_max_eV=d.eps_max_eV, de_eV=d.de_eV)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)"
    return 6800.0, "fallback 6.8 TB/s"


def sweep_source_hash() -> str:
    """Hash of the sweep's source: the kernel file up to the end of the sweep (the device code the
    sweep uses is defined before it; the kernels after it do not change it) and the two headers."""
    h = hashlib.sha256()
    src = open(os.path.join(ROOT, "paper_1608_04601_gb300", "csrc", "pic_kernels.cu"), "rb").read()
    h.update(src[:src.index(b"struct PSum")])
    for f in ("pic_device.cuh", "pic_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1608_04601_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(prec: str, kernel: str, workload_name: str):
    """DRAM bytes per particle-step of the sweep from the committed ncu summary, if it was taken on
    the current kernel source, the same launch shape and a workload of the same kind (the entry for
    the large discharge is a capture of the same physics at fewer particles, scaled per particle)."""
    p = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if not os.path.exists(p):
        return None
    j = json.load(open(p))
    key = prec + ("_c3" if workload_name.startswith("C3") else "")
    e = j.get(key)
    if not e or e.get("source_hash") != sweep_source_hash() or e.get("kernel") != kernel:
        return None
    return e


def sweep_roofline(r: dict, prec: str, block: int, ppt: int, workload_name: str) -> dict:
    """Roofline of the dominant kernel (the sweep) from one measure() result: algorithmic bytes per
    launch (40 B per particle-step in FP32, 72 B in FP64, times the particles one launch processes)
    over the average CUDA-event duration of the sweep launches of the timed steps."""
    peak, peak_note = peaks()
    launch_ps = r["ps"] / max(1, r["sweep_launches"])
    bytes_per_launch = BYTES_PER_PS[prec] * launch_ps
    avg_sweep_s = r["sweep_ms"] * 1e-3 / max(1, r["sweep_launches"])
    achieved = bytes_per_launch / avg_sweep_s / 1e9
    kernel = "k_sweep<%s,%d,%d>" % ("float" if prec == "fp32" else "double", block, ppt)
    tr = recorded_traffic(prec, kernel, workload_name)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": (tr["dram_bytes_per_particle"] * launch_ps) if tr else None,
            "traffic_source": tr.get("source") if tr else None,
            "kernel": kernel, "algorithmic_bytes_per_launch": bytes_per_launch, "peak_source": peak_note,
            "avg_launch_ms": avg_sweep_s * 1e3, "particles_per_launch": launch_ps,
            "kernel_timing": "CUDA events around every sweep launch, on the library's stream, inside the timed "
                             "steps (L2 flushed before every step)",
            "sweep_share_of_step": r["sweep_ms"] / r["total_ms"]}


class Clocks:
    """nvidia-smi samples (every 20 ms) of SM clock, power and throttle reasons. Each sample is
    stamped on arrival; summary() keeps those that arrived inside the marked timed window (widened
    by one sampling interval on each side)."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.samples = []
        self.t0 = self.t1 = None
        self.path = os.path.join(tempfile.gettempdir(), f"pic_bench_clocks_{os.getpid()}.csv")

    def _reader(self):
        for ln in self.proc.stdout:
            self.samples.append((time.time(), ln.strip()))

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "20"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._reader, daemon=True).start()
            t_end = time.time() + 5.0
            while not self.samples and time.time() < t_end:  # sampler running before the window opens
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def mark(self, start: bool):
        if start:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.05)
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except Exception:
                self.proc.kill()
            try:
                with open(self.path, "w") as f:
                    for t, ln in self.samples:
                        f.write(f"{t:.3f}, {ln}\n")
            except OSError:
                pass

    def summary(self):
        if not self.proc or self.t0 is None or self.t1 is None:
            return None
        sm, mx, reasons = [], [], set()
        for t, ln in self.samples:
            if not (self.t0 - 0.025 <= t <= self.t1 + 0.025):
                continue
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "window_s": round(self.t1 - self.t0, 3)}


def reduce_over_ranks(total_ms: float, ps: float, world: int, device: str):
    """Max of the timed duration and sum of the particle-steps over all ranks (no-op for one rank)."""
    if world <= 1:
        return total_ms, ps
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([ps], device=device, dtype=torch.float64)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())


def run_gpu(args, rank: int, world: int):
    import torch
    from paper_1608_04601_gb300 import pic

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    d0 = workload(args.workload)
    d = d0.scaled(seed=d0.seed + rank, discharge_id=rank)
    gas = gas_for(d)
    # a dedicated stream: the library, the L2 flush and the timing events all run on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def measure(prec: str, steps: int, warmup: int, sort_every: int, disc=None, disc_gas=None, leapfrog=False,
                setup=None):
        dd = disc if disc is not None else d
        sim = pic.Simulation(disc_gas if disc_gas is not None else gas, dd, seed=dd.seed, precision=prec,
                             sort_every=sort_every, stream="torch", block=args.block, ppt=args.ppt,
                             leapfrog=leapfrog)
        if setup is not None:
            setup(sim)
        if sort_every > 0:
            # the load draws positions in slot order, so the loaded store is unsorted; a long run spends
            # all but its first sort period on cell-sorted stores, so the store is sorted once here,
            # before the warm-up (the timed steps still include every periodic sort that falls in them)
            sim.sort()
        sim.step(warmup)
        sim.sync()
        electrons0 = sim.count(0, 0)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        counts = []
        sim.sweep_timing(True)
        torch.cuda.synchronize()
        with Clocks(dev) as clk:
            clk.mark(True)
            for k in range(steps):
                counts.append(sim.count(0, 0) + sim.count(0, 1))
                flush.fill_(float(k))
                ev[k][0].record(stream)
                sim.step(1)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            clk.mark(False)
        sim.sync()
        sweep_ms, launches = sim.sweep_timing(False)
        step_ms = [a.elapsed_time(b) for a, b in ev]
        total_ms = sum(step_ms)
        ps = float(sum(counts))
        out = {"ps": ps, "total_ms": total_ms, "sweep_ms": sweep_ms, "sweep_launches": launches,
               "clocks": clk.summary(), "counts": (counts[0], counts[-1]), "electrons0": electrons0}
        # kernels launched per step: the sweep and the post-sweep kernel (region starts, newborn
        # copies, store totals, field, moments, J(t)); when a sort is due its count, row-scan (with
        # the cell scan in its last CTA per store) and scatter (with the dense reset) kernels
        step0 = sim.step_index - steps
        sorts = sum(1 for n in range(step0 + 1, step0 + steps + 1) if sort_every > 0 and n % sort_every == 0)
        out["gpu_launches"] = 2 * steps + 3 * sorts
        sim.close()
        return out

    def measure_e2e(prec: str, steps: int, sort_every: int):
        """Through the public API with host buffers: every step uploads the whole particle state from
        pinned host memory, advances one step and reads the state and the moments back; host wall
        clock around all of it."""
        import numpy as np
        sim = pic.Simulation(gas, d, seed=d.seed, precision=prec, sort_every=sort_every, stream="torch",
                             block=args.block, ppt=args.ppt)
        if sort_every > 0:
            sim.sort()
        sim.step(2)
        rdt = np.float32 if prec == "fp32" else np.float64
        tdt = torch.float32 if prec == "fp32" else torch.float64
        cap = [2 * max(sim.count(0, sp), 1) for sp in (0, 1)]
        pinned = []  # keep the torch tensors alive
        host = []
        for sp in (0, 1):
            t_c = torch.empty(cap[sp], dtype=torch.int32, pin_memory=True)
            t_r = [torch.empty(cap[sp], dtype=tdt, pin_memory=True) for _ in range(4)]
            pinned.append((t_c, t_r))
            host.append({"c": t_c.numpy(), "f": t_r[0].numpy(), "vx": t_r[1].numpy(), "vy": t_r[2].numpy(),
                         "vz": t_r[3].numpy()})
        st = [sim.get_state(0, sp, out=host[sp]) for sp in (0, 1)]
        rb = 4 if prec == "fp32" else 8
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ps = 0
        h2d = d2h = 0
        for _ in range(steps):
            for sp in (0, 1):
                sim.set_state(0, sp, st[sp])
                h2d += st[sp]["c"].size * (4 + 4 * rb)
            sim.step(1)
            st = [sim.get_state(0, sp, out=host[sp]) for sp in (0, 1)]
            m = sim.moments(0)
            ps += sum(x["c"].size for x in st)
            d2h += sum(x["c"].size * (4 + 4 * rb) for x in st) + 3 * 8 * m["n_e"].size
        dt = time.perf_counter() - t0
        sim.close()
        # the host link on its own: one plain pinned copy of a step's upload size in each direction
        nb = int(h2d / steps)
        hbuf = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
        dbuf = torch.empty(nb, dtype=torch.uint8, device="cuda")
        link = {}
        for name, (dst, src) in (("h2d", (dbuf, hbuf)), ("d2h", (hbuf, dbuf))):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(10):
                dst.copy_(src, non_blocking=True)
            b.record(stream)
            b.synchronize()
            link[name] = 10 * nb / (a.elapsed_time(b) * 1e-3) / 1e9
        del hbuf, dbuf
        floor_ms = (h2d / steps / link["h2d"] + d2h / steps / link["d2h"]) / 1e6
        return {"value": ps / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d / steps),
                "d2h_bytes_per_step": int(d2h / steps), "host_memory": "pinned",
                "per_step": "upload of the whole state, one step, download of the state and the moments",
                "ms_per_step": dt * 1e3 / steps,
                "link_gbs": {"h2d": link["h2d"], "d2h": link["d2h"],
                             "note": "one plain pinned copy of the step's upload size, 10 repetitions"},
                "copy_floor_ms": floor_ms}

    def measure_batch(steps: int, warmup: int, sort_every: int):
        """32 discharges of uneven counts (He/Ar-like x 4 pressures x 4 voltages, 1e5..4e6 each) in one
        persistent sweep launch per step, against the same discharges advanced one at a time."""
        from paper_1608_04601_gb300 import xsections as X
        from paper_1608_04601_gb300.workloads import c4
        ds = c4(seed=1)
        gases = [X.he_like(eps_max_eV=1000.0), X.ar_like(eps_max_eV=1000.0)]
        pairs = [(dd, 0 if dd.gas == "he" else 1) for dd in ds]

        def timed(sim, n):
            sim.step(warmup)
            sim.sync()
            tot, ps = 0.0, 0.0
            for k in range(n):
                c = sum(sim.count(i, sp) for i in range(len(sim.N)) for sp in (0, 1))
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sim.step(1)
                b.record(stream)
                b.synchronize()
                tot += a.elapsed_time(b)
                ps += c
            return tot, ps

        sim = pic.Simulation(gases, pairs, seed=1, precision="fp32", sort_every=sort_every, stream="torch",
                             block=args.block, ppt=args.ppt)
        t_b, ps_b = timed(sim, steps)
        sim.close()
        t_s, ps_s = 0.0, 0.0
        for pr in pairs:
            one = pic.Simulation(gases, [pr], seed=1, precision="fp32", sort_every=sort_every, stream="torch",
                                 block=args.block, ppt=args.ppt)
            t, ps = timed(one, max(2, steps // 4))
            one.close()
            t_s += t / max(2, steps // 4)
            ps_s += ps / max(2, steps // 4)
        return {"workload": "32 discharges: {He,Ar}-like x {10,20,40,80} Pa x {150,250,350,500} V, 2.5 cm, "
                            "512 cells, 1e5..4e6 superparticles per species each (seed 1)",
                "value": ps_b / (t_b * 1e-3), "unit": UNIT, "ms_per_step": t_b / steps,
                "one_at_a_time": {"value": ps_s / (t_s * 1e-3), "ms_per_step": t_s},
                "particles": int(ps_b / steps)}

    tuned = None
    if args.autotune:
        # small search of the launch shape and the sort period on this workload (whole steps, L2 flushed)
        from paper_1608_04601_gb300 import autotune
        tuned = autotune.autotune([gas], [(d, 0)], "fp32", tiles=[(256, 2), (256, 4), (128, 4)], ctas=[0],
                                  sorts=[8, 16], use_cache=False)
        args.block, args.ppt, args.sort_every = tuned["block"], tuned["ppt"], tuned["sort_every"]
    sort_every = args.sort_every
    main = measure("fp32", args.steps, args.warmup, sort_every)
    fp64 = e2e = batch = c3 = warm = None
    if not args.quick:
        fp64 = measure("fp64", max(4, args.steps // 2), max(3, args.warmup), sort_every)
        e2e = measure_e2e("fp32", max(3, min(10, args.steps)), sort_every)
        batch = measure_batch(max(4, args.steps // 2), 3, sort_every) if not args.no_batch else None
    if args.c3 and not args.quick and world == 1 and args.workload != "c3":
        # the large workload: 2e7 + 2e7 particles, 2048 cells, secondary emission (800 MB per record
        # buffer, far beyond L2): its own step rate and its own sweep roofline
        dc = workload("c3")
        r3 = measure("fp32", 20, 6, sort_every, disc=dc, disc_gas=gas_for(dc))
        c3 = {"workload": dc.name, "value": r3["ps"] / (r3["total_ms"] * 1e-3), "unit": UNIT,
              "ms_per_step": r3["total_ms"] / 20, "steps": 20, "warmup": 6,
              "particles": int(r3["ps"] / max(1, r3["sweep_launches"])), "clocks": r3["clocks"],
              "roofline": sweep_roofline(r3, "fp32", args.block, args.ppt, dc.name)}
    rows_f = None
    if not args.quick and not args.no_rows_f:
        # the widened rows on the same workload and launch shape: the leapfrog variant (f2); the
        # kinetic diagnostics (f1) taken at every step, whose extra step time is the diagnostics
        # kernel's (20 B read per electron: cell and record); the current-driven mode (f3)
        n_f = max(4, args.steps // 2)
        lf = measure("fp32", n_f, args.warmup, sort_every, leapfrog=True)
        base = measure("fp32", n_f, args.warmup, sort_every)
        dg = measure("fp32", n_f, args.warmup, sort_every,
                     setup=lambda sim: sim.set_diagnostics(period_steps=1, phase_step=0, sample_every=1,
                                                           eedf_bins=400, eedf_de_eV=0.25, fast_eV=d.V_rf_V / 4))
        dr = measure("fp32", n_f, args.warmup, sort_every, setup=lambda sim: sim.set_current_drive(0, 10.0))
        peak, peak_note = peaks()
        extra_ms = (dg["total_ms"] - base["total_ms"]) / n_f
        electrons = float(dg["electrons0"])  # electrons at the first timed step
        diag_gbs = 20.0 * electrons / (extra_ms * 1e-3) / 1e9 if extra_ms > 0 else None
        P = d.steps_per_period
        rows_f = {
            "leapfrog": {"value": lf["ps"] / (lf["total_ms"] * 1e-3), "unit": UNIT, "ms_per_step": lf["total_ms"] / n_f,
                         "roofline": sweep_roofline(lf, "fp32", args.block, args.ppt, d0.name)},
            "verlet_same_run": {"value": base["ps"] / (base["total_ms"] * 1e-3), "unit": UNIT,
                                "ms_per_step": base["total_ms"] / n_f},
            "diagnostics_every_step": {
                "value": dg["ps"] / (dg["total_ms"] * 1e-3), "unit": UNIT, "ms_per_step": dg["total_ms"] / n_f,
                "kernel_ms_per_launch": extra_ms, "electrons_per_launch": electrons,
                "achieved_gbs": diag_gbs, "frac": (diag_gbs / peak) if diag_gbs else None, "peak": peak,
                "peak_source": peak_note,
                "kernel_timing": "step-time difference against the same steps without diagnostics (CUDA events)",
                "overhead_at_paper_schedule": (extra_ms * (1.0 / P + 1.0 / 16)) / (base["total_ms"] / n_f),
                "schedule_note": "snapshot once per rf period and an EEDF sample every 16 steps"},
            "current_drive": {"value": dr["ps"] / (dr["total_ms"] * 1e-3), "unit": UNIT,
                              "ms_per_step": dr["total_ms"] / n_f, "J0_A_m2": 10.0},
        }
    if args.warm_start and not args.quick and world == 1:
        # rf periods to the steady state from the homogeneous start vs from the network's profiles
        from paper_1608_04601_gb300 import warmstart
        warm = warmstart.experiment(n_train=args.ws_train, n_test=args.ws_test, periods=700, train_periods=700,
                                    avg=200)

    # aggregate over ranks: the job took as long as its slowest rank, and did every rank's work
    total_ms, ps = reduce_over_ranks(main["total_ms"], main["ps"], world, "cuda")
    value = ps / (total_ms * 1e-3)
    roofline = sweep_roofline(main, "fp32", args.block, args.ppt, d0.name)

    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": d0.name, "cells": d0.n_cells, "particles_per_species": d0.n_e0,
                      "steps_per_period": d0.steps_per_period, "sort_every": sort_every,
                      "block": args.block, "ppt": args.ppt, "parallelism": f"replicas{world}" if world > 1 else "1gpu",
                      "l2": "flushed (256 MB write) before every timed step",
                      "autotuned": tuned},
           "roofline": roofline, "clocks": main["clocks"], "gpu_launches": main["gpu_launches"]}
    if sort_every > 0:
        res["config"]["initial_sort"] = "the loaded store is sorted by cell once, before the warm-up"
    if fp64:
        res["fp64_path"] = {"value": fp64["ps"] / (fp64["total_ms"] * 1e-3), "unit": UNIT,
                            "ms_per_step": fp64["total_ms"] / max(1, max(4, args.steps // 2)),
                            "sweep_gbs": BYTES_PER_PS["fp64"] * fp64["ps"] / (fp64["sweep_ms"] * 1e-3) / 1e9,
                            "bytes_per_particle_step": BYTES_PER_PS["fp64"]}
    if e2e:
        res["e2e"] = e2e
    if batch:
        res["batch_c4"] = batch
    if c3:
        res["c3"] = c3
    if warm:
        res["warm_start"] = warm
    if rows_f:
        res["rows_f"] = rows_f
    return res


def run_cpu_baseline(args):
    """The FP64 oracle as it stands, single thread, on a bounded sample of the same workload."""
    from oracle import oracle as O
    d = workload(args.workload)
    gas = gas_for(d)
    t0 = time.perf_counter()
    o = O.Oracle(gas, d, "f64", sort_every=args.sort_every)
    t_load = time.perf_counter() - t0
    n_steps = args.cpu_steps
    n0 = o.count(0) + o.count(1)
    t0 = time.perf_counter()
    ps = 0
    for _ in range(n_steps):
        ps += o.count(0) + o.count(1)
        o.step(1)
    dt = time.perf_counter() - t0
    return {"value": ps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{d.name}: full load ({n0} particles, {t_load:.1f} s), {n_steps} FP64 steps, {dt:.1f} s"}


def _oracle_copy(name, sort_every, n_steps, did, barrier, q):
    """One independent copy of the workload in the oracle (its own discharge id, so its own random
    streams), timed after every copy has loaded."""
    from oracle import oracle as O
    d = workload(name).scaled(discharge_id=did)
    o = O.Oracle(gas_for(d), d, "f64", sort_every=sort_every)
    barrier.wait(timeout=600)
    t0 = time.monotonic()
    ps = 0
    for _ in range(n_steps):
        ps += o.count(0) + o.count(1)
        o.step(1)
    q.put((ps, t0, time.monotonic()))


def run_cpu_baseline_all_cores(args):
    """The FP64 oracle as it stands on every host core: one independent copy of the workload per
    core, in processes started by spawn; throughput = all copies' particle-steps over the wall time
    from the first copy's start to the last copy's end."""
    import multiprocessing as mp
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(cores), ctx.Queue()
    n_steps = max(4, args.cpu_steps)
    procs = [ctx.Process(target=_oracle_copy, args=(args.workload, args.sort_every, n_steps, k + 1, barrier, q))
             for k in range(cores)]
    for p in procs:
        p.start()
    try:
        res = [q.get(timeout=900) for _ in procs]
    except Exception as e:  # a copy failed to start or to finish: no all-core figure
        for p in procs:
            p.kill()
        return {"unavailable": f"all-core oracle run failed: {type(e).__name__}"}
    for p in procs:
        p.join()
    ps = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    d = workload(args.workload)
    return {"value": ps / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} independent copies of {d.name} (one per core), {n_steps} FP64 steps each, "
                      f"{wall:.1f} s wall"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--sort-every", type=int, default=16)
    ap.add_argument("--block", type=int, default=256)
    ap.add_argument("--ppt", type=int, default=4)
    ap.add_argument("--cpu-steps", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c3s"],
                    help="measured workload: c2 (the metric's configuration), c3, or c3s (C3 physics at 4e6+4e6)")
    ap.add_argument("--quick", action="store_true",
                    help="main measurement only (no FP64 path, end-to-end, batch, large workload, warm start)")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-rows-f", action="store_true",
                    help="skip the leapfrog, diagnostics and current-drive measurements")
    ap.add_argument("--no-c3", dest="c3", action="store_false", help="skip the 2e7 + 2e7 particle workload")
    ap.add_argument("--no-warm-start", dest="warm_start", action="store_false",
                    help="skip the warm-start experiment (training runs, network training, cold vs warm runs)")
    ap.add_argument("--ws-train", type=int, default=128, help="training discharges of the warm-start experiment")
    ap.add_argument("--ws-test", type=int, default=24, help="held-out discharges of the warm-start experiment")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="use --block/--ppt/--sort-every as given instead of searching")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        if rank != 0:
            return
        from oracle import oracle as O
        O.build()
        d = workload(args.workload)
        gas = gas_for(d)
        o = O.Oracle(gas, d, "f64", sort_every=args.sort_every)
        o.step(args.warmup)
        ps = 0
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ps += o.count(0) + o.count(1)
            o.step(1)
        dt = time.perf_counter() - t0
        v = ps / dt
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": d.name, "sort_every": args.sort_every},
                          "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                           "sample": f"{d.name}, full population, {args.steps} FP64 steps"},
                          "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
        dist.barrier()
    import __graft_entry__ as g
    g.build()
    res = run_gpu(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline and not args.quick:
            res["cpu_baseline"] = run_cpu_baseline(args)
            res["cpu_baseline_all_cores"] = run_cpu_baseline_all_cores(args)
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
