"""Warm start of PIC/MCC runs from network-predicted periodic-state profiles.

The paper notes that its PIC runs needed about 1000 to 4000 rf periods to reach the periodic
state from a homogeneous start, and proposes initial values closer to that state (section
"Numerical parameters and initial values"). This module does that end to end with the library:

1. a family of discharges (He-like gas, pressure, voltage, gap, rf frequency) is run with the
   batched PIC/MCC step from the homogeneous start, and the profiles n_e, n_i and mean electron
   energy, averaged over the last rf periods, are resampled to 256 points;
2. the warm-start network (include/mlp.h: 5 inputs, 4 hidden layers of 512, 768 outputs) is
   trained on them on the GPU;
3. for held-out discharges, the number of rf periods to the steady state (steady.py criterion)
   is compared between the homogeneous start and particles sampled from the network's prediction
   (pic_load_profiles).

Profiles travel as log10(n / 1e14 m^-3) (densities floored at 1e12 m^-3) and mean energy / 10 eV.
"""
from __future__ import annotations

import math

import numpy as np

from . import pic, xsections as X
from .steady import steady_period
from .workloads import Discharge

NPTS = 256
SIZES = [5, 512, 512, 512, 512, 3 * NPTS]
GAS = "he"


def family(n: int, seed: int, first_id: int = 0) -> list:
    """n He-like discharges, parameters uniform (log-uniform pressure) in the family's box."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        p = math.exp(rng.uniform(math.log(16.0), math.log(28.0)))
        V = rng.uniform(200.0, 500.0)
        gap = rng.uniform(0.02, 0.03)
        f = rng.uniform(10e6, 16e6)
        out.append(Discharge(f"ws{first_id + k}", GAS, gap, p, V, 128, 400, 20000, 20000, 4e14, f_rf_Hz=f,
                             periods=400, discharge_id=first_id + k, seed=seed))
    return out


def features(d: Discharge) -> np.ndarray:
    """Network inputs: gas id, log pressure, voltage, gap and frequency, scaled to O(1)."""
    return np.array([0.0 if d.gas == "he" else 1.0, math.log(d.p_Pa / 20.0), d.V_rf_V / 300.0 - 1.0,
                     d.gap_m / 0.025 - 1.0, d.f_rf_Hz / 13e6 - 1.0], np.float32)


def to_target(m: dict, d: Discharge) -> np.ndarray:
    z = np.linspace(0.0, d.gap_m, d.n_cells + 1)
    s = np.linspace(0.0, d.gap_m, NPTS)
    ne = np.interp(s, z, m["n_e"])
    ni = np.interp(s, z, m["n_i"])
    eps = np.interp(s, z, m["mean_eps"])
    return np.concatenate([np.log10(np.maximum(ne, 1e12) / 1e14), np.log10(np.maximum(ni, 1e12) / 1e14),
                           eps / 10.0]).astype(np.float32)


def from_target(y: np.ndarray) -> np.ndarray:
    """(3, NPTS) profiles n_e, n_i (m^-3) and mean energy (eV) from network outputs."""
    y = np.asarray(y, np.float64).reshape(3, NPTS)
    return np.stack([1e14 * 10.0 ** y[0], 1e14 * 10.0 ** y[1], np.maximum(10.0 * y[2], 0.1)])


def _gas():
    return X.he_like(eps_max_eV=800.0, de_eV=1e-2)


def run_batch(ds: list, periods: int, avg: int, warm=None, cap: int = 1000000) -> dict:
    """Runs the discharges together (one persistent sweep per step, one CUDA graph per rf period).
    warm: optional (len(ds), 3, P) profiles to load instead of the homogeneous start.
    Returns per discharge the profiles averaged over the last `avg` periods, the per-period mean
    counts and the period at which the steady-state criterion first held."""
    sim = pic.Simulation(_gas(), ds, precision="fp32", sort_every=8, use_graph=True, load=warm is None,
                         capacity=[(cap, cap)] * len(ds))
    if warm is not None:
        sim.load_profiles(np.asarray(warm, np.float64))
    spp = ds[0].steps_per_period
    sim.step((periods - avg) * spp)
    sim.reset_moments()
    sim.step(avg * spp)
    sim.sync()
    out = {"targets": [], "counts": [], "steady": []}
    for i, d in enumerate(ds):
        m = sim.moments(i)
        c = sim.period_counts(i)
        out["targets"].append(to_target(m, d))
        out["counts"].append(c)
        out["steady"].append(steady_period(c))
    sim.close()
    return out


def generate(ds: list, periods: int = 400, avg: int = 100, batch: int = 64) -> dict:
    res = {"targets": [], "counts": [], "steady": []}
    for k in range(0, len(ds), batch):
        r = run_batch(ds[k:k + batch], periods, avg)
        for key in res:
            res[key] += r[key]
    res["features"] = [features(d) for d in ds]
    return res


def train(Xf: np.ndarray, Y: np.ndarray, steps: int = 3000, lr: float = 1e-3, seed: int = 1):
    """Full-batch Adam on the GPU; returns the network and the loss history (every 100 steps)."""
    import torch
    from .mlp import MLP
    net = MLP(SIZES, max_batch=len(Xf), seed=seed)
    x = torch.as_tensor(np.asarray(Xf, np.float32), device="cuda")
    t = torch.as_tensor(np.asarray(Y, np.float32), device="cuda")
    hist = []
    for k in range(steps):
        lr_k = lr * (0.1 ** (k / steps))  # exponential decay to lr / 10
        if k % 100 == 0:
            hist.append(net.train_step(x, t, lr_k))
        else:
            net.train_step(x, t, lr_k, sync=False)
    hist.append(net.loss_grad(x, t))
    return net, hist


def predict(net, ds: list) -> np.ndarray:
    y = net.forward(np.stack([features(d) for d in ds])).cpu().numpy()
    return np.stack([from_target(r) for r in y])


def profile_error(pred: np.ndarray, target: np.ndarray) -> dict:
    """Relative L2 errors of predicted n_e, n_i and mean energy against PIC profiles (network units
    converted back to physical ones)."""
    out = {}
    tp = np.stack([from_target(t) for t in target])
    for k, name in enumerate(("n_e", "n_i", "mean_eps")):
        a, b = pred[:, k], tp[:, k]
        out[name] = float(np.median(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))
    return out


def experiment(n_train: int = 128, n_test: int = 16, periods: int = 800, train_periods: int = 600, avg: int = 100,
               train_steps: int = 3000, seed: int = 7) -> dict:
    """Data generation, training, and cold vs warm periods to steady state on held-out discharges."""
    import time
    t0 = time.time()
    tr = generate(family(n_train, seed), periods=train_periods, avg=avg)
    t1 = time.time()
    net, hist = train(np.stack(tr["features"]), np.stack(tr["targets"]), train_steps)
    t2 = time.time()
    test = family(n_test, seed + 1, first_id=10000)
    cold = run_batch(test, periods, avg)
    warm_prof = predict(net, test)
    warm = run_batch(test, periods, avg, warm=warm_prof)
    t3 = time.time()
    net.close()

    def med(v):
        v = [periods if s is None else s for s in v]  # never steady within the run: counted as the run length
        return float(np.median(v))

    return {"family": "He-like, 16-28 Pa (log-uniform), 200-500 V, 2-3 cm, 10-16 MHz, 128 cells, 400 steps/period, "
                      "2e4 + 2e4 initial superparticles at 4e14 m^-3",
            "train_runs": n_train, "test_runs": n_test, "train_periods": train_periods, "test_periods": periods,
            "avg_periods": avg,
            "train_loss_first_last": [hist[0], hist[-1]],
            "profile_rel_l2_median": profile_error(warm_prof, np.stack(cold["targets"])),
            "periods_to_steady_cold": [None if s is None else int(s) for s in cold["steady"]],
            "periods_to_steady_warm": [None if s is None else int(s) for s in warm["steady"]],
            "median_periods_cold": med(cold["steady"]), "median_periods_warm": med(warm["steady"]),
            "seconds": {"generate": round(t1 - t0, 1), "train": round(t2 - t1, 1), "evaluate": round(t3 - t2, 1)}}
