"""Warm start of PIC/MCC runs from network-predicted periodic-state profiles.

The paper notes that its PIC runs needed about 1000 to 4000 rf periods to reach the periodic
state from a homogeneous start, and proposes initial values closer to that state (section
"Numerical parameters and initial values"). This module does that end to end with the library:

1. a family of discharges (He-like gas, pressure, voltage, gap, rf frequency) is run with the
   batched PIC/MCC step from the homogeneous start, and the profiles n_e, n_i and mean electron
   energy, averaged over the last rf periods, are resampled to 256 points;
2. the warm-start network (include/mlp.h: 5 inputs, 4 hidden layers of 512, 768 outputs) is
   trained on them on the GPU;
3. for held-out discharges, the number of rf periods to the steady state (the library's
   criterion, pic_moments) is compared between the homogeneous start (FP64 path) and particles
   sampled from the network's prediction (pic_load_profiles, FP32 path), and the two steady
   states are compared with each other.

Profiles travel as log10(n / 1e14 m^-3) (densities floored at 1e12 m^-3) and mean energy / 10 eV.
"""
from __future__ import annotations

import math

import numpy as np

from . import pic, xsections as X
from .workloads import Discharge

NPTS = 256
SIZES = [5, 512, 512, 512, 512, 3 * NPTS]
GAS = "he"


# The family's box: self-sustained discharges of the synthetic He-like gas that settle within about
# 1000 rf periods (at lower pressure they die out; with wider gaps many keep growing for longer).
P_RANGE, V_RANGE, GAP_RANGE, F_RANGE = (22.0, 30.0), (300.0, 450.0), (0.020, 0.024), (12e6, 16e6)


def family(n: int, seed: int, first_id: int = 0) -> list:
    """n He-like discharges, parameters uniform (log-uniform pressure) in the family's box."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        p = math.exp(rng.uniform(math.log(P_RANGE[0]), math.log(P_RANGE[1])))
        V = rng.uniform(*V_RANGE)
        gap = rng.uniform(*GAP_RANGE)
        f = rng.uniform(*F_RANGE)
        out.append(Discharge(f"ws{first_id + k}", GAS, gap, p, V, 128, 400, 20000, 20000, 4e14, f_rf_Hz=f,
                             periods=400, discharge_id=first_id + k, seed=seed))
    return out


def features(d: Discharge) -> np.ndarray:
    """Network inputs: gas id, log pressure, voltage, gap and frequency, scaled to O(1)."""
    return np.array([0.0 if d.gas == "he" else 1.0, math.log(d.p_Pa / 20.0), d.V_rf_V / 300.0 - 1.0,
                     d.gap_m / 0.025 - 1.0, d.f_rf_Hz / 13e6 - 1.0], np.float32)


def encode(prof: np.ndarray) -> np.ndarray:
    """Network outputs for (3, NPTS) physical profiles n_e, n_i (m^-3), mean energy (eV)."""
    ne, ni, eps = np.asarray(prof, np.float64)
    return np.concatenate([np.log10(np.maximum(ne, 1e12) / 1e14), np.log10(np.maximum(ni, 1e12) / 1e14),
                           eps / 10.0]).astype(np.float32)


def to_target(m: dict, d: Discharge) -> np.ndarray:
    """Network outputs for the moments m (N+1 nodes) of discharge d."""
    return encode(_resample(m, d))


def from_target(y: np.ndarray) -> np.ndarray:
    """(3, NPTS) profiles n_e, n_i (m^-3) and mean energy (eV) from network outputs."""
    y = np.asarray(y, np.float64).reshape(3, NPTS)
    return np.stack([1e14 * 10.0 ** y[0], 1e14 * 10.0 ** y[1], np.maximum(10.0 * y[2], 0.1)])


def _gas():
    return X.he_like(eps_max_eV=800.0, de_eV=1e-2)


def _resample(m: dict, d: Discharge) -> np.ndarray:
    """(3, NPTS) physical profiles on the uniform grid of the network."""
    z = np.linspace(0.0, d.gap_m, d.n_cells + 1)
    s = np.linspace(0.0, d.gap_m, NPTS)
    return np.stack([np.interp(s, z, m[k]) for k in ("n_e", "n_i", "mean_eps")])


def run_batch(ds: list, periods: int, avg: int, warm=None, cap: int = 1000000, precision: str = "fp32",
              blocks: int = 4) -> dict:
    """Runs the discharges together (one persistent sweep per step, one CUDA graph per rf period).
    warm: optional (len(ds), 3, P) profiles to load instead of the homogeneous start.
    Returns per discharge: the profiles averaged over the last `avg` periods (network units and
    physical), the same over `blocks` consecutive blocks of those periods (their scatter is the
    run's own noise), the per-period mean counts, and the library's steady-state period."""
    sim = pic.Simulation(_gas(), ds, precision=precision, sort_every=8, use_graph=True, load=warm is None,
                         capacity=[(cap, cap)] * len(ds))
    if warm is not None:
        sim.load_profiles(np.asarray(warm, np.float64))
    spp = ds[0].steps_per_period
    sim.step((periods - avg) * spp)
    blk = [[] for _ in ds]
    for b in range(blocks):
        sim.reset_moments()
        sim.step((avg // blocks) * spp)
        for i, d in enumerate(ds):
            blk[i].append(_resample(sim.moments(i), d))
    sim.sync()
    out = {"targets": [], "profiles": [], "blocks": [], "counts": [], "steady": []}
    for i, d in enumerate(ds):
        m = sim.moments(i)
        prof = np.mean(blk[i], axis=0)
        out["profiles"].append(prof)
        out["blocks"].append(np.stack(blk[i]))
        out["targets"].append(encode(prof))
        out["counts"].append(sim.period_counts(i))
        out["steady"].append(m["steady_period"])
    sim.close()
    return out


def generate(ds: list, periods: int = 600, avg: int = 100, batch: int = 64) -> dict:
    """Training data: runs of the family from the homogeneous start; only the runs that the
    library declares steady within `periods` are kept (their profiles are averaged over the last
    `avg` periods, after the steady state was reached when it came early enough)."""
    res = {"targets": [], "features": [], "steady": [], "dropped": 0}
    for k in range(0, len(ds), batch):
        part = ds[k:k + batch]
        r = run_batch(part, periods, avg)
        for d, t, st in zip(part, r["targets"], r["steady"]):
            if st is None or st > periods - avg:
                res["dropped"] += 1
                continue
            res["targets"].append(t)
            res["features"].append(features(d))
            res["steady"].append(st)
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
    """Relative L2 errors of predicted n_e, n_i and mean energy against PIC profiles."""
    out = {}
    for k, name in enumerate(("n_e", "n_i", "mean_eps")):
        a, b = pred[:, k], target[:, k]
        nb = np.linalg.norm(b, axis=1)
        live = nb > 0  # runs that died out have no profile to compare with
        out[name] = float(np.median(np.linalg.norm(a - b, axis=1)[live] / nb[live])) if live.any() else float("nan")
    return out


def agreement(a: dict, b: dict, i: int) -> dict:
    """Steady-state profiles of run i of two run_batch results: relative L2 distance of the means
    (densities, and mean energy away from the two wall points) against 3 sigma, sigma from the
    scatter of each run's block means about its mean."""
    out = {}
    for k, name in enumerate(("n_e", "n_i", "mean_eps")):
        sl = slice(2, -2) if name == "mean_eps" else slice(None)
        A, B = a["blocks"][i][:, k, sl], b["blocks"][i][:, k, sl]
        am, bm = A.mean(0), B.mean(0)
        nb = A.shape[0]
        sa = math.sqrt(np.sum((A - am) ** 2) / (nb - 1) / nb)   # standard error of the mean profile (L2)
        sb = math.sqrt(np.sum((B - bm) ** 2) / (nb - 1) / nb)
        nb_ = float(np.linalg.norm(bm))
        if not nb_ > 0 or not float(np.linalg.norm(am)) > 0:  # a run that died out has no steady profile
            out[name] = {"rel_l2": float("inf"), "sigma": 0.0, "ok": False}
            continue
        dist = float(np.linalg.norm(am - bm) / nb_)
        sigma = math.sqrt(sa ** 2 + sb ** 2) / nb_
        out[name] = {"rel_l2": dist, "sigma": sigma, "ok": dist <= max(0.03, 3 * sigma)}
    return out


def sign_test_p(wins: int, n: int) -> float:
    """One-sided sign test: probability of at least `wins` successes in n fair coin flips."""
    return float(sum(math.comb(n, k) for k in range(wins, n + 1)) / 2.0 ** n)


def experiment(n_train: int = 48, n_test: int = 8, periods: int = 700, train_periods: int = 700, avg: int = 100,
               train_steps: int = 3000, seed: int = 7, cold_precision: str = "fp64") -> dict:
    """Data generation, training, and cold vs warm periods to steady state on held-out discharges
    (cold: the homogeneous start on the `cold_precision` path; warm: particles sampled from the
    network's profiles, FP32 path), with the agreement of the two steady states."""
    import time
    t0 = time.time()
    tr = generate(family(n_train, seed), periods=train_periods, avg=avg)
    t1 = time.time()
    net, hist = train(np.stack(tr["features"]), np.stack(tr["targets"]), train_steps)
    t2 = time.time()
    test = family(n_test, seed + 1, first_id=10000)
    cold = run_batch(test, periods, avg, precision=cold_precision)
    warm_prof = predict(net, test)
    warm = run_batch(test, periods, avg, warm=warm_prof)
    t3 = time.time()
    net.close()
    runlen = lambda s: periods + 1 if s is None else s  # never steady within the run: beyond its length
    # a discharge that dies out (no electrons left) has no steady state to reach: such a pair is a tie
    dead = [cold["counts"][i][-1][0] == 0 or warm["counts"][i][-1][0] == 0 for i in range(n_test)]
    pairs = [(c, w) for c, w, x in zip(cold["steady"], warm["steady"], dead) if not x]
    wins = sum(1 for c, w in pairs if runlen(w) < runlen(c))
    ties = n_test - sum(1 for c, w in pairs if runlen(w) != runlen(c))
    agree = [agreement(warm, cold, i) for i in range(n_test)]
    both = [i for i in range(n_test) if cold["steady"][i] is not None and warm["steady"][i] is not None and not dead[i]]
    return {"family": "He-like, 22-30 Pa (log-uniform), 300-450 V, 2.0-2.4 cm, 12-16 MHz, 128 cells, "
                      "400 steps/period, 2e4 + 2e4 initial superparticles at 4e14 m^-3",
            "train_runs": n_train, "train_runs_steady": len(tr["targets"]), "test_runs": n_test,
            "train_periods": train_periods, "test_periods": periods, "avg_periods": avg,
            "cold_path": cold_precision, "warm_path": "fp32",
            "train_loss_first_last": [hist[0], hist[-1]],
            "profile_rel_l2_median": profile_error(warm_prof, np.stack(cold["profiles"])),
            "periods_to_steady_cold": [None if s is None else int(s) for s in cold["steady"]],
            "periods_to_steady_warm": [None if s is None else int(s) for s in warm["steady"]],
            "median_periods_cold": float(np.median([runlen(s) for s in cold["steady"]])),
            "median_periods_warm": float(np.median([runlen(s) for s in warm["steady"]])),
            "warm_faster": wins, "ties": ties, "died_out": int(sum(dead)),
            "sign_test_p": sign_test_p(wins, n_test - ties),
            "steady_state_agreement": [{k: v["rel_l2"] for k, v in a.items()} for a in agree],
            "steady_state_agree_all": bool(all(all(v["ok"] for v in agree[i].values()) for i in both)),
            "steady_state_compared": len(both),
            "seconds": {"generate": round(t1 - t0, 1), "train": round(t2 - t1, 1), "evaluate": round(t3 - t2, 1)}}
