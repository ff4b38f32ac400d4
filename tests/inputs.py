"""Seeded synthetic inputs shared by the oracle pins and the GPU parity tests.

Nothing here does any PIC/MCC arithmetic: it only draws particle states and
node fields with numpy's seeded generator and builds parameter records.
"""
from __future__ import annotations

import numpy as np

from paper_1608_04601_gb300.workloads import Discharge

E_CH = 1.602176634e-19
M_E = 9.1093837015e-31
K_B = 1.380649e-23
EPS0 = 8.8541878128e-12
AMU = 1.66053906660e-27


def discharge(**kw) -> Discharge:
    base = dict(name="test", gas="he", gap_m=0.025, p_Pa=30.0, V_rf_V=0.0, n_cells=64, steps_per_period=400,
                n_e0=1, n_i0=1, n_init_m3=1e14)
    base.update(kw)
    return Discharge(**base)


def maxwell_state(rng, n: int, n_cells: int, sigma_v: float, dtype=np.float64, cells=None, f=None,
                  drift=(0.0, 0.0, 0.0)) -> dict:
    """n particles, uniform in [0, n_cells) (or at the given cells), Maxwellian velocities."""
    if cells is None:
        x = rng.uniform(0.0, n_cells, n)
        c = np.minimum(np.floor(x).astype(np.int32), n_cells - 1)
        ff = (x - c).astype(dtype)
    else:
        c = np.broadcast_to(np.asarray(cells, np.int32), (n,)).copy()
        ff = rng.uniform(0.0, 1.0, n).astype(dtype) if f is None else np.broadcast_to(f, (n,)).astype(dtype)
    ff = np.minimum(ff, np.nextafter(dtype(1), dtype(0))).astype(dtype)
    v = rng.normal(0.0, sigma_v, (3, n)) + np.asarray(drift)[:, None]
    return {"c": c, "f": ff, "vx": v[0].astype(dtype), "vy": v[1].astype(dtype), "vz": v[2].astype(dtype)}


def speed_state(rng, n: int, n_cells: int, speed: float, dtype=np.float64, cell=None) -> dict:
    """n particles with one speed and isotropic random directions."""
    mu = rng.uniform(-1, 1, n)
    ph = rng.uniform(0, 2 * np.pi, n)
    st = np.sqrt(1 - mu ** 2)
    cc = np.full(n, n_cells // 2 if cell is None else cell, np.int32)
    return {"c": cc, "f": rng.uniform(0, 1, n).astype(dtype),
            "vx": (speed * st * np.cos(ph)).astype(dtype), "vy": (speed * st * np.sin(ph)).astype(dtype),
            "vz": (speed * mu).astype(dtype)}


def energy_state(rng, n: int, n_cells: int, eps_lo: float, eps_hi: float, mass: float, dtype=np.float64) -> dict:
    """n particles with energies uniform in [eps_lo, eps_hi] eV, isotropic directions, random cells."""
    eps = rng.uniform(eps_lo, eps_hi, n)
    sp = np.sqrt(2 * E_CH * eps / mass)
    st = speed_state(rng, n, n_cells, 1.0, np.float64)
    x = rng.uniform(0.0, n_cells, n)
    c = np.minimum(np.floor(x).astype(np.int32), n_cells - 1)
    return {"c": c, "f": np.minimum(x - c, 1 - 1e-7).astype(dtype), "vx": (sp * st["vx"]).astype(dtype),
            "vy": (sp * st["vy"]).astype(dtype), "vz": (sp * st["vz"]).astype(dtype)}


def mixed_state(rng, n: int, n_cells: int, species: int, dtype=np.float32, gap_m=0.025, dt_s=1e-10) -> dict:
    """A parity-test population: thermal bulk, fast particles crossing several cells, particles at
    and next to both electrodes, particles exactly on nodes, and (electrons) energies across all
    collision thresholds."""
    dx = gap_m / n_cells
    if species == 0:
        sig, mass = np.sqrt(E_CH * 3.0 / M_E), M_E
    else:
        sig, mass = np.sqrt(K_B * 600.0 / (4.0026 * AMU)), 4.0026 * AMU
    st = maxwell_state(rng, n, n_cells, sig, np.float64)
    k = n // 8
    idx = rng.permutation(n)
    # fast particles: several cells per step either way
    fast = idx[:k]
    vmax = 6.0 * dx / dt_s
    st["vz"][fast] = rng.uniform(-vmax, vmax, fast.size)
    if species == 0:
        hot = idx[k:2 * k]
        e = rng.uniform(5.0, 80.0, hot.size)
        sp = np.sqrt(2 * E_CH * e / mass)
        mu = rng.uniform(-1, 1, hot.size)
        st["vz"][hot] = sp * mu
        st["vx"][hot] = sp * np.sqrt(1 - mu ** 2)
        st["vy"][hot] = 0.0
    wall = idx[2 * k:3 * k]
    half = wall.size // 2
    st["c"][wall[:half]] = 0
    st["c"][wall[half:]] = n_cells - 1
    st["f"][wall[:half]] = rng.uniform(0, 0.05, half)
    st["f"][wall[half:]] = rng.uniform(0.95, 1.0, wall.size - half)
    st["vz"][wall[:half]] = -np.abs(st["vz"][wall[:half]]) * 3
    st["vz"][wall[half:]] = np.abs(st["vz"][wall[half:]]) * 3
    node = idx[3 * k:3 * k + k // 4]
    st["f"][node] = 0.0
    for key in ("f", "vx", "vy", "vz"):
        st[key] = st[key].astype(dtype)
    st["f"] = np.minimum(st["f"], np.nextafter(dtype(1), dtype(0))).astype(dtype)
    # cell-sorted, as the library keeps its store
    order = np.argsort(st["c"], kind="stable")
    return {key: np.ascontiguousarray(v[order]) for key, v in st.items()}


def random_field(rng, n_cells: int, scale: float, dtype=np.float32) -> np.ndarray:
    """A smooth random node field (V/m) with sheath-like edges."""
    z = np.linspace(0, 1, n_cells + 1)
    E = scale * (np.sin(2 * np.pi * (z * rng.uniform(0.5, 2) + rng.uniform())) + 4 * (z - 0.5) ** 3)
    E += rng.normal(0, 0.05 * scale, n_cells + 1)
    return E.astype(dtype)
