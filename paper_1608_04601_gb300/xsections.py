"""Synthetic cross-section tables for He-like and Ar-like background gases.

The paper's reaction set (Table "reactions": electron elastic, excitation and
ionization; ion isotropic and backward elastic) uses Biagi and Phelps data that
are not available here. These analytic stand-ins keep the same processes,
thresholds, energy frames and orders of magnitude; they are not fits to the
real data, and nothing computed with them is comparable to the paper's printed
plasma parameters.

This module only produces input arrays (cross sections in m^2 on a uniform
energy grid); it holds none of the PIC/MCC arithmetic, and both the CUDA
library and the CPU oracle consume its output.

Forms, with x = eps / eps_threshold:
  He-like electron elastic   6e-20 / sqrt(1 + eps / 25 eV)
  Ar-like electron elastic   1e-19 (1 - 0.9 exp(-ln(eps / 0.25 eV)^2 / 0.5)), a Ramsauer-like dip
  excitation / ionization    sigma_pk e ln(x) / x for x > 1 (maximum sigma_pk at x = e), else 0
  ion isotropic / backward   sigma0 sqrt(1 eV / max(eps_cm, 0.1 eV)); the 0.1 eV floor follows the
                             paper's lower limit for the argon ion data (section "Physical data").
Electron tables are in lab energy; ion tables in centre-of-mass energy, the frame the paper
uses for the helium ion data.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

AMU = 1.66053906660e-27


@dataclass
class GasTables:
    name: str
    mass_kg: float
    eps_exc_eV: tuple
    eps_iz_eV: float
    de_eV: float
    sigma_e: np.ndarray  # (n_pts, 2 + n_exc): elastic, excitation levels..., ionization
    sigma_i: np.ndarray  # (n_pts, 2): isotropic, backward
    gas_id: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_exc(self) -> int:
        return len(self.eps_exc_eV)

    @property
    def n_pts(self) -> int:
        return int(self.sigma_e.shape[0])


def _grid(n_pts: int, de_eV: float) -> np.ndarray:
    return np.arange(n_pts, dtype=np.float64) * de_eV


def _threshold_form(eps: np.ndarray, eps_th: float, sigma_pk: float) -> np.ndarray:
    x = eps / eps_th
    out = np.zeros_like(eps)
    m = x > 1.0
    out[m] = sigma_pk * np.e * np.log(x[m]) / x[m]
    return out


def _ion_form(eps: np.ndarray, sigma0: float) -> np.ndarray:
    return sigma0 * np.sqrt(1.0 / np.maximum(eps, 0.1))


def he_like(eps_max_eV: float = 1000.0, de_eV: float = 1e-3) -> GasTables:
    """He-like gas: elastic, triplet (19.8 eV) and singlet (20.61 eV) excitation, ionization (24.6 eV)."""
    n_pts = int(round(eps_max_eV / de_eV)) + 1
    eps = _grid(n_pts, de_eV)
    sig_e = np.stack([
        6e-20 / np.sqrt(1.0 + eps / 25.0),
        _threshold_form(eps, 19.8, 1.0e-21),
        _threshold_form(eps, 20.61, 5.0e-22),
        _threshold_form(eps, 24.6, 3.5e-21),
    ], axis=1)
    sig_i = np.stack([_ion_form(eps, 2.5e-19), _ion_form(eps, 2.5e-19)], axis=1)
    return GasTables("He-like", 4.002602 * AMU, (19.8, 20.61), 24.6, de_eV,
                     np.ascontiguousarray(sig_e), np.ascontiguousarray(sig_i), gas_id=0)


def ar_like(eps_max_eV: float = 1000.0, de_eV: float = 1e-3) -> GasTables:
    """Ar-like gas: elastic with a Ramsauer-like dip, excitation (11.5 eV), ionization (15.8 eV)."""
    n_pts = int(round(eps_max_eV / de_eV)) + 1
    eps = _grid(n_pts, de_eV)
    with np.errstate(divide="ignore"):
        lg = np.log(np.where(eps > 0, eps, 1e-300) / 0.25)
    el = 1e-19 * (1.0 - 0.9 * np.exp(-(lg ** 2) / 0.5))
    el[eps == 0] = 1e-19
    sig_e = np.stack([
        el,
        _threshold_form(eps, 11.5, 1.5e-20),
        _threshold_form(eps, 15.8, 3.0e-20),
    ], axis=1)
    sig_i = np.stack([_ion_form(eps, 4e-19), _ion_form(eps, 6e-19)], axis=1)
    return GasTables("Ar-like", 39.948 * AMU, (11.5,), 15.8, de_eV,
                     np.ascontiguousarray(sig_e), np.ascontiguousarray(sig_i), gas_id=1)


def by_name(name: str, **kw) -> GasTables:
    name = name.lower()
    if name.startswith("he"):
        return he_like(**kw)
    if name.startswith("ar"):
        return ar_like(**kw)
    raise ValueError(f"unknown gas {name!r}")


# ---- tables used only by the pins on the collision statistics -------------

def constant_sigma(sigma_el: float = 1e-19, mass_kg: float = 4.002602 * AMU, eps_max_eV: float = 100.0,
                   de_eV: float = 1e-2, n_exc: int = 1, thresholds=(1e9,), eps_iz_eV: float = 2e9,
                   sigma_ion=(0.0, 0.0)) -> GasTables:
    """Constant elastic cross section, inelastic channels closed (thresholds far away)."""
    n_pts = int(round(eps_max_eV / de_eV)) + 1
    sig_e = np.zeros((n_pts, 2 + n_exc))
    sig_e[:, 0] = sigma_el
    sig_i = np.zeros((n_pts, 2))
    sig_i[:, 0], sig_i[:, 1] = sigma_ion
    th = tuple(thresholds[:n_exc]) if len(thresholds) >= n_exc else tuple(thresholds) * n_exc
    return GasTables("const-sigma", mass_kg, th, eps_iz_eV, de_eV, sig_e, sig_i)


def constant_nu(k_el: float, mass_kg: float, eps_max_eV: float = 100.0, de_eV: float = 1e-2,
                k_iz: float = 0.0, k_ion=(0.0, 0.0)) -> GasTables:
    """Cross sections proportional to 1/v so that sigma*v is constant (Maxwell molecules).

    k_el, k_iz: electron rate coefficients sigma*v in m^3/s; the ionization channel has a
    zero threshold when k_iz > 0. k_ion: ion isotropic/backward rate coefficients sigma*g.
    """
    n_pts = int(round(eps_max_eV / de_eV)) + 1
    eps = _grid(n_pts, de_eV)
    e = 1.602176634e-19
    me = 9.1093837015e-31
    v = np.sqrt(2.0 * e * np.maximum(eps, de_eV * 1e-3) / me)
    g = np.sqrt(4.0 * e * np.maximum(eps, de_eV * 1e-3) / mass_kg)
    sig_e = np.zeros((n_pts, 3))
    sig_e[:, 0] = k_el / v
    sig_e[:, 2] = k_iz / v
    sig_i = np.stack([k_ion[0] / g, k_ion[1] / g], axis=1)
    return GasTables("const-nu", mass_kg, (1e9,), 0.0 if k_iz > 0 else 2e9, de_eV, sig_e, sig_i)
