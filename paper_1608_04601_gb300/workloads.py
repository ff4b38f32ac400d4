"""Named discharge workloads (synthetic inputs; no method arithmetic here).

C1..C4 below are the discharges this library is measured and checked on. Their
gases are the synthetic He-like / Ar-like tables of ``xsections``; weights follow
from the paper's initial plasma densities for the PIC runs (Table
"numericalparameters": 4e14 m^-3 for helium, 4e15 m^-3 for argon) as
w = n_init * gap / N_superparticles.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

F_RF = 13.56e6


@dataclass
class Discharge:
    name: str
    gas: str                 # "he" or "ar"
    gap_m: float
    p_Pa: float
    V_rf_V: float
    n_cells: int
    steps_per_period: int
    n_e0: int
    n_i0: int
    n_init_m3: float
    T_gas_K: float = 300.0
    f_rf_Hz: float = F_RF
    T_e0_eV: float = 2.0
    T_i0_K: float = 300.0
    gamma_see: float = 0.0
    periods: int = 1
    eps_max_eV: float = 1000.0
    de_eV: float = 1e-3
    seed: int = 1
    discharge_id: int = 0

    @property
    def dt_s(self) -> float:
        return 1.0 / (self.f_rf_Hz * self.steps_per_period)

    @property
    def w_e(self) -> float:
        return self.n_init_m3 * self.gap_m / self.n_e0

    @property
    def w_i(self) -> float:
        return self.n_init_m3 * self.gap_m / self.n_i0

    def capacity(self, factor: float = 2.0) -> tuple:
        return (int(self.n_e0 * factor) + 4096, int(self.n_i0 * factor) + 4096)

    def scaled(self, **kw) -> "Discharge":
        return replace(self, **kw)


def c1() -> Discharge:
    """He-like, 30 Pa, 2.5 cm, 200 V, 128 cells, 400 steps/period, 2e4 + 2e4, 10 periods."""
    return Discharge("C1 he-like 30Pa 2.5cm 200V N128 2e4+2e4", "he", 0.025, 30.0, 200.0, 128, 400,
                     20_000, 20_000, 4e14, periods=10)


def c2() -> Discharge:
    """Ar-like, 10 Pa, 2.5 cm, 300 V, 512 cells, 2000 steps/period, 1e6 + 1e6."""
    return Discharge("C2 ar-like 10Pa 2.5cm 300V N512 1e6+1e6", "ar", 0.025, 10.0, 300.0, 512, 2000,
                     1_000_000, 1_000_000, 4e15, periods=1000)


def c3() -> Discharge:
    """He-like, 80 Pa, 5 cm, 500 V, 2048 cells, 4000 steps/period, 2e7 + 2e7, gamma 0.1."""
    return Discharge("C3 he-like 80Pa 5cm 500V N2048 2e7+2e7 gamma0.1", "he", 0.05, 80.0, 500.0, 2048, 4000,
                     20_000_000, 20_000_000, 4e14, gamma_see=0.1, eps_max_eV=2000.0)


def c4(seed: int = 1) -> list:
    """32 discharges: {He-like, Ar-like} x p in {10,20,40,80} Pa x V_rf in {150,250,350,500} V,
    2.5 cm, 512 cells, 2000 steps/period, 1e5..4e6 particles each (log-uniform, seeded)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    k = 0
    for gas in ("he", "ar"):
        for p in (10.0, 20.0, 40.0, 80.0):
            for V in (150.0, 250.0, 350.0, 500.0):
                n = int(round(float(np.exp(rng.uniform(np.log(1e5), np.log(4e6))))))
                out.append(Discharge(f"C4[{k}] {gas} {p:g}Pa {V:g}V n{n}", gas, 0.025, p, V, 512, 2000, n, n,
                                     4e14 if gas == "he" else 4e15, eps_max_eV=1000.0, discharge_id=k,
                                     seed=seed))
                k += 1
    return out


WORKLOADS = {"c1": c1, "c2": c2, "c3": c3}
