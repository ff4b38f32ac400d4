"""ctypes wrapper of the plain CPU PIC/MCC oracle (pic_oracle.c).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline / reference arm use this module. The CUDA library never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBS = {"f64": os.path.join(HERE, "liboracle_f64.so"), "f32": os.path.join(HERE, "liboracle_f32.so")}
SRC = os.path.join(HERE, "pic_oracle.c")


def build(force: bool = False) -> None:
    """Compile both precisions of the oracle with gcc (no FP contraction)."""
    for tag, out in LIBS.items():
        if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
                os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "pic_oracle.h"))):
            continue
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-Wall", "-Wno-unused-function", SRC, "-o", out + ".tmp", "-lm"]
        if tag == "f32":
            cmd.insert(1, "-DORC_F32")
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)


class OrcGas(C.Structure):
    _fields_ = [("mass_kg", C.c_double), ("n_exc", C.c_int32), ("n_pts", C.c_int32), ("de_eV", C.c_double),
                ("eps_exc_eV", C.c_double * 2), ("eps_iz_eV", C.c_double),
                ("sigma_e", C.POINTER(C.c_double)), ("sigma_i", C.POINTER(C.c_double))]


class OrcParams(C.Structure):
    _fields_ = [("gap_m", C.c_double), ("p_Pa", C.c_double), ("T_gas_K", C.c_double), ("f_rf_Hz", C.c_double),
                ("V_rf_V", C.c_double), ("dt_s", C.c_double), ("w_e", C.c_double), ("w_i", C.c_double),
                ("T_e0_eV", C.c_double), ("T_i0_K", C.c_double), ("gamma_see", C.c_double),
                ("n_e0", C.c_int64), ("n_i0", C.c_int64), ("seed", C.c_uint64), ("n_cells", C.c_int32),
                ("sort_every", C.c_int32), ("discharge_id", C.c_uint32), ("pad_", C.c_int32)]


class OrcCounters(C.Structure):
    _fields_ = [("absorbed", (C.c_int64 * 2) * 2), ("collisions_e", C.c_int64 * 4),
                ("collisions_i", C.c_int64 * 2), ("null_inelastic", C.c_int64), ("see_emitted", C.c_int64),
                ("candidates", C.c_int64 * 2), ("table_clamped", C.c_int64 * 2)]

    def as_dict(self) -> dict:
        return {"absorbed": [[self.absorbed[a][b] for b in range(2)] for a in range(2)],
                "collisions_e": list(self.collisions_e), "collisions_i": list(self.collisions_i),
                "null_inelastic": self.null_inelastic, "see_emitted": self.see_emitted,
                "candidates": list(self.candidates), "table_clamped": list(self.table_clamped)}


class OrcDerived(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("dx", "n_gas", "kmax_e", "kmax_i", "numax_e", "numax_i",
                                          "pnull_e", "pnull_i")] + \
               [("thr_e", C.c_uint32), ("thr_i", C.c_uint32)] + \
               [(n, C.c_double) for n in ("K_e", "K_i", "dtdx", "kappa_e", "kappa_i", "kappa_E", "beta_e",
                                          "omb_e")] + \
               [("de2_exc", C.c_double * 2)] + \
               [(n, C.c_double) for n in ("de2_iz", "sig_n", "sig_e0", "sig_i0", "sig_see", "sig_see_n")]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if name == "de2_exc" else v
        return out


class OrcDiagConfig(C.Structure):
    _fields_ = [("period_steps", C.c_int32), ("phase_step", C.c_int32), ("sample_every", C.c_int32),
                ("eedf_bins", C.c_int32), ("eedf_de_eV", C.c_double), ("fast_eV", C.c_double)]


class OrcMomentInfo(C.Structure):
    _fields_ = [("steps", C.c_int64), ("absorbed", (C.c_double * 2) * 2)]


_libs = {}


def _lib(prec: str):
    if prec not in _libs:
        if not os.path.exists(LIBS[prec]):
            build()
        L = C.CDLL(LIBS[prec])
        vp = C.c_void_p
        L.orc_create.restype = vp
        L.orc_create.argtypes = [C.POINTER(OrcGas), C.POINTER(OrcParams)]
        L.orc_destroy.argtypes = [vp]
        for name in ("orc_load", "orc_sweep", "orc_sort", "orc_solve"):
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = C.c_int
        L.orc_step.argtypes = [vp, C.c_int64]
        L.orc_count.argtypes = [vp, C.c_int]
        L.orc_count.restype = C.c_int64
        L.orc_get_state.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp]
        L.orc_set_state.argtypes = [vp, C.c_int, C.c_int64, vp, vp, vp, vp, vp]
        for name in ("orc_get_field", "orc_set_field", "orc_get_phi", "orc_get_efield64",
                     "orc_get_energy_deposit"):
            getattr(L, name).argtypes = [vp, vp]
        L.orc_get_deposit.argtypes = [vp, C.c_int, vp]
        L.orc_set_deposit.argtypes = [vp, C.c_int, vp]
        L.orc_get_step.argtypes = [vp]
        L.orc_get_step.restype = C.c_int64
        L.orc_set_step.argtypes = [vp, C.c_int64]
        L.orc_get_counters.argtypes = [vp, C.POINTER(OrcCounters)]
        L.orc_get_derived.argtypes = [vp, C.POINTER(OrcDerived)]
        L.orc_get_tables.argtypes = [vp, vp, vp]
        L.orc_moments.argtypes = [vp, vp, vp, vp, C.POINTER(OrcMomentInfo)]
        L.orc_reset_moments.argtypes = [vp]
        L.orc_last_current.argtypes = [vp, vp]
        L.orc_set_current_drive.argtypes = [vp, C.c_int, C.c_double]
        L.orc_set_current_drive.restype = C.c_int
        L.orc_set_scheme.argtypes = [vp, C.c_int]
        L.orc_set_scheme.restype = C.c_int
        L.orc_period_history.argtypes = [vp, vp, vp, C.c_int64, vp]
        L.orc_period_history.restype = C.c_int64
        L.orc_set_diagnostics.argtypes = [vp, C.POINTER(OrcDiagConfig)]
        L.orc_set_diagnostics.restype = C.c_int
        L.orc_reset_diagnostics.argtypes = [vp]
        L.orc_diagnostics.argtypes = [vp] + [vp] * 10 + [C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.orc_diagnostics.restype = C.c_int
        L.orc_load_profiles.argtypes = [vp, C.c_int, vp, vp, vp]
        L.orc_load_profiles.restype = C.c_int
        L.orc_real_bytes.restype = C.c_int
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_uniform.argtypes = [C.c_uint32]
        L.orc_uniform.restype = C.c_float
        L.orc_logf.argtypes = [C.c_float]
        L.orc_logf.restype = C.c_float
        L.orc_sincospif.argtypes = [C.c_float, C.POINTER(C.c_float), C.POINTER(C.c_float)]
        L.orc_box_muller.argtypes = [C.c_float, C.c_float, C.POINTER(C.c_float), C.POINTER(C.c_float)]
        L.orc_isotropic.argtypes = [C.c_float, C.c_float, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                    C.POINTER(C.c_float)]
        L.orc_poisson.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, vp, vp, vp]
        _libs[prec] = L
    return _libs[prec]


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ---- building blocks -------------------------------------------------------

def philox(ctr, key) -> np.ndarray:
    L = _lib("f64")
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    L.orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def uniform(x: int) -> float:
    return float(_lib("f64").orc_uniform(int(x) & 0xFFFFFFFF))


def logf(x: float) -> float:
    return float(_lib("f64").orc_logf(float(x)))


def sincospif(y: float):
    s, c = C.c_float(), C.c_float()
    _lib("f64").orc_sincospif(float(y), C.byref(s), C.byref(c))
    return s.value, c.value


def box_muller(ua: float, ub: float):
    a, b = C.c_float(), C.c_float()
    _lib("f64").orc_box_muller(float(ua), float(ub), C.byref(a), C.byref(b))
    return a.value, b.value


def isotropic(ua: float, ub: float):
    x, y, z = C.c_float(), C.c_float(), C.c_float()
    _lib("f64").orc_isotropic(float(ua), float(ub), C.byref(x), C.byref(y), C.byref(z))
    return x.value, y.value, z.value


def poisson(rho: np.ndarray, dx: float, V0: float, VN: float = 0.0):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    N = rho.size - 1
    phi = np.zeros(N + 1)
    E = np.zeros(N + 1)
    _lib("f64").orc_poisson(N, dx, V0, VN, _p(rho), _p(phi), _p(E))
    return phi, E


# ---- a whole discharge -----------------------------------------------------

def make_gas(g) -> tuple:
    """OrcGas from an xsections.GasTables; returns (struct, keep-alive arrays)."""
    se = np.ascontiguousarray(g.sigma_e, dtype=np.float64)
    si = np.ascontiguousarray(g.sigma_i, dtype=np.float64)
    exc = list(g.eps_exc_eV) + [0.0] * (2 - len(g.eps_exc_eV))
    s = OrcGas(g.mass_kg, len(g.eps_exc_eV), se.shape[0], g.de_eV, (C.c_double * 2)(*exc), g.eps_iz_eV,
               se.ctypes.data_as(C.POINTER(C.c_double)), si.ctypes.data_as(C.POINTER(C.c_double)))
    return s, (se, si)


def make_params(d, sort_every: int = 0) -> OrcParams:
    return OrcParams(d.gap_m, d.p_Pa, d.T_gas_K, d.f_rf_Hz, d.V_rf_V, d.dt_s, d.w_e, d.w_i, d.T_e0_eV,
                     d.T_i0_K, d.gamma_see, d.n_e0, d.n_i0, d.seed, d.n_cells, sort_every, d.discharge_id, 0)


class Oracle:
    """One discharge in the oracle. precision: 'f64' (physics) or 'f32' (decision precision of the
    FP32 kernel)."""

    def __init__(self, gas, discharge, precision: str = "f64", sort_every: int = 0, load: bool = True):
        self.L = _lib(precision)
        self.prec = precision
        self.dtype = np.float32 if precision == "f32" else np.float64
        self.N = discharge.n_cells
        self.discharge = discharge
        g, keep = make_gas(gas)
        p = make_params(discharge, sort_every)
        self.h = self.L.orc_create(C.byref(g), C.byref(p))
        del keep
        if not self.h:
            raise ValueError("orc_create rejected the parameters")
        if load:
            self.load()

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.orc_destroy(h)
            self.h = None

    def load(self):
        if self.L.orc_load(self.h):
            raise RuntimeError("orc_load failed")

    def load_profiles(self, n_e, n_i, mean_eps):
        a = [np.ascontiguousarray(x, np.float64) for x in (n_e, n_i, mean_eps)]
        if self.L.orc_load_profiles(self.h, a[0].size, *[_p(x) for x in a]):
            raise RuntimeError("orc_load_profiles failed")

    def sweep(self):
        if self.L.orc_sweep(self.h):
            raise RuntimeError("orc_sweep failed")

    def sort(self):
        self.L.orc_sort(self.h)

    def solve(self):
        self.L.orc_solve(self.h)

    def step(self, n: int = 1):
        if self.L.orc_step(self.h, int(n)):
            raise RuntimeError("orc_step failed")

    @property
    def step_index(self) -> int:
        return int(self.L.orc_get_step(self.h))

    @step_index.setter
    def step_index(self, n: int):
        self.L.orc_set_step(self.h, int(n))

    def count(self, species: int) -> int:
        return int(self.L.orc_count(self.h, species))

    def get_state(self, species: int) -> dict:
        n = self.count(species)
        c = np.zeros(n, np.int32)
        arrs = [np.zeros(n, self.dtype) for _ in range(4)]
        self.L.orc_get_state(self.h, species, _p(c), *[_p(a) for a in arrs])
        return {"c": c, "f": arrs[0], "vx": arrs[1], "vy": arrs[2], "vz": arrs[3]}

    def set_state(self, species: int, st: dict):
        c = np.ascontiguousarray(st["c"], np.int32)
        arrs = [np.ascontiguousarray(st[k], self.dtype) for k in ("f", "vx", "vy", "vz")]
        rc = self.L.orc_set_state(self.h, species, c.size, _p(c), *[_p(a) for a in arrs])
        if rc:
            raise ValueError(f"orc_set_state failed ({rc})")

    def get_field(self) -> np.ndarray:
        E = np.zeros(self.N + 1, self.dtype)
        self.L.orc_get_field(self.h, _p(E))
        return E

    def set_field(self, E):
        E = np.ascontiguousarray(E, self.dtype)
        assert E.size == self.N + 1
        self.L.orc_set_field(self.h, _p(E))

    def get_field64(self) -> np.ndarray:
        E = np.zeros(self.N + 1)
        self.L.orc_get_efield64(self.h, _p(E))
        return E

    def get_phi(self) -> np.ndarray:
        phi = np.zeros(self.N + 1)
        self.L.orc_get_phi(self.h, _p(phi))
        return phi

    def get_deposit(self, species: int) -> np.ndarray:
        D = np.zeros(self.N + 1, np.int64)
        self.L.orc_get_deposit(self.h, species, _p(D))
        return D

    def set_deposit(self, species: int, D):
        D = np.ascontiguousarray(D, np.int64)
        self.L.orc_set_deposit(self.h, species, _p(D))

    def get_energy_deposit(self) -> np.ndarray:
        Q = np.zeros(self.N + 1, np.int64)
        self.L.orc_get_energy_deposit(self.h, _p(Q))
        return Q

    def counters(self) -> dict:
        c = OrcCounters()
        self.L.orc_get_counters(self.h, C.byref(c))
        return c.as_dict()

    def derived(self) -> dict:
        d = OrcDerived()
        self.L.orc_get_derived(self.h, C.byref(d))
        return d.as_dict()

    def tables(self, n_pts: int):
        Te = np.zeros((n_pts, 4), self.dtype)
        Ti = np.zeros((n_pts, 2), self.dtype)
        self.L.orc_get_tables(self.h, _p(Te), _p(Ti))
        return Te, Ti

    def moments(self) -> dict:
        ne = np.zeros(self.N + 1)
        ni = np.zeros(self.N + 1)
        me = np.zeros(self.N + 1)
        info = OrcMomentInfo()
        self.L.orc_moments(self.h, _p(ne), _p(ni), _p(me), C.byref(info))
        return {"n_e": ne, "n_i": ni, "mean_eps": me, "steps": info.steps,
                "absorbed": [[info.absorbed[a][b] for b in range(2)] for a in range(2)]}

    def reset_moments(self):
        self.L.orc_reset_moments(self.h)

    def set_diagnostics(self, period_steps: int, phase_step: int, sample_every: int, eedf_bins: int,
                        eedf_de_eV: float, fast_eV: float):
        cfg = OrcDiagConfig(period_steps, phase_step, sample_every, eedf_bins, eedf_de_eV, fast_eV)
        if self.L.orc_set_diagnostics(self.h, C.byref(cfg)):
            raise ValueError("orc_set_diagnostics rejected the configuration")
        self._eedf_bins = eedf_bins

    def reset_diagnostics(self):
        self.L.orc_reset_diagnostics(self.h)

    def diagnostics(self) -> dict:
        N1 = self.N + 1
        keys = ("E", "n_e", "mean_eps", "gamma_e", "q_e", "heating", "ion_rate", "n_fast", "n_fast_avg")
        out = {k: np.zeros(N1) for k in keys}
        out["eedf"] = np.zeros(self._eedf_bins)
        sn, sm = C.c_int64(), C.c_int64()
        if self.L.orc_diagnostics(self.h, *[_p(out[k]) for k in keys], _p(out["eedf"]), C.byref(sn), C.byref(sm)):
            raise RuntimeError("diagnostics not configured")
        out["snapshots"], out["samples"] = sn.value, sm.value
        return out

    def set_current_drive(self, period_steps: int, J_target: float = 0.0):
        """First-harmonic amplitude of J(0,t) per rf period; J_target > 0: adapt V0 after every period."""
        if self.L.orc_set_current_drive(self.h, int(period_steps), float(J_target)):
            raise ValueError("orc_set_current_drive rejected the arguments")

    def set_scheme(self, leapfrog: bool):
        """Velocity Verlet (collisions at v_n, default) or the leapfrog variant (at v_{n+1/2})."""
        if self.L.orc_set_scheme(self.h, 1 if leapfrog else 0):
            raise ValueError("orc_set_scheme rejected the argument")

    def period_history(self):
        """(J_calc per completed period, V0 applied in it, V0 now)."""
        Vn = C.c_double()
        n = self.L.orc_period_history(self.h, None, None, 0, None)
        amp, V0 = np.zeros(n), np.zeros(n)
        self.L.orc_period_history(self.h, _p(amp), _p(V0), n, C.byref(Vn))
        return amp, V0, Vn.value

    def last_current(self) -> np.ndarray:
        """J(t) of the last solved step at z = 0 and at z = d, A/m^2."""
        J = np.zeros(2)
        self.L.orc_last_current(self.h, _p(J))
        return J


if __name__ == "__main__":
    build(force="--force" in sys.argv)
