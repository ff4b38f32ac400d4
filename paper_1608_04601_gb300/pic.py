"""Python face of the PIC/MCC library: argument marshalling around include/pic.h.

Every step of the computation runs in libpic.so's CUDA kernels; this module
only converts numpy arrays and dataclasses to the C structures and back.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native as NV
from .workloads import Discharge
from .xsections import GasTables

FP32, FP64 = 0, 1


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def gas_struct(g: GasTables):
    se = np.ascontiguousarray(g.sigma_e, np.float64)
    si = np.ascontiguousarray(g.sigma_i, np.float64)
    exc = list(g.eps_exc_eV) + [0.0] * (2 - len(g.eps_exc_eV))
    s = NV.PicGas(g.mass_kg, len(g.eps_exc_eV), se.shape[0], g.de_eV, (C.c_double * 2)(*exc), g.eps_iz_eV,
                  se.ctypes.data_as(C.POINTER(C.c_double)), si.ctypes.data_as(C.POINTER(C.c_double)))
    return s, (se, si)


def discharge_struct(d: Discharge, gas_index: int = 0, capacity=None) -> NV.PicDischarge:
    cap_e, cap_i = capacity if capacity is not None else d.capacity()
    w = NV.PicWeights(d.w_e, d.w_i, d.n_e0, d.n_i0, cap_e, cap_i, d.T_e0_eV, d.T_i0_K, d.gamma_see,
                      d.steps_per_period, 0)
    return NV.PicDischarge(gas_index, d.n_cells, d.gap_m, d.p_Pa, d.T_gas_K, d.f_rf_Hz, d.V_rf_V, d.dt_s, w,
                           d.discharge_id, 0)


class Simulation:
    """A batch of discharges advanced together on one GPU.

    gases: list of GasTables; discharges: list of (Discharge, gas_index) or Discharge (gas 0).
    precision: "fp32" (FP32 particles, fixed-point deposits, FP64 field) or "fp64".
    """

    def __init__(self, gases, discharges, seed=None, precision: str = "fp32", sort_every: int = 0,
                 block: int = 256, ppt: int = 4, ctas_per_sm: int = 0, use_graph: bool = False,
                 stream=None, load: bool = True, capacity=None, leapfrog: bool = False):
        self.L = NV.lib()
        if isinstance(gases, GasTables):
            gases = [gases]
        if isinstance(discharges, Discharge):
            discharges = [discharges]
        self.gases = gases
        self.discharges = [d if isinstance(d, tuple) else (d, 0) for d in discharges]
        self.fp64 = precision == "fp64"
        self.dtype = np.float64 if self.fp64 else np.float32
        gs, keep = [], []
        for g in gases:
            s, k = gas_struct(g)
            gs.append(s)
            keep.append(k)
        garr = (NV.PicGas * len(gs))(*gs)
        caps = capacity if capacity is not None else [None] * len(self.discharges)
        darr = (NV.PicDischarge * len(self.discharges))(
            *[discharge_struct(d, gi, caps[i]) for i, (d, gi) in enumerate(self.discharges)])
        opt = NV.PicOptions()
        self.L.pic_default_options(C.byref(opt))
        opt.precision = FP64 if self.fp64 else FP32
        opt.sort_every = sort_every
        opt.block = block
        opt.ppt = ppt
        opt.ctas_per_sm = ctas_per_sm
        opt.use_graph = 1 if use_graph else 0
        opt.load = 1 if load else 0
        opt.leapfrog = 1 if leapfrog else 0
        if stream == "torch":
            import torch
            opt.cuda_stream = torch.cuda.current_stream().cuda_stream
        elif stream is not None:
            opt.cuda_stream = int(stream)
        if seed is None:
            seed = self.discharges[0][0].seed
        h = C.c_void_p()
        st = self.L.pic_batch_create(C.byref(h), garr, len(gs), darr, len(self.discharges), seed, C.byref(opt))
        del keep
        if st != NV.PIC_OK:
            raise NV.PicError(st, "pic_batch_create")
        self.h = h
        self.N = [d.n_cells for d, _ in self.discharges]

    # ---- lifecycle
    def close(self):
        if getattr(self, "h", None):
            self.L.pic_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _ck(self, st):
        NV.check(st, self.h)

    # ---- stepping
    def step(self, n: int = 1):
        self._ck(self.L.pic_step(self.h, int(n)))

    def sweep(self):
        self._ck(self.L.pic_sweep(self.h))

    def sort(self):
        self._ck(self.L.pic_sort(self.h))

    def solve(self):
        self._ck(self.L.pic_solve(self.h))

    def sync(self):
        self._ck(self.L.pic_sync(self.h))

    @property
    def step_index(self) -> int:
        v = C.c_int64()
        self._ck(self.L.pic_get_step(self.h, C.byref(v)))
        return v.value

    @step_index.setter
    def step_index(self, n: int):
        self._ck(self.L.pic_set_step(self.h, int(n)))

    # ---- state
    def count(self, d: int, species: int) -> int:
        v = C.c_int64()
        self._ck(self.L.pic_get_count(self.h, d, species, C.byref(v)))
        return v.value

    def get_state(self, d: int, species: int, out: dict = None) -> dict:
        """The store of (d, species) as host arrays; `out` may hold preallocated arrays (keys c, f,
        vx, vy, vz, e.g. in pinned memory) of at least the store's size, which are then filled."""
        if out is not None:  # the library reads the count itself
            c = out["c"]
            arrs = [out[k] for k in ("f", "vx", "vy", "vz")]
            assert c.dtype == np.int32 and all(a.dtype == self.dtype for a in arrs)
            cap = min(c.size, *[a.size for a in arrs])
        else:
            n = self.count(d, species)
            c = np.zeros(max(n, 1), np.int32)
            arrs = [np.zeros(max(n, 1), self.dtype) for _ in range(4)]
            cap = max(n, 1)
        got = C.c_int64()
        self._ck(self.L.pic_get_state(self.h, d, species, cap, _ptr(c), *[_ptr(a) for a in arrs], C.byref(got)))
        n = got.value
        return {"c": c[:n], "f": arrs[0][:n], "vx": arrs[1][:n], "vy": arrs[2][:n], "vz": arrs[3][:n]}

    def set_state(self, d: int, species: int, st: dict):
        c = np.ascontiguousarray(st["c"], np.int32)
        arrs = [np.ascontiguousarray(st[k], self.dtype) for k in ("f", "vx", "vy", "vz")]
        self._ck(self.L.pic_set_state(self.h, d, species, c.size, _ptr(c), *[_ptr(a) for a in arrs]))

    def get_field(self, d: int = 0):
        N1 = self.N[d] + 1
        E = np.zeros(N1, self.dtype)
        E64 = np.zeros(N1)
        phi = np.zeros(N1)
        self._ck(self.L.pic_get_field(self.h, d, _ptr(E), _ptr(E64), _ptr(phi)))
        return E, E64, phi

    def set_field(self, d: int, E):
        E = np.ascontiguousarray(E, self.dtype)
        assert E.size == self.N[d] + 1
        self._ck(self.L.pic_set_field(self.h, d, _ptr(E)))

    def get_deposit(self, d: int, species: int) -> np.ndarray:
        D = np.zeros(self.N[d] + 1, np.int64)
        self._ck(self.L.pic_get_deposit(self.h, d, species, _ptr(D)))
        return D

    def set_deposit(self, d: int, species: int, D):
        D = np.ascontiguousarray(D, np.int64)
        self._ck(self.L.pic_set_deposit(self.h, d, species, _ptr(D)))

    def get_energy_deposit(self, d: int = 0) -> np.ndarray:
        Q = np.zeros(self.N[d] + 1, np.int64)
        self._ck(self.L.pic_get_energy_deposit(self.h, d, _ptr(Q)))
        return Q

    def counters(self, d: int = 0) -> dict:
        c = NV.PicCounters()
        self._ck(self.L.pic_get_counters(self.h, d, C.byref(c)))
        return c.as_dict()

    def derived(self, d: int = 0) -> dict:
        o = NV.PicDerived()
        self._ck(self.L.pic_get_derived(self.h, d, C.byref(o)))
        return o.as_dict()

    def tables(self, g: int = 0):
        n = self.gases[g].n_pts
        Te = np.zeros((n, 4), self.dtype)
        Ti = np.zeros((n, 2), self.dtype)
        self._ck(self.L.pic_get_tables(self.h, g, _ptr(Te), _ptr(Ti)))
        return Te, Ti

    def moments(self, d: int = 0) -> dict:
        N1 = self.N[d] + 1
        ne, ni, me = np.zeros(N1), np.zeros(N1), np.zeros(N1)
        m = NV.PicMoments()
        m.n_e, m.n_i, m.mean_eps = ne.ctypes.data, ni.ctypes.data, me.ctypes.data
        self._ck(self.L.pic_moments(self.h, d, C.byref(m)))
        return {"n_e": ne, "n_i": ni, "mean_eps": me, "steps": m.steps, "count": list(m.count),
                "absorbed": [[m.absorbed[a][b] for b in range(2)] for a in range(2)],
                "flux": [[m.flux[a][b] for b in range(2)] for a in range(2)], "surface_charge": m.surface_charge,
                "periods_done": m.periods_done, "steady_period": None if m.steady_period < 0 else m.steady_period,
                "steady_metric": m.steady_metric, "steady": bool(m.steady), "J_amp": m.J_amp, "J_last": m.J_last}

    def reset_moments(self):
        self._ck(self.L.pic_reset_moments(self.h))

    def load_profiles(self, profiles):
        """Warm start from profiles (n_discharges, 3, n_pts): n_e, n_i (m^-3), mean electron energy (eV)."""
        a = np.ascontiguousarray(profiles, np.float64)
        if a.ndim == 2:
            a = a[None]
        assert a.shape[0] == len(self.N) and a.shape[1] == 3
        self._ck(self.L.pic_load_profiles(self.h, a.shape[2], _ptr(a)))

    def period_counts(self, d: int = 0, first: int = 0, n=None) -> np.ndarray:
        """(periods, 2) mean superparticle counts per completed rf period (electrons, ions)."""
        done = C.c_int64()
        self._ck(self.L.pic_period_counts(self.h, d, 0, 0, None, C.byref(done)))
        if n is None:
            n = done.value - first
        out = np.zeros((max(n, 0), 2))
        if n > 0:
            self._ck(self.L.pic_period_counts(self.h, d, first, n, _ptr(out), C.byref(done)))
        return out

    def current(self, d: int = 0, first: int = 0, n=None) -> np.ndarray:
        """(steps, 2) discharge current density J(t) at z = 0 and z = d of steps first.., A/m^2."""
        done = C.c_int64()
        self._ck(self.L.pic_current(self.h, d, 0, 0, None, C.byref(done)))
        if n is None:
            n = done.value - first
        out = np.zeros((max(n, 0), 2))
        if n > 0:
            self._ck(self.L.pic_current(self.h, d, first, n, _ptr(out), C.byref(done)))
        return out

    def current_amplitude(self, d: int = 0, first: int = 0, n=None) -> np.ndarray:
        """First-harmonic amplitude of J(t) at z = 0 of each completed rf period, A/m^2."""
        done = C.c_int64()
        self._ck(self.L.pic_current_amplitude(self.h, d, 0, 0, None, C.byref(done)))
        if n is None:
            n = done.value - first
        out = np.zeros(max(n, 0))
        if n > 0:
            self._ck(self.L.pic_current_amplitude(self.h, d, first, n, _ptr(out), C.byref(done)))
        return out

    def set_current_drive(self, d: int = 0, J0: float = 0.0):
        """Current-driven mode (pic_set_current_drive): V0 <- V0 J0 / J_calc after every rf period."""
        self._ck(self.L.pic_set_current_drive(self.h, d, float(J0)))

    def voltage_amplitude(self, d: int = 0, first: int = 0, n=None):
        """(V0 applied in each completed rf period, V0 in effect now)."""
        done, vn = C.c_int64(), C.c_double()
        self._ck(self.L.pic_voltage_amplitude(self.h, d, 0, 0, None, C.byref(done), C.byref(vn)))
        if n is None:
            n = done.value - first
        out = np.zeros(max(n, 0))
        if n > 0:
            self._ck(self.L.pic_voltage_amplitude(self.h, d, first, n, _ptr(out), C.byref(done), None))
        return out, vn.value

    def set_diagnostics(self, period_steps: int = 0, phase_step: int = 0, sample_every: int = 0,
                        eedf_bins: int = 200, eedf_de_eV: float = 0.5, fast_eV: float = 0.0, off: bool = False):
        """Kinetic diagnostics of the electrons (pic_set_diagnostics): rf-phase snapshots at the
        steps n with n % period_steps == phase_step, EEDF and fast-electron samples every
        sample_every steps. off=True switches them off."""
        if off:
            self._ck(self.L.pic_set_diagnostics(self.h, None))
            self._eedf_bins = 0
            return
        cfg = NV.PicDiagConfig(period_steps, phase_step, sample_every, eedf_bins, eedf_de_eV, fast_eV)
        self._ck(self.L.pic_set_diagnostics(self.h, C.byref(cfg)))
        self._eedf_bins = eedf_bins

    def reset_diagnostics(self):
        self._ck(self.L.pic_reset_diagnostics(self.h))

    def diagnostics(self, d: int = 0) -> dict:
        """Read-out of pic_diagnostics: node profiles (N+1) E, n_e, mean_eps, gamma_e, q_e, heating,
        ion_rate, n_fast (snapshot averages), n_fast_avg (sample average), the EEDF f0(U)/n_e at
        the bin centres, and the numbers of snapshots and samples."""
        N1 = self.N[d] + 1
        keys = ("E", "n_e", "mean_eps", "gamma_e", "q_e", "heating", "ion_rate", "n_fast", "n_fast_avg")
        out = {k: np.zeros(N1) for k in keys}
        out["eedf"] = np.zeros(max(getattr(self, "_eedf_bins", 0), 1))
        sn, sm = C.c_int64(), C.c_int64()
        self._ck(self.L.pic_diagnostics(self.h, d, *[_ptr(out[k]) for k in keys], _ptr(out["eedf"]),
                                        C.byref(sn), C.byref(sm)))
        out["snapshots"], out["samples"] = sn.value, sm.value
        return out

    def sweep_timing(self, enable: bool = True):
        ms = C.c_double()
        n = C.c_int64()
        self._ck(self.L.pic_sweep_timing(self.h, 1 if enable else 0, C.byref(ms), C.byref(n)))
        return ms.value, n.value


def debug_wait(arrive: bool, tries: int) -> int:
    """Status of pic_debug_wait (PIC_OK or PIC_ERR_TIMEOUT), returned rather than raised."""
    return int(NV.lib().pic_debug_wait(1 if arrive else 0, int(tries)))


def debug_philox(ctr: np.ndarray, key) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros_like(ctr)
    NV.check(NV.lib().pic_debug_philox(ctr.shape[0], _ptr(ctr), _ptr(k), _ptr(out)))
    return out


def debug_math(x: np.ndarray, y: np.ndarray):
    x = np.ascontiguousarray(x, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    lg, sn, cs = (np.zeros_like(x) for _ in range(3))
    NV.check(NV.lib().pic_debug_math(x.size, _ptr(x), _ptr(y), _ptr(lg), _ptr(sn), _ptr(cs)))
    return lg, sn, cs
