"""ctypes binding of libpic.so (include/pic.h): structures and prototypes only.

There is no fallback: if the CUDA library cannot be loaded, importing the
binding raises, and every computation happens in the library's kernels.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpic.so")

PIC_OK = 0
STATUS = {0: "PIC_OK", -1: "PIC_ERR_ARG", -2: "PIC_ERR_CUDA", -3: "PIC_ERR_CAPACITY", -4: "PIC_ERR_TIMEOUT",
          -5: "PIC_ERR_TABLE", -6: "PIC_ERR_NONFINITE", -7: "PIC_ERR_STATE"}


class PicGas(C.Structure):
    _fields_ = [("mass_kg", C.c_double), ("n_exc", C.c_int32), ("n_pts", C.c_int32), ("de_eV", C.c_double),
                ("eps_exc_eV", C.c_double * 2), ("eps_iz_eV", C.c_double),
                ("sigma_e", C.POINTER(C.c_double)), ("sigma_i", C.POINTER(C.c_double))]


class PicWeights(C.Structure):
    _fields_ = [("w_e", C.c_double), ("w_i", C.c_double), ("n_e0", C.c_int64), ("n_i0", C.c_int64),
                ("capacity_e", C.c_int64), ("capacity_i", C.c_int64), ("T_e0_eV", C.c_double),
                ("T_i0_K", C.c_double), ("gamma_see", C.c_double), ("steps_per_period", C.c_int32),
                ("reserved", C.c_int32)]


class PicDischarge(C.Structure):
    _fields_ = [("gas", C.c_int32), ("n_cells", C.c_int32), ("gap_m", C.c_double), ("p_Pa", C.c_double),
                ("T_gas_K", C.c_double), ("f_rf_Hz", C.c_double), ("V_rf_V", C.c_double), ("dt_s", C.c_double),
                ("weights", PicWeights), ("discharge_id", C.c_uint32), ("reserved", C.c_int32)]


class PicOptions(C.Structure):
    _fields_ = [("precision", C.c_int32), ("sort_every", C.c_int32), ("block", C.c_int32), ("ppt", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("use_graph", C.c_int32), ("cuda_stream", C.c_void_p),
                ("load", C.c_int32), ("leapfrog", C.c_int32)]


class PicMoments(C.Structure):
    _fields_ = [("n_e", C.c_void_p), ("n_i", C.c_void_p), ("mean_eps", C.c_void_p), ("steps", C.c_int64),
                ("count", C.c_int64 * 2), ("absorbed", (C.c_double * 2) * 2), ("flux", (C.c_double * 2) * 2),
                ("surface_charge", C.c_double), ("periods_done", C.c_int64), ("steady_period", C.c_int64),
                ("steady_metric", C.c_double), ("steady", C.c_int32), ("reserved", C.c_int32),
                ("J_amp", C.c_double), ("J_last", C.c_double)]


class PicDiagConfig(C.Structure):
    _fields_ = [("period_steps", C.c_int32), ("phase_step", C.c_int32), ("sample_every", C.c_int32),
                ("eedf_bins", C.c_int32), ("eedf_de_eV", C.c_double), ("fast_eV", C.c_double)]


class PicCounters(C.Structure):
    _fields_ = [("absorbed", (C.c_int64 * 2) * 2), ("collisions_e", C.c_int64 * 4),
                ("collisions_i", C.c_int64 * 2), ("null_inelastic", C.c_int64), ("see_emitted", C.c_int64),
                ("candidates", C.c_int64 * 2), ("table_clamped", C.c_int64 * 2)]

    def as_dict(self) -> dict:
        return {"absorbed": [[self.absorbed[a][b] for b in range(2)] for a in range(2)],
                "collisions_e": list(self.collisions_e), "collisions_i": list(self.collisions_i),
                "null_inelastic": self.null_inelastic, "see_emitted": self.see_emitted,
                "candidates": list(self.candidates), "table_clamped": list(self.table_clamped)}


class PicDerived(C.Structure):
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


# name -> (restype, argtypes)
_vp, _i32, _i64, _u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
PROTOTYPES = {
    "pic_default_options": (None, [C.POINTER(PicOptions)]),
    "pic_batch_create": (C.c_int, [C.POINTER(_vp), C.POINTER(PicGas), _i32, C.POINTER(PicDischarge), _i32, _u64,
                                   C.POINTER(PicOptions)]),
    "pic_create": (C.c_int, [C.POINTER(_vp), C.POINTER(PicGas), C.c_double, C.c_double, C.c_double, C.c_double,
                             C.c_double, _i32, C.c_double, C.POINTER(PicWeights), _u64, C.POINTER(PicOptions)]),
    "pic_step": (C.c_int, [_vp, _i64]),
    "pic_sweep": (C.c_int, [_vp]),
    "pic_sort": (C.c_int, [_vp]),
    "pic_solve": (C.c_int, [_vp]),
    "pic_sync": (C.c_int, [_vp]),
    "pic_moments": (C.c_int, [_vp, _i32, C.POINTER(PicMoments)]),
    "pic_reset_moments": (C.c_int, [_vp]),
    "pic_destroy": (None, [_vp]),
    "pic_last_error": (C.c_char_p, [_vp]),
    "pic_status_string": (C.c_char_p, [C.c_int]),
    "pic_get_count": (C.c_int, [_vp, _i32, _i32, C.POINTER(_i64)]),
    "pic_get_state": (C.c_int, [_vp, _i32, _i32, _i64, _vp, _vp, _vp, _vp, _vp, C.POINTER(_i64)]),
    "pic_set_state": (C.c_int, [_vp, _i32, _i32, _i64, _vp, _vp, _vp, _vp, _vp]),
    "pic_get_field": (C.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "pic_set_field": (C.c_int, [_vp, _i32, _vp]),
    "pic_get_deposit": (C.c_int, [_vp, _i32, _i32, _vp]),
    "pic_set_deposit": (C.c_int, [_vp, _i32, _i32, _vp]),
    "pic_get_energy_deposit": (C.c_int, [_vp, _i32, _vp]),
    "pic_get_step": (C.c_int, [_vp, C.POINTER(_i64)]),
    "pic_set_step": (C.c_int, [_vp, _i64]),
    "pic_get_counters": (C.c_int, [_vp, _i32, C.POINTER(PicCounters)]),
    "pic_get_derived": (C.c_int, [_vp, _i32, C.POINTER(PicDerived)]),
    "pic_get_tables": (C.c_int, [_vp, _i32, _vp, _vp]),
    "pic_sweep_timing": (C.c_int, [_vp, _i32, C.POINTER(C.c_double), C.POINTER(_i64)]),
    "pic_debug_philox": (C.c_int, [_i64, _vp, _vp, _vp]),
    "pic_debug_math": (C.c_int, [_i64, _vp, _vp, _vp, _vp, _vp]),
    "pic_sort_noalloc": (C.c_int, [_vp, _vp, _vp, _vp, _i64, _i32, _i32, _vp]),
    "pic_period_counts": (C.c_int, [_vp, _i32, _i64, _i64, _vp, C.POINTER(_i64)]),
    "pic_current": (C.c_int, [_vp, _i32, _i64, _i64, _vp, C.POINTER(_i64)]),
    "pic_current_amplitude": (C.c_int, [_vp, _i32, _i64, _i64, _vp, C.POINTER(_i64)]),
    "pic_load_profiles": (C.c_int, [_vp, _i32, _vp]),
    "pic_debug_wait": (C.c_int, [_i32, _i32]),
    "pic_set_current_drive": (C.c_int, [_vp, _i32, C.c_double]),
    "pic_voltage_amplitude": (C.c_int, [_vp, _i32, _i64, _i64, _vp, C.POINTER(_i64), C.POINTER(C.c_double)]),
    "pic_set_diagnostics": (C.c_int, [_vp, C.POINTER(PicDiagConfig)]),
    "pic_reset_diagnostics": (C.c_int, [_vp]),
    "pic_diagnostics": (C.c_int, [_vp, _i32] + [_vp] * 10 + [C.POINTER(_i64), C.POINTER(_i64)]),
    # include/mlp.h
    "mlp_create": (C.c_int, [C.POINTER(_vp), _i32, _vp, _i32, _u64, _vp]),
    "mlp_param_count": (_i64, [_vp]),
    "mlp_set_params": (C.c_int, [_vp, _vp]),
    "mlp_get_params": (C.c_int, [_vp, _vp]),
    "mlp_forward": (C.c_int, [_vp, _i32, _vp, _vp]),
    "mlp_loss_grad": (C.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "mlp_get_grads": (C.c_int, [_vp, _vp]),
    "mlp_adam": (C.c_int, [_vp, C.c_float, C.c_float, C.c_float, C.c_float]),
    "mlp_train_step": (C.c_int, [_vp, _i32, _vp, _vp, C.c_float, _vp]),
    "mlp_sync": (C.c_int, [_vp]),
    "mlp_destroy": (None, [_vp]),
    "mlp_last_error": (C.c_char_p, [_vp]),
}

_lib = None


def lib() -> C.CDLL:
    """Loads libpic.so (built by paper_1608_04601_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpic.so not found at {LIB_PATH}: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class PicError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


def check(status: int, ctx=None) -> None:
    if status != PIC_OK:
        msg = ""
        if ctx:
            m = lib().pic_last_error(ctx)
            msg = m.decode() if m else ""
        raise PicError(status, msg)
