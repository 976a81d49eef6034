"""ctypes declarations of the C ABI in include/helios.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(HERE, "libhelios.so")

HELIOS_OK, HELIOS_EINVAL, HELIOS_ENOMEM, HELIOS_ECUDA, HELIOS_ENOCONV = 0, -1, -2, -3, -5
HELIOS_DIRECT = -1          # n_passes: the exact column solve instead of scattering passes
ATM_ACTIVE, ATM_CONVERGED, ATM_NOT_CONVERGED, ATM_NONFINITE, ATM_OUT_OF_RANGE = 0, 1, 2, 3, 4

c_int, c_double, c_void_p, c_int64 = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64


class KTable(ctypes.Structure):
    _fields_ = [("nP", c_int), ("nT", c_int), ("L", c_int), ("G", c_int),
                ("log10P0", c_double), ("dlog10P", c_double), ("T0", c_double), ("dT", c_double),
                ("kappa", c_void_p)]


class Batch(ctypes.Structure):
    _fields_ = [("A", c_int), ("n_layers", c_void_p), ("n_bins", c_void_p), ("table_id", c_void_p),
                ("P_top_bar", c_void_p), ("P_bot_bar", c_void_p), ("grav", c_void_p), ("T_irr", c_void_p),
                ("T_int", c_void_p), ("T_star", c_void_p), ("nu_edges", c_void_p), ("omega0", c_void_p),
                ("g0", c_void_p), ("species_off", c_void_p), ("species_table", c_void_p),
                ("species_weight", c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("D", c_double), ("dtau_iso", c_double), ("w0_pure", c_double), ("tol", c_double),
                ("fpre_num", c_double), ("fpre_exp", c_double), ("osc_down", c_double), ("osc_up", c_double),
                ("mult_max", c_double), ("T_floor", c_double), ("n_scat", c_int), ("max_iter", c_int),
                ("grey_mode", c_int), ("printed_gradient", c_int), ("bins_per_item", c_int),
                ("check_every", c_int), ("persistent", c_int), ("iso_layers", c_int), ("device_loop", c_int), ("direct", c_int), ("rayleigh", c_int),
                ("col_lanes", c_int), ("tabulate", c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("layers", c_int64), ("interfaces", c_int64), ("points", c_int64), ("bins", c_int64),
                ("cells", c_int64), ("passes", c_int), ("workspace_bytes", c_int64), ("sweep_launches", c_int),
                ("fused_finalize", c_int), ("warm_floats", c_int64), ("spec_floats", c_int64)]


EXPORTS = ["helios_default_params", "helios_version", "helios_last_error", "helios_create", "helios_destroy",
           "helios_plan_create", "helios_plan_destroy", "helios_plan_info", "helios_plan_state_bytes",
           "helios_plan_state_export", "helios_plan_state_import", "helios_interp_opacity",
           "helios_flux_sweep", "helios_temp_update", "helios_re_step", "helios_re_step_host", "helios_solve_re", "helios_measure_peaks", "helios_device_recip", "helios_plan_set_timing",
           "helios_plan_last_sweep_ms", "helios_plan_sweep_times", "helios_flux_sweep_noalloc",
           "helios_autotune", "helios_mlp_create", "helios_mlp_destroy", "helios_mlp_params", "helios_mlp_params_changed", "helios_mlp_forward",
           "helios_mlp_grad", "helios_mlp_adam", "helios_mlp_train_step", "helios_mlp_initial_profiles", "helios_mlp_error",
           "helios_column_stats", "helios_standardize"]

_lib = None


def load(path: str = SO_PATH):
    """Load libhelios.so; raises if the CUDA library has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing: build it with paper_1606_05474_b300/_build.py")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp = c_void_p
    lib.helios_default_params.argtypes = [P(Params)]
    lib.helios_default_params.restype = None
    lib.helios_version.restype = c_int
    lib.helios_last_error.restype = ctypes.c_char_p
    lib.helios_create.argtypes = [P(vp), c_int]
    lib.helios_destroy.argtypes = [vp]
    lib.helios_plan_create.argtypes = [vp, P(Batch), P(KTable), c_int, P(Params), P(vp)]
    lib.helios_plan_destroy.argtypes = [vp]
    lib.helios_plan_info.argtypes = [vp, P(PlanInfo)]
    lib.helios_plan_state_bytes.argtypes = [vp, P(c_int64)]
    lib.helios_plan_state_export.argtypes = [vp, vp, vp]
    lib.helios_plan_state_import.argtypes = [vp, vp, vp]
    lib.helios_interp_opacity.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.helios_flux_sweep.argtypes = [vp, vp, c_int, c_int, vp, vp, vp, vp, vp, vp]
    lib.helios_temp_update.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.helios_re_step.argtypes = [vp, vp, c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.helios_re_step_host.argtypes = [vp, vp, vp, c_int, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.helios_measure_peaks.argtypes = [vp, P(c_double), P(c_double)]
    lib.helios_device_recip.argtypes = [vp, vp, c_int, vp]
    lib.helios_solve_re.argtypes = [vp, vp, vp, vp, vp]
    lib.helios_plan_set_timing.argtypes = [vp, c_int]
    lib.helios_plan_last_sweep_ms.argtypes = [vp, P(ctypes.c_float)]
    lib.helios_plan_sweep_times.argtypes = [vp, vp, c_int, P(c_int)]
    lib.helios_autotune.argtypes = [vp, P(Batch), P(KTable), c_int, P(Params), ctypes.c_char_p, P(Params)]
    lib.helios_mlp_create.argtypes = [vp, c_int, c_int, c_int, c_int, ctypes.c_ulonglong, c_int, P(vp)]
    lib.helios_mlp_destroy.argtypes = [vp]
    lib.helios_mlp_params.argtypes = [vp, P(vp), P(vp), P(ctypes.c_longlong)]
    lib.helios_mlp_params_changed.argtypes = [vp]
    lib.helios_mlp_forward.argtypes = [vp, vp, vp, c_int, vp]
    lib.helios_mlp_grad.argtypes = [vp, vp, vp, c_int, vp, vp]
    lib.helios_mlp_adam.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, vp]
    lib.helios_mlp_train_step.argtypes = [vp, vp, vp, c_int, ctypes.c_float, vp, vp]
    lib.helios_mlp_initial_profiles.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, c_double, c_double, vp, vp, vp]
    lib.helios_mlp_error.argtypes = [vp, P(c_int)]
    lib.helios_column_stats.argtypes = [vp, c_int, c_int, c_double, vp, vp, vp]
    lib.helios_standardize.argtypes = [vp, vp, vp, c_int, c_int, vp, vp]
    lib.helios_flux_sweep_noalloc.argtypes = [P(Batch), P(KTable), P(Params), vp, c_int, vp, vp, vp, vp]
    for name in EXPORTS:
        if name not in ("helios_default_params", "helios_version", "helios_last_error"):
            getattr(lib, name).restype = c_int
    _lib = lib
    return lib


class HeliosError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"helios error {code}: {msg}")
        self.code = code


def check(rc: int):
    if rc != HELIOS_OK:
        raise HeliosError(rc, load().helios_last_error().decode(errors="replace"))
    return rc
