"""ctypes binding of libcmc.so (include/cmc.h): names and arguments as in C.

Argument marshalling only.  The shared library must have been built
(``paper_1206_5878_gb300._build.build()``); importing this module without it
raises, so nothing can silently run elsewhere.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

_d = ctypes.c_double
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_p = ctypes.c_void_p
_pp = ctypes.POINTER(ctypes.c_void_p)

CMC_OK, CMC_EINVAL, CMC_ENOMEM, CMC_ECUDA, CMC_ENOCONV, CMC_ETIMEOUT, CMC_EPOISONED = range(7)
STATUS_NAMES = {0: "CMC_OK", 1: "CMC_EINVAL", 2: "CMC_ENOMEM", 3: "CMC_ECUDA",
                4: "CMC_ENOCONV", 5: "CMC_ETIMEOUT", 6: "CMC_EPOISONED"}
STAT_NAMES = ("escaped", "degenerate", "cap_hits", "trials", "violations", "clamps",
              "angle_fails", "ties", "fp64_trials", "clamp_energy", "collisions",
              "collision_energy", "envelope_fp64")
CMC_NSTATS = len(STAT_NAMES)
DIAG_FIELDS = ("step", "dt", "nbound", "K", "W", "E_total", "M_esc", "E_esc", "trials",
               "err")
STAGE_NAMES = ("timestep", "relax", "turning", "orbit", "sort", "gather", "potential",
               "correction", "end")


class cmc_config(ctypes.Structure):
    _fields_ = [("precision", _i32), ("bin_size", _i32), ("theta_max", _d), ("gamma", _d),
                ("max_trials", _i32), ("energy_correction", _i32), ("orbit_block", _i32),
                ("autotune", _i32), ("orbit_variant", _i32), ("rng", _i32),
                ("relax_variant", _i32), ("collisions", _i32), ("diag_ring", _i32),
                ("binaries", _i32), ("x_bb", _d), ("x_bs", _d), ("sort_packed", _i32)]


# exported symbol -> (restype, argtypes); the list is the ABI of include/cmc.h
SIGNATURES = {
    "cmc_config_default": (None, [ctypes.POINTER(cmc_config)]),
    "cmc_init": (_i32, [_pp, ctypes.POINTER(cmc_config), _i32, _p, _p, _p, _p, _p, _p, _p,
                        _i32, _p]),
    "cmc_step": (_i32, [_p, _i32]),
    "cmc_step_profiled": (_i32, [_p, _i32, _p]),
    "cmc_energy": (_i32, [_p, _p]),
    "cmc_lagrange_radii": (_i32, [_p, _p, _i32, _p]),
    "cmc_core": (_i32, [_p, _p]),
    "cmc_get_rng_state": (_i32, [_p, _p, _p]),
    "cmc_set_rng_state": (_i32, [_p, _p, _i64]),
    "cmc_get_state": (_i32, [_p, _p, _p, _p, _p, _p, _p, _p, _i32]),
    "cmc_set_state": (_i32, [_p, _p, _p, _p, _p, _p, _i64, _i32]),
    "cmc_get_nbound": (_i32, [_p, _p]),
    "cmc_get_dt": (_i32, [_p, _p]),
    "cmc_get_stats": (_i32, [_p, _p]),
    "cmc_get_escaped": (_i32, [_p, _p]),
    "cmc_get_diagnostics": (_i32, [_p, _p, _p]),
    "cmc_debug_check": (_i32, [_p]),
    "cmc_is_debug_build": (_i32, []),
    "cmc_set_escaped": (_i32, [_p, _p]),
    "cmc_kernels_per_step": (_i32, [_p]),
    "cmc_get_tuning": (_i32, [_p, _p]),
    "cmc_set_stream": (_i32, [_p, _p]),
    "cmc_last_error": (ctypes.c_char_p, [_p]),
    "cmc_destroy": (None, [_p]),
    "cmc_rng_philox": (_i32, [_i64, _p, _u64, _p, _p]),
    "cmc_sort_radius": (_i32, [_i64, _p, _p, _p, _p]),
    "cmc_potential": (_i32, [_i64, _p, _p, _p, _p, _p]),
    "cmc_timestep": (_i32, [_i64, _p, _p, _p, _p, _i32, _d, _d, _p, _p, _p]),
    "cmc_relax": (_i32, [_i64, _p, _p, _p, _p, _p, _i32, _d, _d, _u64, _u32, _p]),
    "cmc_orbit": (_i32, [_i64, _p, _p, _p, _p, _p, _u64, _u32, _i32, _i32, _p, _p, _p, _p, _p,
                         _p, _p, _p, _p]),
    "cmc_energy_correction": (_i32, [_i64, _p, _p, _p, _p, _p, _p, _p]),
    "cmc_potential_static": (_i32, [_i64, _p, _p, _p, _p, _p]),
    "cmc_check_arith": (_i32, [_i32, _u64, _u64, _p]),
    "cmc_set_wait_limits": (_i32, [_i32, _i64]),
    "cmc_set_radii": (_i32, [_p, _p, _i32]),
    "cmc_get_radii": (_i32, [_p, _p, _i32]),
    "cmc_set_binaries": (_i32, [_p, _p, _i32]),
    "cmc_get_binaries": (_i32, [_p, _p, _i32]),
    "cmc_set_dt_cap": (_i32, [_p, _p]),
    "cmc_tse": (_d, [_d, _d, _d]),
}

_libs = {}


def lib_path(debug: bool = False) -> str:
    return _build.LIB_DEBUG if debug else _build.LIB


def load(debug: bool = False):
    """Load libcmc.so, or with debug=True libcmc_debug.so (the build with
    device-side index checks); raises RuntimeError when it has not been
    built."""
    if debug in _libs:
        return _libs[debug]
    path = lib_path(debug)
    if not os.path.exists(path):
        raise RuntimeError(
            "%s is not built; run paper_1206_5878_gb300._build.build(debug=%s) "
            "(needs nvcc) before using the CUDA path" % (os.path.basename(path), debug))
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _libs[debug] = lib
    return lib


class CMCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def check(status: int, ctx=None, lib=None):
    if status != CMC_OK:
        msg = (lib or load()).cmc_last_error(ctx)
        raise CMCError(status, msg.decode() if msg else "")
