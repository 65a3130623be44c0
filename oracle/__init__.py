"""Oracle for the Henon Monte Carlo timestep: plain, slow, FP64 C code.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may.  The C source (``cmc_oracle.c``) shares no code with the
CUDA library; both follow the same paper (Pattabiraman et al., sections 2.1
and 3.3) and the same readings of it.

``build()`` compiles the C file with gcc into ``liboracle_cmc.so`` beside it
(no fused multiply-add contraction, IEEE round-to-nearest throughout); the
wrappers below take and return numpy arrays.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_cmc.so")
_lock = threading.Lock()
_lib = None

GAMMA = 0.1              # Coulomb logarithm ln(gamma N), gamma = 0.1 (Eq. 20)
BIN_SIZE = 20            # timestep bins of 20 stars (section 3.3)
THETA_MAX = math.pi / 2  # maximum deflection angle in Eq. 7


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (seconds); returns the library path."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
           "-fno-strict-aliasing", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            _declare(lib)
            _lib = lib
    return _lib


_d = ctypes.c_double
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_p = ctypes.c_void_p


def _declare(lib):
    sig = {
        "or_philox_bulk": (None, [_i64, _p, _u64, _p]),
        "or_u01": (_d, [_u32, _u32]),
        "or_sort_perm": (None, [_i64, _p, _p, _p]),
        "or_potential_recursion": (None, [_i64, _p, _p, _p]),
        "or_potential_brute": (None, [_i64, _p, _p, _p]),
        "or_potential_dd": (None, [_i64, _p, _p, _p]),
        "or_phi_of_r": (_d, [_i64, _p, _p, _d]),
        "or_timestep": (_d, [_i64, _p, _p, _p, _p, _i32, _d, _d, _p]),
        "or_encounter": (ctypes.c_int, [_d, _d, _d, _d, _d, _d, _d, _d, _d, _u64, _u32,
                                        _u32, _p]),
        "or_disk_angle_pub": (ctypes.c_int, [_u64, _u32, _u32, _u32, _p]),
        "or_relax": (_i64, [_i64, _p, _p, _p, _p, _p, _i32, _d, _d, _u64, _u32]),
        "or_orbit_star": (ctypes.c_int, [_i64, _i64, _p, _p, _d, _d, _u32, _u64, _u32,
                                         _i32, _p, _p]),
        "or_orbit_star_env": (ctypes.c_int, [_i64, _i64, _p, _p, _d, _d, _u32, _u64, _u32,
                                             _i32, _d, _p, _p]),
        "or_orbit_sample": (None, [_i64, _p, _p, _p, _p, _p, _i64, _p, _u64, _u32, _i32,
                                   _p]),
        "or_orbit_all": (None, [_i64, _p, _p, _p, _p, _p, _u64, _u32, _i32,
                                _p, _p, _p, _p, _p, _p, _p, _p, _p]),
        "or_energy_correction": (_i64, [_i64, _p, _p, _p, _p, _p, _p, _p]),
        "or_energy": (None, [_i64, _p, _p, _p, _p, _p]),
        "or_energy_W_brute": (_d, [_i64, _p, _p]),
        "or_lagrange_radii": (None, [_i64, _p, _p, _p, _i32, _p]),
        "or_core": (None, [_i64, _p, _p, _p]),
        "or_taus_next": (_u32, [_p]),
        "or_taus_pow2": (None, [ctypes.c_int, ctypes.c_int, _p]),
        "or_taus_pow": (None, [ctypes.c_int, _u64, _p]),
        "or_gf2_apply_pub": (_u32, [_p, _u32]),
        "or_taus_seed": (None, [_u64, _p]),
        "or_taus_streams": (None, [_u64, _i64, _p]),
        "or_taus_bind": (None, [_p]),
        "or_core_rho": (None, [_i64, _p, _p, _p]),
        "or_step": (_d, [_i64, _p, _p, _p, _p, _p, _p, _p, _u64, _u32, _i32, _d, _d,
                         _i32, _i32, _i32, _p, _p]),
        "or_step_col": (_d, [_i64, _p, _p, _p, _p, _p, _p, _p, _p, _u64, _u32, _i32, _d, _d,
                             _i32, _i32, _i32, _p, _p, _p, _p, _d, _d, _d]),
        "or_tbinary": (_d, [_i64, _p, _p, _p, _p, _p, _d, _d, _p]),
        "or_tse": (_d, [_d, _d, _d]),
        "or_encounter_radii": (ctypes.c_int, [_d, _d, _d, _d, _d, _d, _d, _d, _d, _d, _d,
                                              _u64, _u32, _u32, _p]),
        "or_relax_col": (_i64, [_i64, _p, _p, _p, _p, _p, _p, _i32, _d, _d, _u64, _u32, _p, _p,
                                _p]),
        "or_tcoll": (_d, [_i64, _p, _p, _p, _p, _p]),
        "or_cbrt": (_d, [_d]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u32a(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


# --------------------------------------------------------------------------
# parameters derived on the host
# --------------------------------------------------------------------------
def t_rel_prefactor(theta_max: float = THETA_MAX) -> float:
    """(theta_max / (pi/2)) * (pi/32), the constant of Eq. 7."""
    return (theta_max / (math.pi / 2)) * (math.pi / 32)


def coulomb_log(n: int, gamma: float = GAMMA) -> float:
    """ln(gamma N) (Eq. 7, with gamma = 0.1 as in Eq. 20)."""
    return math.log(gamma * float(n))


# --------------------------------------------------------------------------
# stage wrappers
# --------------------------------------------------------------------------
def philox(ctr: np.ndarray, seed: int) -> np.ndarray:
    """Philox4x32-10 blocks for counters ctr (n x 4 uint32), key = seed."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    _L().or_philox_bulk(ctr.shape[0], _ptr(ctr), seed, _ptr(out))
    return out


def u01(lo: int, hi: int) -> float:
    return _L().or_u01(lo, hi)


def sort_perm(r, ids) -> np.ndarray:
    r = _f64(r)
    ids = _u32a(ids)
    perm = np.empty(r.shape[0], dtype=np.int64)
    _L().or_sort_perm(r.shape[0], _ptr(r), _ptr(ids), _ptr(perm))
    return perm


def potential(r, m, mode: str = "recursion") -> np.ndarray:
    r = _f64(r)
    m = _f64(m)
    phi = np.empty_like(r)
    fn = {"recursion": "or_potential_recursion", "brute": "or_potential_brute",
          "dd": "or_potential_dd"}[mode]
    getattr(_L(), fn)(r.shape[0], _ptr(r), _ptr(m), _ptr(phi))
    return phi


def phi_of_r(r, phi, rq: float) -> float:
    r = _f64(r)
    phi = _f64(phi)
    return _L().or_phi_of_r(r.shape[0], _ptr(r), _ptr(phi), float(rq))


def timestep(r, vr, vt, m, lnL: float, bin_size: int = BIN_SIZE,
             pref: float | None = None):
    r, vr, vt, m = _f64(r), _f64(vr), _f64(vt), _f64(m)
    nb = r.shape[0]
    if pref is None:
        pref = t_rel_prefactor()
    nbin = np.zeros(max(1, (nb + bin_size - 1) // bin_size))
    dt = _L().or_timestep(nb, _ptr(r), _ptr(vr), _ptr(vt), _ptr(m), bin_size, pref,
                          lnL, _ptr(nbin))
    return dt, nbin[: (nb + bin_size - 1) // bin_size]


def relax(vr, vt, m, ids, nbin, dt: float, lnL: float, seed: int, step: int,
          bin_size: int = BIN_SIZE):
    vr = _f64(vr).copy()
    vt = _f64(vt).copy()
    m = _f64(m)
    ids = _u32a(ids)
    nbin = _f64(nbin)
    if nbin.shape[0] == 0:
        nbin = np.zeros(1)
    fails = _L().or_relax(vr.shape[0], _ptr(vr), _ptr(vt), _ptr(m), _ptr(ids), _ptr(nbin),
                          bin_size, dt, lnL, seed, step)
    return vr, vt, fails


def encounter_radii(m1, m2, vr1, vt1, vr2, vt2, R1, R2, n, dt, lnL, seed, ident, step):
    """The encounter with stellar radii (sticky spheres): 20 doubles, status
    out[15] = 2 for a merger, out[16] the collision probability, out[17]
    the dissipated energy."""
    out = np.zeros(20)
    _L().or_encounter_radii(m1, m2, vr1, vt1, vr2, vt2, R1, R2, n, dt, lnL, seed, ident, step,
                            _ptr(out))
    return out


def relax_radii(vr, vt, m, R, ids, nbin, dt: float, lnL: float, seed: int, step: int, r,
                phi, bin_size: int = BIN_SIZE):
    """Relaxation with sticky-sphere mergers (r, phi: the sorted radii and
    their potential); returns (vr, vt, m, R, mergers, their change of
    K + W)."""
    vr, vt, m, R = (_f64(a).copy() for a in (vr, vt, m, R))
    r, phi = _f64(r), _f64(phi)
    col = np.zeros(2)
    _L().or_relax_col(vr.shape[0], _ptr(vr), _ptr(vt), _ptr(m), _ptr(R), _ptr(_u32a(ids)),
                      _ptr(_f64(nbin)), bin_size, dt, lnL, seed, step, _ptr(col), _ptr(r),
                      _ptr(phi))
    return vr, vt, m, R, int(col[0]), col[1]


def tcoll(r, vr, vt, m, R) -> float:
    """Eq. 8's collision timestep over the innermost 300 bound stars."""
    r, vr, vt, m, R = (_f64(a) for a in (r, vr, vt, m, R))
    return _L().or_tcoll(r.shape[0], _ptr(r), _ptr(vr), _ptr(vt), _ptr(m), _ptr(R))


def tbinary(r, vr, vt, m, A, x_bb: float = 1.0, x_bs: float = 1.0):
    """Eqs. 9 and 10's binary-binary and binary-single timesteps over the
    innermost 300 bound stars (binaries: A > 0); returns (T_bb, T_bs)."""
    r, vr, vt, m, A = (_f64(a) for a in (r, vr, vt, m, A))
    tbs = np.zeros(1)
    tbb = _L().or_tbinary(r.shape[0], _ptr(r), _ptr(vr), _ptr(vt), _ptr(m), _ptr(A),
                          float(x_bb), float(x_bs), _ptr(tbs))
    return tbb, float(tbs[0])


def tse(M: float, T_prev: float, dm_se: float) -> float:
    """Eq. 11's stellar-evolution timestep."""
    return _L().or_tse(float(M), float(T_prev), float(dm_se))


def cbrt(v: float) -> float:
    return _L().or_cbrt(float(v))


def encounter(m1, m2, vr1, vt1, vr2, vt2, n, dt, lnL, seed, ident, step):
    """One representative encounter: dict with 3-D velocities before/after."""
    out = np.zeros(16)
    fails = _L().or_encounter(m1, m2, vr1, vt1, vr2, vt2, n, dt, lnL, seed, ident, step,
                              _ptr(out))
    return {"v1": out[0:3].copy(), "v2": out[3:6].copy(), "v1p": out[6:9].copy(),
            "v2p": out[9:12].copy(), "s2": out[12], "cosb": out[13], "w": out[14],
            "status": int(out[15]), "fails": fails}


def disk_angle(seed: int, ident: int, step: int, tag: int):
    cs = np.zeros(2)
    rc = _L().or_disk_angle_pub(seed, ident, step, tag, _ptr(cs))
    return cs[0], cs[1], rc


def orbit_star(k: int, r, phi, vr: float, vt: float, ident: int, seed: int, step: int,
               max_trials: int = 1000, F=None):
    """One star's orbit step (section 2.1 step 5).  F (optional, > 0): the
    rejection bound to use instead of 1.2 max g(s_j)."""
    r, phi = _f64(r), _f64(phi)
    out = np.zeros(8)
    viol = np.zeros(1, dtype=np.int64)
    if F is None:
        rc = _L().or_orbit_star(k, r.shape[0], _ptr(r), _ptr(phi), float(vr), float(vt),
                                int(ident), seed, step, max_trials, _ptr(out), _ptr(viol))
    else:
        rc = _L().or_orbit_star_env(k, r.shape[0], _ptr(r), _ptr(phi), float(vr), float(vt),
                                    int(ident), seed, step, max_trials, float(F), _ptr(out),
                                    _ptr(viol))
    return {"code": rc, "r_new": out[0], "vr": out[1], "vt": out[2], "phi_new": out[3],
            "rmin": out[4], "rmax": out[5], "F": out[6], "trials": int(out[7]),
            "violations": int(viol[0])}


def orbit_sample(r, phi, vr, vt, ids, ks, seed: int, step: int, max_trials: int = 1000):
    """New radii of the stars at sorted positions ks only (or_orbit_sample)."""
    r, phi, vr, vt = _f64(r), _f64(phi), _f64(vr), _f64(vt)
    ids = _u32a(ids)
    ks = np.ascontiguousarray(ks, dtype=np.int64)
    out = np.zeros(ks.shape[0])
    _L().or_orbit_sample(r.shape[0], _ptr(r), _ptr(phi), _ptr(vr), _ptr(vt), _ptr(ids),
                         ks.shape[0], _ptr(ks), seed, step, max_trials, _ptr(out))
    return out


def orbit_all(r, phi, vr, vt, ids, seed: int, step: int, max_trials: int = 1000):
    r, phi, vr, vt = _f64(r), _f64(phi), _f64(vr), _f64(vt)
    ids = _u32a(ids)
    nb = r.shape[0]
    outs = {k: np.zeros(nb) for k in ("r_new", "vr", "vt", "phi_new", "rmin", "rmax", "F")}
    code = np.zeros(nb, dtype=np.int32)
    stats = np.zeros(5, dtype=np.int64)
    _L().or_orbit_all(nb, _ptr(r), _ptr(phi), _ptr(vr), _ptr(vt), _ptr(ids), seed, step,
                      max_trials, _ptr(outs["r_new"]), _ptr(outs["vr"]), _ptr(outs["vt"]),
                      _ptr(outs["phi_new"]), _ptr(outs["rmin"]), _ptr(outs["rmax"]),
                      _ptr(outs["F"]), _ptr(code), _ptr(stats))
    outs["code"] = code
    outs["stats"] = stats
    return outs


def energy_correction(r, phi, vr, vt, r_old, c, want_tp: bool = False):
    r, phi, r_old, c = _f64(r), _f64(phi), _f64(r_old), _f64(c)
    vr = _f64(vr).copy()
    vt = _f64(vt).copy()
    tp = np.zeros(r.shape[0])
    clamps = _L().or_energy_correction(r.shape[0], _ptr(r), _ptr(phi), _ptr(vr), _ptr(vt),
                                       _ptr(r_old), _ptr(c), _ptr(tp))
    if want_tp:
        return vr, vt, clamps, tp
    return vr, vt, clamps


def energy(r, vr, vt, m):
    r, vr, vt, m = _f64(r), _f64(vr), _f64(vt), _f64(m)
    out = np.zeros(3)
    _L().or_energy(r.shape[0], _ptr(r), _ptr(vr), _ptr(vt), _ptr(m), _ptr(out))
    return out


def energy_W_brute(r, m) -> float:
    r, m = _f64(r), _f64(m)
    return _L().or_energy_W_brute(r.shape[0], _ptr(r), _ptr(m))


def lagrange_radii(r, m, fracs):
    r, m = _f64(r), _f64(m)
    fracs = _f64(fracs)
    out = np.zeros(fracs.shape[0])
    _L().or_lagrange_radii(r.shape[0], _ptr(r), _ptr(m), _ptr(fracs), fracs.shape[0],
                           _ptr(out))
    return out


def core(r, m):
    """Core density and density-weighted core radius (Eq. 19) from the
    6th-order radial density estimator: (rho_c, r_c, number of estimates)."""
    r, m = _f64(r), _f64(m)
    out = np.zeros(3)
    _L().or_core(r.shape[0], _ptr(r), _ptr(m), _ptr(out))
    return out[0], out[1], int(out[2])


def core_rho(r, m):
    """The per-star density estimates behind core() (0 where none)."""
    r, m = _f64(r), _f64(m)
    out = np.zeros(r.shape[0])
    _L().or_core_rho(r.shape[0], _ptr(r), _ptr(m), _ptr(out))
    return out


def taus_next(z, count=1):
    """count outputs of the combined Tausworthe generator from the four
    words z (a uint32 array of 4, advanced in place)."""
    assert z.dtype == np.uint32 and z.shape == (4,)
    return np.array([_L().or_taus_next(_ptr(z)) for _ in range(count)], dtype=np.uint32)


def taus_pow(j, D):
    """T_j^D as 32 columns (uint32), component j = 0..3."""
    out = np.zeros(32, dtype=np.uint32)
    _L().or_taus_pow(int(j), int(D), _ptr(out))
    return out


def taus_pow2(j, e):
    out = np.zeros(32, dtype=np.uint32)
    _L().or_taus_pow2(int(j), int(e), _ptr(out))
    return out


def gf2_apply(cols, v):
    cols = np.ascontiguousarray(cols, dtype=np.uint32)
    return int(_L().or_gf2_apply_pub(_ptr(cols), int(v)))


def taus_seed(seed):
    z = np.zeros(4, dtype=np.uint32)
    _L().or_taus_seed(int(seed), _ptr(z))
    return z


def taus_streams(seed, n_ids):
    """Starting words of the streams of ids 0..n_ids-1 (4 per id)."""
    t = np.zeros(4 * int(n_ids), dtype=np.uint32)
    _L().or_taus_streams(int(seed), int(n_ids), _ptr(t))
    return t


class taus_bound:
    """Within the block, the method's draws come from the given stream table
    (4 words per id, advanced in place) instead of Philox counters."""

    def __init__(self, table):
        assert table.dtype == np.uint32 and table.flags.c_contiguous
        self.table = table

    def __enter__(self):
        _L().or_taus_bind(_ptr(self.table))
        return self.table

    def __exit__(self, *a):
        _L().or_taus_bind(None)


def half_mass_relaxation_time(n, r_h, mass=1.0, gamma=0.1):
    """Eq. 20: t_rh = 0.138 N / ln(gamma N) (r_h^3 / (G M))^(1/2), G = 1."""
    return 0.138 * n / math.log(gamma * n) * math.sqrt(r_h ** 3 / mass)


# --------------------------------------------------------------------------
# a cluster advanced step by step
# --------------------------------------------------------------------------
STAT_NAMES = ("escaped", "degenerate", "cap_hits", "trials", "violations", "clamps",
              "angle_fails")


class Cluster:
    """One cluster's state (sorted SoA + potential), advanced by ``or_step``.

    ``pot_mode`` "recursion" follows Eqs. 2-5 literally; "dd" uses the
    double-double scan form of Eq. 1.
    """

    def __init__(self, r, vr, vt, m, ids, seed: int, *, theta_max: float = THETA_MAX,
                 gamma: float = GAMMA, bin_size: int = BIN_SIZE, max_trials: int = 1000,
                 energy_correction: bool = True, pot_mode: str = "recursion",
                 rng: str = "philox", radii=None, semi_major=None, x_bb: float = 1.0,
                 x_bs: float = 1.0):
        r, vr, vt, m = _f64(r), _f64(vr), _f64(vt), _f64(m)
        ids = _u32a(ids)
        n = r.shape[0]
        perm = sort_perm(r, ids)
        self.r = r[perm].copy()
        self.vr = vr[perm].copy()
        self.vt = vt[perm].copy()
        self.m = m[perm].copy()
        self.id = ids[perm].copy()
        # stellar radii (sticky-sphere collisions and the Eq. 8 timestep)
        self.R = None if radii is None else _f64(radii)[perm].copy()
        # binaries' semi-major axes (0: a single star) and Eqs. 9-10's X
        self.A = None if semi_major is None else _f64(semi_major)[perm].copy()
        self.x_bb, self.x_bs = float(x_bb), float(x_bs)
        # an outside bound on the next timesteps (e.g. Eq. 11's), 0: none
        self.dt_cap = 0.0
        # mergers so far and the energy they dissipated
        self.collisions = np.zeros(2)
        self.n = n
        self.nb = int(np.count_nonzero(np.isfinite(self.r)))
        self.seed = int(seed)
        self.step_no = 0
        self.bin_size = bin_size
        self.pref = t_rel_prefactor(theta_max)
        self.lnL = coulomb_log(n, gamma)
        self.max_trials = max_trials
        self.ecorr = 1 if energy_correction else 0
        self.pot_mode = {"recursion": 0, "dd": 1}[pot_mode]
        self.phi = np.zeros(n)
        self.phi[: self.nb] = potential(self.r[: self.nb], self.m[: self.nb],
                                        "dd" if self.pot_mode == 1 else "recursion")
        self.last_stats = None
        self.last_dt = None
        # mass and energy carried off by escapers (section 4.2's budget)
        self.escaped = np.zeros(2)
        # "taus113": one combined-Tausworthe stream per id (section 3.6)
        self.taus = None
        if rng == "taus113":
            self.taus = taus_streams(self.seed, int(self.id.max()) + 1 if n else 0)
        elif rng != "philox":
            raise ValueError("rng: philox or taus113")

    def step(self, nsteps: int = 1):
        for _ in range(nsteps):
            nb = np.array([self.nb], dtype=np.int64)
            stats = np.zeros(7, dtype=np.int64)
            if self.taus is not None:
                _L().or_taus_bind(_ptr(self.taus))
            try:
                if self.R is None and self.A is None and not self.dt_cap > 0.0:
                    dt = _L().or_step(self.n, _ptr(nb), _ptr(self.r), _ptr(self.vr),
                                      _ptr(self.vt), _ptr(self.m), _ptr(self.id),
                                      _ptr(self.phi), self.seed, self.step_no, self.bin_size,
                                      self.pref, self.lnL, self.max_trials, self.ecorr,
                                      self.pot_mode, _ptr(stats), _ptr(self.escaped))
                else:
                    opt = lambda a: None if a is None else _ptr(a)
                    dt = _L().or_step_col(self.n, _ptr(nb), _ptr(self.r), _ptr(self.vr),
                                          _ptr(self.vt), _ptr(self.m), opt(self.R),
                                          _ptr(self.id), _ptr(self.phi), self.seed,
                                          self.step_no, self.bin_size, self.pref, self.lnL,
                                          self.max_trials, self.ecorr, self.pot_mode,
                                          _ptr(stats), _ptr(self.escaped),
                                          _ptr(self.collisions), opt(self.A), self.x_bb,
                                          self.x_bs, float(self.dt_cap))
            finally:
                _L().or_taus_bind(None)
            self.nb = int(nb[0])
            self.step_no += 1
            self.last_dt = dt
            self.last_stats = dict(zip(STAT_NAMES, (int(x) for x in stats)))
        return self

    def energy(self):
        nb = self.nb
        return energy(self.r[:nb], self.vr[:nb], self.vt[:nb], self.m[:nb])

    def total_energy(self) -> float:
        """K + W of the bound stars plus the energy the escapers took."""
        return self.energy()[2] + self.escaped[1]

    def lagrange_radii(self, fracs):
        nb = self.nb
        return lagrange_radii(self.r[:nb], self.m[:nb], fracs)

    def core(self):
        nb = self.nb
        return core(self.r[:nb], self.m[:nb])
