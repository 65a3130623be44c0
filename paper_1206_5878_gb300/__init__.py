"""GB300 hot path of the Henon Monte Carlo method (Pattabiraman et al.).

Python face of libcmc.so.  ``Cluster`` wraps a context (cmc_init /
cmc_step / cmc_energy / cmc_lagrange_radii ...); the ``stage_*`` functions
wrap the single-step entry points on torch CUDA tensors.  PyTorch only
provides device memory and streams; every step runs in the library's
kernels.  The binding raises if the library has not been built.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import CMCError, STAT_NAMES, cmc_config, check, load

__all__ = ["Cluster", "CMCError", "config", "load", "STAT_NAMES", "stage_philox",
           "stage_sort_radius", "stage_potential", "stage_timestep", "stage_relax",
           "stage_orbit", "stage_energy_correction", "tse"]


def config(**kw) -> cmc_config:
    """cmc_config with the library defaults, overridden by keyword."""
    cfg = cmc_config()
    load().cmc_config_default(ctypes.byref(cfg))
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def _ptr(a):
    """Address of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


class Cluster:
    """One or more clusters advanced together by the CUDA library.

    state: dict with r, vr, vt, m (float64) and id (uint32) arrays, either
    numpy (host) or torch CUDA tensors (device), clusters concatenated.
    sizes: stars per cluster (default: one cluster); seeds: one per cluster.
    """

    def __init__(self, state, seeds, sizes=None, stream=None, debug=False, **cfg):
        """cfg: cmc_config fields by name; rng may also be given as
        "philox" (0) or "taus113" (1)."""
        self.lib = load(debug)  # debug: the build with device-side index checks
        if isinstance(cfg.get("rng"), str):
            cfg["rng"] = {"philox": 0, "taus113": 1}[cfg["rng"]]
        r = state["r"]
        n = int(r.shape[0])
        sizes = [n] if sizes is None else [int(s) for s in sizes]
        seeds = [int(s) for s in np.atleast_1d(seeds)]
        if sum(sizes) != n or len(seeds) != len(sizes):
            raise ValueError("sizes must sum to the number of stars, one seed per cluster")
        self.n = n
        self.sizes = sizes
        self.n_clusters = len(sizes)
        self.cfg = config(**cfg)
        self.stream = _stream_ptr(stream)
        kind = 0 if isinstance(r, np.ndarray) else 1
        arrs = [self._prep(state[k], k, kind) for k in ("r", "vr", "vt", "m", "id")]
        self._sizes = np.asarray(sizes, dtype=np.int64)
        self._seeds = np.asarray(seeds, dtype=np.uint64)
        ctx = ctypes.c_void_p()
        st = self.lib.cmc_init(ctypes.byref(ctx), ctypes.byref(self.cfg), self.n_clusters,
                               self._sizes.ctypes.data, self._seeds.ctypes.data,
                               *[_ptr(a) for a in arrs], kind, self.stream)
        check(st, None, self.lib)
        self.ctx = ctx

    @staticmethod
    def _prep(a, name, kind):
        if kind == 0:
            return np.ascontiguousarray(a, dtype=np.uint32 if name == "id" else np.float64)
        import torch
        want = torch.int32 if name == "id" else torch.float64
        if name == "id" and a.dtype in (torch.int32, torch.uint32):
            return a.contiguous()
        return a.to(want).contiguous()

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.cmc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- API ---------------------------------------------------------------
    def step(self, n_steps: int = 1):
        check(self.lib.cmc_step(self.ctx, int(n_steps)), self.ctx, self.lib)
        return self

    def step_profiled(self, n_steps: int = 1) -> dict:
        """Like step(); returns the summed device milliseconds per stage."""
        ms = np.zeros(len(_native.STAGE_NAMES))
        check(self.lib.cmc_step_profiled(self.ctx, int(n_steps), ms.ctypes.data), self.ctx, self.lib)
        return dict(zip(_native.STAGE_NAMES, (float(v) for v in ms)))

    def energy(self) -> np.ndarray:
        out = np.zeros((self.n_clusters, 3))
        check(self.lib.cmc_energy(self.ctx, out.ctypes.data), self.ctx, self.lib)
        return out

    def lagrange_radii(self, fracs) -> np.ndarray:
        fr = np.ascontiguousarray(fracs, dtype=np.float64)
        out = np.zeros((self.n_clusters, fr.shape[0]))
        check(self.lib.cmc_lagrange_radii(self.ctx, fr.ctypes.data, fr.shape[0],
                                          out.ctypes.data), self.ctx, self.lib)
        return out

    def rng_state(self) -> np.ndarray:
        """The Tausworthe stream states (4 words per slot), rng = taus113 only."""
        nw = np.zeros(1, dtype=np.int64)
        check(self.lib.cmc_get_rng_state(self.ctx, None, nw.ctypes.data), self.ctx, self.lib)
        out = np.zeros(int(nw[0]), dtype=np.uint32)
        check(self.lib.cmc_get_rng_state(self.ctx, out.ctypes.data, nw.ctypes.data), self.ctx, self.lib)
        return out

    def set_rng_state(self, words):
        words = np.ascontiguousarray(words, dtype=np.uint32)
        check(self.lib.cmc_set_rng_state(self.ctx, words.ctypes.data, words.shape[0]), self.ctx, self.lib)

    def core(self) -> np.ndarray:
        """Per cluster {rho_c, r_c, number of estimates} (Eq. 19)."""
        out = np.zeros((self.n_clusters, 3))
        check(self.lib.cmc_core(self.ctx, out.ctypes.data), self.ctx, self.lib)
        return out

    def get_state(self, out=None):
        """Sorted state as numpy arrays (or into the given torch tensors)."""
        step = np.zeros(1, dtype=np.int64)
        if out is None:
            out = {k: np.empty(self.n) for k in ("r", "vr", "vt", "m", "phi")}
            out["id"] = np.empty(self.n, dtype=np.uint32)
            kind = 0
        else:
            kind = 0 if isinstance(out["r"], np.ndarray) else 1
        check(self.lib.cmc_get_state(self.ctx, _ptr(out.get("r")), _ptr(out.get("vr")),
                                     _ptr(out.get("vt")), _ptr(out.get("m")),
                                     _ptr(out.get("id")), _ptr(out.get("phi")),
                                     step.ctypes.data, kind), self.ctx, self.lib)
        out["step"] = int(step[0])
        return out

    def set_radii(self, R):
        """Stellar radii of the stars in get_state order (collisions=1)."""
        R = np.ascontiguousarray(R, dtype=np.float64)
        check(self.lib.cmc_set_radii(self.ctx, R.ctypes.data, 0), self.ctx, self.lib)

    def radii(self) -> np.ndarray:
        out = np.empty(self.n)
        check(self.lib.cmc_get_radii(self.ctx, out.ctypes.data, 0), self.ctx, self.lib)
        return out

    def set_binaries(self, a):
        """Semi-major axes of the stars in get_state order (binaries=1; 0 for
        a single star): the binary timesteps of Eqs. 9 and 10 then bound
        the step."""
        a = np.ascontiguousarray(a, dtype=np.float64)
        check(self.lib.cmc_set_binaries(self.ctx, a.ctypes.data, 0), self.ctx, self.lib)

    def binaries(self) -> np.ndarray:
        out = np.empty(self.n)
        check(self.lib.cmc_get_binaries(self.ctx, out.ctypes.data, 0), self.ctx, self.lib)
        return out

    def set_dt_cap(self, cap):
        """An outside bound on each cluster's next timesteps (0 = none):
        Eq. 11's stellar-evolution step (tse), say."""
        cap = np.ascontiguousarray(np.broadcast_to(np.asarray(cap, dtype=np.float64),
                                                   (self.n_clusters,)))
        check(self.lib.cmc_set_dt_cap(self.ctx, cap.ctypes.data), self.ctx, self.lib)

    def set_state(self, state, step: int):
        kind = 0 if isinstance(state["r"], np.ndarray) else 1
        arrs = [self._prep(state[k], k, kind) for k in ("r", "vr", "vt", "m", "id")]
        check(self.lib.cmc_set_state(self.ctx, *[_ptr(a) for a in arrs], int(step), kind),
              self.ctx, self.lib)

    def nbound(self) -> np.ndarray:
        out = np.zeros(self.n_clusters, dtype=np.int64)
        check(self.lib.cmc_get_nbound(self.ctx, out.ctypes.data), self.ctx, self.lib)
        return out

    def dt(self) -> np.ndarray:
        out = np.zeros(self.n_clusters)
        check(self.lib.cmc_get_dt(self.ctx, out.ctypes.data), self.ctx, self.lib)
        return out

    def stats(self) -> list:
        out = np.zeros((self.n_clusters, _native.CMC_NSTATS), dtype=np.int64)
        check(self.lib.cmc_get_stats(self.ctx, out.ctypes.data), self.ctx, self.lib)
        return [dict(zip(STAT_NAMES, (int(v) for v in row))) for row in out]

    def escaped(self) -> np.ndarray:
        """(n_clusters, 2): mass and energy carried off by escapers; the
        conserved total is energy()[:, 2] + escaped()[:, 1]."""
        out = np.zeros((self.n_clusters, 2))
        check(self.lib.cmc_get_escaped(self.ctx, out.ctypes.data), self.ctx, self.lib)
        return out

    def diagnostics(self) -> np.ndarray:
        """(n_clusters, records, len(DIAG_FIELDS)): the per-step diagnostics
        ring (config diag_ring > 0), oldest record first."""
        nrec = ctypes.c_int32(0)
        check(self.lib.cmc_get_diagnostics(self.ctx, None, ctypes.byref(nrec)), self.ctx, self.lib)
        cap = self.cfg.diag_ring
        out = np.zeros((self.n_clusters, cap, len(_native.DIAG_FIELDS)))
        check(self.lib.cmc_get_diagnostics(self.ctx, out.ctypes.data, ctypes.byref(nrec)),
              self.ctx, self.lib)
        return out[:, : nrec.value]

    def set_escaped(self, budget):
        b = np.ascontiguousarray(budget, dtype=np.float64).reshape(self.n_clusters, 2)
        check(self.lib.cmc_set_escaped(self.ctx, b.ctypes.data), self.ctx, self.lib)

    def total_energy(self) -> np.ndarray:
        """K + W of the bound stars plus the energy the escapers took."""
        return self.energy()[:, 2] + self.escaped()[:, 1]

    def kernels_per_step(self) -> int:
        return int(self.lib.cmc_kernels_per_step(self.ctx))

    def tuning(self) -> dict:
        """Kernel shapes in use: orbit block size, sort keys per thread,
        multisplit (match or ballot), the mixed-mode orbit variant and the
        relaxation variant."""
        out = np.zeros(5, dtype=np.int32)
        check(self.lib.cmc_get_tuning(self.ctx, out.ctypes.data), self.ctx, self.lib)
        return {"orbit_block": int(out[0]), "sort_keys_per_thread": int(out[1]),
                "sort_multisplit": "ballot" if out[2] else "match",
                "orbit_variant": int(out[3]), "relax_variant": int(out[4])}

    def set_stream(self, stream):
        self.stream = _stream_ptr(stream)
        check(self.lib.cmc_set_stream(self.ctx, self.stream), self.ctx, self.lib)


# --------------------------------------------------------------- stages
# Single-cluster entry points on torch CUDA tensors (sorted inputs).
def _t(a):
    return _ptr(a)


def stage_philox(ctr, seed: int, stream=None):
    import torch
    out = torch.empty_like(ctr)
    check(load().cmc_rng_philox(ctr.shape[0], _t(ctr), int(seed), _t(out),
                                _stream_ptr(stream)))
    return out


def stage_sort_radius(r, ids, stream=None):
    import torch
    perm = torch.empty(r.shape[0], dtype=torch.int32, device=r.device)
    check(load().cmc_sort_radius(r.shape[0], _t(r), _t(ids), _t(perm), _stream_ptr(stream)))
    return perm


def stage_potential(r, m, want_M: bool = False, stream=None):
    import torch
    phi = torch.empty_like(r)
    M = torch.empty_like(r) if want_M else None
    check(load().cmc_potential(r.shape[0], _t(r), _t(m), _t(phi), _t(M), _stream_ptr(stream)))
    return (phi, M) if want_M else phi


def stage_timestep(r, vr, vt, m, lnL: float, bin_size: int = 20, theta_max: float = None,
                   stream=None):
    import math

    import torch
    if theta_max is None:
        theta_max = math.pi / 2
    n = r.shape[0]
    nbin = torch.zeros(max(1, (n + bin_size - 1) // bin_size), dtype=torch.float64,
                       device=r.device)
    dt = torch.zeros(1, dtype=torch.float64, device=r.device)
    check(load().cmc_timestep(n, _t(r), _t(vr), _t(vt), _t(m), bin_size, theta_max, lnL,
                              _t(nbin), _t(dt), _stream_ptr(stream)))
    return dt, nbin[: (n + bin_size - 1) // bin_size]


def stage_relax(vr, vt, m, ids, nbin, dt: float, lnL: float, seed: int, step: int,
                bin_size: int = 20, stream=None):
    vr = vr.clone()
    vt = vt.clone()
    check(load().cmc_relax(vr.shape[0], _t(vr), _t(vt), _t(m), _t(ids), _t(nbin), bin_size,
                           float(dt), float(lnL), int(seed), int(step), _stream_ptr(stream)))
    return vr, vt


def stage_orbit(r, phi, vr, vt, ids, seed: int, step: int, max_trials: int = 1000,
                precision: int = 0, stream=None):
    import torch
    n = r.shape[0]
    f = lambda: torch.empty(n, dtype=torch.float64, device=r.device)
    out = {k: f() for k in ("r_new", "vr", "vt", "phi_new", "rmin", "rmax", "F")}
    out["code"] = torch.empty(n, dtype=torch.int32, device=r.device)
    check(load().cmc_orbit(n, _t(r), _t(phi), _t(vr), _t(vt), _t(ids), int(seed), int(step),
                           int(max_trials), int(precision), _t(out["r_new"]), _t(out["vr"]),
                           _t(out["vt"]), _t(out["phi_new"]), _t(out["rmin"]),
                           _t(out["rmax"]), _t(out["F"]), _t(out["code"]),
                           _stream_ptr(stream)))
    return out


def stage_energy_correction(r, phi, vr, vt, r_old, c, stream=None):
    vr = vr.clone()
    vt = vt.clone()
    check(load().cmc_energy_correction(r.shape[0], _t(r), _t(phi), _t(vr), _t(vt), _t(r_old),
                                       _t(c), _stream_ptr(stream)))
    return vr, vt


def tse(M: float, T_prev: float, dm_se: float) -> float:
    """The stellar-evolution timestep of Eq. 11 (+inf without mass loss)."""
    return float(load().cmc_tse(float(M), float(T_prev), float(dm_se)))


def set_wait_limits(lookback_polls: int = 0, tie_moves: int = 0):
    """Limits of the sort's bounded device waits on the current device
    (cmc_set_wait_limits; 0 restores the defaults)."""
    check(load().cmc_set_wait_limits(int(lookback_polls), int(tie_moves)))


def check_arith(op: int, n: int, seed: int = 1) -> int:
    """Mismatches between the kernels' integer-pipe FP64 operation `op`
    (0 product, 1 quotient, 2 square root) and the FP64 hardware one over
    n hashed operand pairs (cmc_check_arith)."""
    import numpy as np
    out = np.zeros(1, dtype=np.uint64)
    check(load().cmc_check_arith(int(op), int(n), int(seed), out.ctypes.data))
    return int(out[0])

