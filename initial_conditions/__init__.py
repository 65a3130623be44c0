"""Seeded synthetic initial conditions: Plummer spheres in Henon units.

This module is the one input source shared by the CUDA path, the oracle, the
tests and the benchmark.  It holds none of the timestep method's arithmetic
(no potential, no orbit, no relaxation); it only draws stars.

Recipe (the paper evolves Plummer models, sections 4.1-4.3, sampled from the
distribution function f(E, J), section 2.1):

* units G = M = 1 with Plummer scale a = 3 pi / 16, so that the analytic
  total energy is -3 pi G M^2 / (64 a) = -1/4;
* radius from the enclosed-mass fraction X ~ U(0,1):
  r = a / sqrt(X^(-2/3) - 1) (no truncation);
* speed v = q v_esc(r), v_esc = sqrt(2) (1 + r^2/a^2)^(-1/4) sqrt(G M / a),
  with q drawn by von Neumann rejection from q^2 (1 - q^2)^(7/2) under the
  bound 0.1 (Aarseth, Henon & Wielen 1974);
* isotropic split: cos(theta) ~ U(-1, 1), v_r = v cos(theta),
  v_t = v sin(theta) >= 0;
* masses equal (1/N) or Salpeter dN/dm ~ m^-2.35 on [0.1, 100] by the
  inverse CDF, rescaled so that they sum to 1; masses are independent of
  position;
* ids 0..N-1 in draw order; the stars come out unsorted.

The random numbers come from numpy's Philox bit generator keyed by ``seed``.
"""
from __future__ import annotations

import math

import numpy as np

PLUMMER_A = 3.0 * math.pi / 16.0


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(stream)]))


def plummer(n: int, seed: int = 1, masses: str = "equal", a: float = PLUMMER_A):
    """Return dict(r, vr, vt, m, id) for an N-star Plummer sphere."""
    n = int(n)
    g = _rng(seed)
    # radii: resample the (probability ~0) draws that would give r = 0 or inf
    X = g.random(n)
    bad = (X <= 0.0) | (X >= 1.0)
    while bad.any():
        X[bad] = g.random(int(bad.sum()))
        bad = (X <= 0.0) | (X >= 1.0)
    r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    # speeds by rejection on q^2 (1 - q^2)^3.5 <= 0.1
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        qq = g.random(todo.size)
        yy = 0.1 * g.random(todo.size)
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    v = q * math.sqrt(2.0) * (1.0 + r * r / (a * a)) ** (-0.25) * math.sqrt(1.0 / a)
    ct = 2.0 * g.random(n) - 1.0
    vr = v * ct
    vt = v * np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    if masses == "equal":
        m = np.full(n, 1.0 / n)
    elif masses == "salpeter":
        m = salpeter_masses(n, seed)
    else:
        raise ValueError("masses must be 'equal' or 'salpeter'")
    return {"r": r, "vr": vr, "vt": vt, "m": m, "id": np.arange(n, dtype=np.uint32)}


def salpeter_masses(n: int, seed: int, alpha: float = 2.35, mlo: float = 0.1,
                    mhi: float = 100.0) -> np.ndarray:
    """dN/dm ~ m^-alpha on [mlo, mhi] by inverse CDF, rescaled to sum 1."""
    g = _rng(seed, 1)
    u = g.random(n)
    e = 1.0 - alpha
    lo, hi = mlo ** e, mhi ** e
    m = (lo + u * (hi - lo)) ** (1.0 / e)
    return m / m.sum()


def ensemble_sizes(n_clusters: int = 64, seed: int = 1, nmin: int = 10_000,
                   nmax: int = 200_000) -> np.ndarray:
    """Cluster sizes uniform in [nmin, nmax]: nmin + floor(U (nmax - nmin + 1))."""
    g = _rng(seed, 2)
    u = g.random(n_clusters)
    return (nmin + np.floor(u * (nmax - nmin + 1))).astype(np.int64)


def ensemble(n_clusters: int = 64, seed: int = 1, sizes=None, masses: str = "equal"):
    """Concatenated SoA of independent Plummer clusters; cluster c uses seed
    1000 + c.  Returns (dict of arrays, sizes, seeds)."""
    if sizes is None:
        sizes = ensemble_sizes(n_clusters, seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    seeds = np.array([1000 + c for c in range(len(sizes))], dtype=np.uint64)
    parts = [plummer(int(nc), int(sc), masses) for nc, sc in zip(sizes, seeds)]
    cat = {k: np.concatenate([p[k] for p in parts]) for k in ("r", "vr", "vt", "m", "id")}
    return cat, sizes, seeds


def quantile_plummer(n: int, a: float = PLUMMER_A) -> np.ndarray:
    """Deterministic radii at enclosed-mass fractions (k + 1/2)/N, sorted."""
    X = (np.arange(n) + 0.5) / n
    return a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
