"""Pins of the oracle's binary and stellar-evolution timesteps (section 2.1
step 2, Eqs. 9-11): the binary-binary and binary-single timesteps on a
construction with known central density, dispersion, binary fraction and
semi-major axes; their geometric and gravitational-focusing scalings; the
innermost-300 rule and the cases without binaries or single stars; Eq. 11's
mass-loss bound; and a timestep that the binaries or an outside bound
shorten."""
import math

import numpy as np
import pytest

import initial_conditions as ic


def _core(P=300, rmax=0.02, a=0.3, b=0.4, m0=1e-5, a0=1e-3, every=3, extra=0):
    """P stars filling a sphere of radius rmax at equal volume steps (the
    estimator's n = 3 (P - 1) / (4 pi rmax^3) exactly), equal speeds and
    masses; every `every`-th star a binary of semi-major axis a0; `extra`
    more single stars outside."""
    r = rmax * (np.arange(P) / (P - 1)) ** (1 / 3)
    r[0] = 0.0
    r = np.concatenate([r, rmax * (1 + np.arange(1, extra + 1) / 10.0)])
    n = P + extra
    A = np.zeros(n)
    A[:P:every] = a0
    return r, np.full(n, a), np.full(n, b), np.full(n, m0), A


def test_binary_timesteps_closed_form():
    import oracle
    r, vr, vt, m, A = _core()
    tbb, tbs = oracle.tbinary(r, vr, vt, m, A, 1.0, 1.0)
    P, nbin = 300, 100
    n = 3 * (P - 1) / (4 * math.pi * 0.02 ** 3)
    nb, ns = n * nbin / P, n * (P - nbin) / P
    sig2 = (0.3 ** 2 + 0.4 ** 2) / 3
    sig = math.sqrt(sig2)
    a2, ma, am, mm = 1e-6, 1e-5 * 1e-3, 1e-3, 1e-5
    inv_bb = 16 * math.sqrt(math.pi) * nb * a2 * sig * (1 + ma / (2 * sig2 * a2))
    inv_bs = 4 * math.sqrt(math.pi) * ns * a2 * sig * (1 + mm * am / (sig2 * a2))
    assert abs(tbb * inv_bb - 1) < 1e-13
    assert abs(tbs * inv_bs - 1) < 1e-13
    # the strong-interaction parameters enter squared (geometric) ...
    tbb2, tbs2 = oracle.tbinary(r, vr, vt, m * 1e-9, A, 2.0, 2.0)
    tbb1, tbs1 = oracle.tbinary(r, vr, vt, m * 1e-9, A, 1.0, 1.0)
    assert abs(tbb2 / tbb1 - 0.25) < 1e-6 and abs(tbs2 / tbs1 - 0.25) < 1e-6
    # ... and so does the semi-major axis; focusing-dominated, 1/T grows as M a
    tbb3, tbs3 = oracle.tbinary(r, vr, vt, m * 1e-9, A * 2, 1.0, 1.0)
    assert abs(tbb3 / tbb1 - 0.25) < 1e-6 and abs(tbs3 / tbs1 - 0.25) < 1e-6
    slow = (vr * 1e-3, vt * 1e-3)
    f1 = oracle.tbinary(r, *slow, m * 1e3, A, 1.0, 1.0)
    f2 = oracle.tbinary(r, *slow, m * 2e3, A, 1.0, 1.0)
    assert abs(f1[0] / f2[0] - 2) < 1e-3 and abs(f1[1] / f2[1] - 2) < 1e-3


def test_binary_timesteps_cases():
    import oracle
    r, vr, vt, m, A = _core()
    base = oracle.tbinary(r, vr, vt, m, A)
    # only the innermost 300 count: binaries further out change nothing
    r2, vr2, vt2, m2, A2 = _core(extra=40)
    A2[300:] = 5.0
    assert oracle.tbinary(r2, vr2, vt2, m2, A2) == base
    # no binary: no binary timestep; no single star: no binary-single one
    assert oracle.tbinary(r, vr, vt, m, np.zeros_like(A)) == (math.inf, math.inf)
    tbb, tbs = oracle.tbinary(r, vr, vt, m, np.full_like(A, 1e-3))
    assert math.isfinite(tbb) and tbs == math.inf
    # more binaries, more binary-binary encounters: twice the binaries, twice
    # the rate (geometric limit, the same <a^2>)
    half = oracle.tbinary(r, vr, vt, m * 1e-9, A, 1.0, 1.0)
    _, _, _, _, A6 = _core(every=6)
    sixth = oracle.tbinary(r, vr, vt, m * 1e-9, A6, 1.0, 1.0)
    assert abs(sixth[0] / half[0] - 2) < 1e-6


def test_stellar_evolution_timestep():
    import oracle
    M, T, dm = 0.83, 0.02, 3e-5
    t = oracle.tse(M, T, dm)
    # in T_se, losing mass at the last step's rate takes 0.1% of M
    assert abs((dm / T) * t / (0.001 * M) - 1) < 1e-15
    assert oracle.tse(M, T, 0.0) == math.inf and oracle.tse(M, T, -1.0) == math.inf


def test_step_takes_the_binary_and_outside_bounds():
    import oracle
    n = 4000
    d = ic.plummer(n, seed=2)
    plain = oracle.Cluster(d["r"], d["vr"], d["vt"], d["m"], d["id"], seed=2)
    plain.step(1)
    # wide binaries make the binary-single timestep the shortest
    A = np.where(np.arange(n) % 4 == 0, 0.05, 0.0)
    o = oracle.Cluster(d["r"], d["vr"], d["vt"], d["m"], d["id"], seed=2, semi_major=A)
    nb = o.nb
    tbb, tbs = oracle.tbinary(o.r[:nb], o.vr[:nb], o.vt[:nb], o.m[:nb], o.A[:nb])
    assert min(tbb, tbs) < plain.last_dt
    o.step(1)
    assert o.last_dt == min(tbb, tbs)
    # the semi-major axes travel with their stars
    assert sorted(o.A[o.A > 0].tolist()) == [0.05] * int((A > 0).sum())
    # an outside bound (Eq. 11's step, say) shorter than every other
    c = oracle.Cluster(d["r"], d["vr"], d["vt"], d["m"], d["id"], seed=2)
    c.dt_cap = oracle.tse(1.0, plain.last_dt, 0.5)
    c.step(1)
    assert c.last_dt == c.dt_cap < plain.last_dt
