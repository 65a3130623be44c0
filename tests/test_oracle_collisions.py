"""Pins of the oracle's stellar collisions (section 2.1 step 2, Eq. 8, and
step 3(iii), sticky spheres): the collision timestep on a construction with
known density, dispersion and radii; the merger's conservation laws; the
collision probability's geometric and gravitational-focusing limits and its
frequency; the cube root the merged radius needs; and a few whole timesteps
whose energy budget closes."""
import math

import numpy as np
import pytest
import scipy.stats as sst

import initial_conditions as ic

EPS = np.finfo(float).eps


def test_cube_root():
    import oracle
    for k in range(-60, 61, 7):
        assert oracle.cbrt(2.0 ** (3 * k)) == 2.0 ** k  # exact cubes
    assert oracle.cbrt(27.0) == 3.0 and oracle.cbrt(0.125) == 0.5
    g = np.random.default_rng(1)
    for v in 10.0 ** g.uniform(-40, 40, 2000):
        y = oracle.cbrt(v)
        assert abs(y / np.cbrt(v) - 1) < 4 * EPS  # numpy's cbrt: within an ulp
        assert abs(y ** 3 / v - 1) < 8 * EPS
    assert oracle.cbrt(0.0) == 0.0


def _uniform_core(P=300, rmax=0.02, a=0.3, b=0.4, R0=1e-4, m0=1e-5, extra=0):
    """P stars filling a sphere of radius rmax at equal volume steps (the
    estimator's n = 3 (P - 1) / (4 pi rmax^3) exactly), equal speeds, radii
    and masses; `extra` more stars outside."""
    r = rmax * (np.arange(P) / (P - 1)) ** (1 / 3)
    r[0] = 0.0
    r = np.concatenate([r, rmax * (1 + np.arange(1, extra + 1) / 10.0)])
    n = P + extra
    return (r, np.full(n, a), np.full(n, b), np.full(n, m0), np.full(n, R0))


def test_collision_timestep_closed_form():
    import oracle
    r, vr, vt, m, R = _uniform_core()
    T = oracle.tcoll(r, vr, vt, m, R)
    n = 3 * 299 / (4 * math.pi * 0.02 ** 3)
    sig2 = (0.3 ** 2 + 0.4 ** 2) / 3
    inv = 16 * math.sqrt(math.pi) * n * 1e-8 * math.sqrt(sig2) * (1 + 1e-9 / (2 * sig2 * 1e-8))
    assert abs(T * inv - 1) < 1e-13
    # only the innermost 300 count; no radii, no timestep
    r2, vr2, vt2, m2, R2 = _uniform_core(extra=50)
    R2[300:] = 1.0
    assert oracle.tcoll(r2, vr2, vt2, m2, R2) == T
    assert oracle.tcoll(r, vr, vt, m, np.zeros_like(R)) == math.inf
    # scalings: 1/T ~ <R^2> when focusing is negligible, ~ <M R> sigma^-1 when
    # it dominates
    Tl = oracle.tcoll(r, vr, vt, m * 1e-6, R)
    T4 = oracle.tcoll(r, vr, vt, m * 1e-6, 2 * R)
    assert abs(T4 / Tl - 0.25) < 1e-5
    big = oracle.tcoll(r, vr * 1e-3, vt * 1e-3, m * 1e6, R)
    big2 = oracle.tcoll(r, vr * 1e-3, vt * 1e-3, m * 2e6, R)
    assert abs(big / big2 - 2) < 1e-3


def _enc(R1, R2, **kw):
    import oracle
    p = dict(m1=0.3, m2=0.7, vr1=0.8, vt1=0.2, vr2=-0.5, vt2=0.6, n=50.0, dt=1e-3, lnL=9.0,
             seed=3, ident=11, step=4)
    p.update(kw)
    return oracle.encounter_radii(p["m1"], p["m2"], p["vr1"], p["vt1"], p["vr2"], p["vt2"],
                                  R1, R2, p["n"], p["dt"], p["lnL"], p["seed"], p["ident"],
                                  p["step"]), p


def test_no_radii_is_the_plain_encounter():
    import oracle
    o, p = _enc(0.0, 0.0)
    plain = oracle.encounter(p["m1"], p["m2"], p["vr1"], p["vt1"], p["vr2"], p["vt2"], p["n"],
                             p["dt"], p["lnL"], p["seed"], p["ident"], p["step"])
    np.testing.assert_array_equal(o[6:9], plain["v1p"])
    np.testing.assert_array_equal(o[9:12], plain["v2p"])
    assert o[12] == plain["s2"] and o[15] == plain["status"] == 0 and o[16] == 0.0


@pytest.mark.parametrize("ident", range(8))
def test_merger_conserves_mass_momentum_and_dissipates_the_relative_energy(ident):
    o, p = _enc(10.0, 10.0, ident=ident)
    assert o[15] == 2.0 and o[16] >= 1.0  # certain collision
    m1, m2 = p["m1"], p["m2"]
    v1, v2 = o[0:3], o[3:6]  # the 3-D velocities before (with the azimuth psi)
    vc = o[6:9]
    np.testing.assert_allclose(vc * (m1 + m2), m1 * v1 + m2 * v2, rtol=0, atol=8 * EPS)
    assert vc[0] * (m1 + m2) == pytest.approx(m1 * p["vr1"] + m2 * p["vr2"], abs=4 * EPS)
    k_before = 0.5 * m1 * np.dot(v1, v1) + 0.5 * m2 * np.dot(v2, v2)
    k_after = 0.5 * (m1 + m2) * np.dot(vc, vc)
    assert abs((k_before - k_after) - o[17]) < 16 * EPS * k_before
    assert o[17] > 0


def test_collision_probability_limits():
    # geometric limit (fast pairs, tiny masses): P = n pi (R1 + R2)^2 |w| dt
    o, p = _enc(1e-3, 2e-3, m1=1e-12, m2=1e-12)
    w = o[14]
    assert abs(o[16] / (p["n"] * math.pi * 9e-6 * w * p["dt"]) - 1) < 1e-9
    # gravitational focusing dominates for slow heavy pairs: P grows as 1/|w|
    a, _ = _enc(1e-6, 1e-6, vr1=1e-3, vr2=-1e-3, vt1=0, vt2=0, m1=0.5, m2=0.5)
    b, _ = _enc(1e-6, 1e-6, vr1=2e-3, vr2=-2e-3, vt1=0, vt2=0, m1=0.5, m2=0.5)
    assert abs(a[16] / b[16] - 2) < 1e-5
    # linear in dt and n
    c, _ = _enc(1e-3, 2e-3, dt=2e-3)
    d, _ = _enc(1e-3, 2e-3, n=100.0)
    e, _ = _enc(1e-3, 2e-3)
    assert abs(c[16] / e[16] - 2) < 1e-14 and abs(d[16] / e[16] - 2) < 1e-14


def test_collision_frequency():
    # one draw per pair: over many pairs the fraction that merge is P
    hits, P = 0, None
    trials = 20000
    for i in range(trials):
        o, _ = _enc(0.03, 0.03, ident=1000 + i, dt=1e-2)
        P = o[16]
        hits += o[15] == 2.0
    assert 0.05 < P < 0.5
    assert sst.binomtest(hits, trials, P).pvalue > 1e-4


def test_relax_with_radii_merges_and_keeps_mass():
    import oracle
    n = 2000
    d = ic.plummer(n, seed=4)
    p = np.lexsort((d["id"], d["r"]))
    s = {k: v[p] for k, v in d.items()}
    R = np.full(n, 2e-3)
    lnL = oracle.coulomb_log(n)
    dt, nbin = oracle.timestep(s["r"], s["vr"], s["vt"], s["m"], lnL)
    phi = oracle.potential(s["r"], s["m"], "dd")
    vr, vt, m, R2, merged, e_col = oracle.relax_radii(s["vr"], s["vt"], s["m"], R, s["id"],
                                                      nbin, dt, lnL, 4, 0, s["r"], phi)
    assert merged > 0
    # what the mergers book is the change of K + W: the energies before and
    # after by brute force (the relaxed pairs keep their energy; a merged
    # star's kinetic energy is that of its radial and transverse speed)
    W0 = oracle.energy_W_brute(s["r"], s["m"])
    W1 = oracle.energy_W_brute(s["r"], m)
    K0 = 0.5 * np.sum(s["m"] * (s["vr"] ** 2 + s["vt"] ** 2))
    K1 = 0.5 * np.sum(m * (vr ** 2 + vt ** 2))
    # (the brute-force sums of N^2 / 2 terms round at ~N eps of |W|)
    assert abs((K1 + W1) - (K0 + W0) - e_col) < 1e-11 * abs(K0 + W0)
    assert abs(m.sum() - s["m"].sum()) < 4 * EPS
    gone = np.flatnonzero(R2 < 0)
    assert len(gone) == merged and np.all(m[gone] == 0.0) and np.all(gone % 2 == 1)
    first = gone - 1
    assert np.all(m[first] == s["m"][first] + s["m"][gone])
    np.testing.assert_allclose(R2[first] ** 3, R[first] ** 3 + R[gone] ** 3, rtol=8 * EPS)
    # radial momentum of every merged pair is kept
    np.testing.assert_allclose(m[first] * vr[first],
                               s["m"][first] * s["vr"][first] + s["m"][gone] * s["vr"][gone],
                               rtol=0, atol=8 * EPS)


def test_steps_with_collisions_close_the_energy_budget():
    """Ten timesteps of N = 5000 with radii that make about one star in a
    hundred merge: merged-away stars leave (mass 0, no energy carried off),
    the mass is conserved, and K + W + E_esc less what the mergers changed of
    K + W stays within the paper's bound.  (New orbits in a step with mergers
    are drawn in the potential from before them, as the potential is
    computed once per step; the energy correction absorbs most of that, and
    what remains was measured at 2e-6 of |E| per merger.)"""
    import oracle
    n = 5000
    d = ic.plummer(n, seed=6)
    R = np.full(n, 2e-5)
    o = oracle.Cluster(d["r"], d["vr"], d["vt"], d["m"], d["id"], seed=6, radii=R)
    E0 = o.total_energy()
    M0 = o.m.sum()
    o.step(10)
    assert o.collisions[0] > 0
    assert abs(o.m[: o.nb].sum() + o.escaped[0] - M0) < 1e-12
    assert np.all(o.R[o.nb:] < 0) or np.all(np.isinf(o.r[o.nb:]))
    budget = o.total_energy() - o.collisions[1]
    assert abs(budget / E0 - 1) < 4e-4
    assert abs(budget / E0 - 1) < 5e-6 * o.collisions[0]
    # the collision timestep took part: it can only shorten the step
    plain = oracle.Cluster(d["r"], d["vr"], d["vt"], d["m"], d["id"], seed=6)
    plain.step(1)
    o2 = oracle.Cluster(d["r"], d["vr"], d["vt"], d["m"], d["id"], seed=6, radii=R)
    o2.step(1)
    assert o2.last_dt <= plain.last_dt
