"""Binaries and outside timestep bounds on the GPU: the binary-binary and
binary-single timesteps of Eqs. 9 and 10 (configuration binaries = 1) and a
per-cluster cap on the step (Eq. 11's stellar-evolution step, say), section
2.1 step 2, against the oracle.

Before each step the oracle takes the GPU's state, potential and semi-major
axes (as in test_gpu_parity_steps.py); the timestep must then be the
oracle's bit for bit, the new radii too, and the semi-major axes must have
travelled with their stars through the sort."""
import numpy as np
import pytest

import initial_conditions as ic
from test_gpu_parity_steps import _oracle_from
from test_gpu_step import _compare_states

pytestmark = pytest.mark.gpu


def _axes(d, every, a0):
    """Every `every`-th star (by id) a binary of semi-major axis a0 (times a
    spread of 1..2, so that <a^2>, <a> and <M a> are not trivial)."""
    n = len(d["id"])
    A = np.zeros(n)
    k = np.arange(0, n, every)
    A[k] = a0 * (1.0 + (k % 7) / 6.0)
    return A


def _cluster(g, d, seed, A=None, R=None, **cfg):
    extra = {}
    if A is not None:
        extra["binaries"] = 1
    if R is not None:
        extra["collisions"] = 1
    c = g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [seed], **extra, **cfg)
    # per-star attributes belong to the sorted order the context keeps:
    # map them by id
    ids = c.get_state()["id"]
    for vals, setter in ((A, c.set_binaries if A is not None else None),
                         (R, c.set_radii if R is not None else None)):
        if vals is None:
            continue
        byid = np.empty(len(d["id"]))
        byid[d["id"]] = vals
        setter(byid[ids])
    return c


def _orc(orc, c, seed, x_bb=1.0, x_bs=1.0):
    st = c.get_state()
    o = _oracle_from(orc, st, seed, st["step"], c.escaped()[0])
    if c.cfg.binaries:
        o.A = c.binaries().copy()
        o.x_bb, o.x_bs = x_bb, x_bs
    if c.cfg.collisions:
        o.R = c.radii().copy()
    return o


def _binary_dt(orc, o):
    nb = o.nb
    return orc.tbinary(o.r[:nb], o.vr[:nb], o.vt[:nb], o.m[:nb], o.A[:nb], o.x_bb, o.x_bs)


@pytest.mark.parametrize("n,every,a0,x,dominates", [
    (5000, 4, 0.02, (1.0, 1.0), True),      # wide binaries: Eqs. 9-10 set the step
    (20_011, 3, 1e-5, (1.0, 1.0), False),   # tight ones: Eq. 7 does
    (7001, 2, 3e-3, (2.0, 0.5), None),      # other strong-interaction parameters
])
def test_fp64_steps_with_binaries_match_oracle(g_stage, orc, n, every, a0, x, dominates):
    g = g_stage
    d = ic.plummer(n, seed=n)
    A = _axes(d, every, a0)
    c = _cluster(g, d, 3, A=A, precision=0, x_bb=x[0], x_bs=x[1])
    took = []
    for step in range(4):
        o = _orc(orc, c, 3, *x)
        tbb, tbs = _binary_dt(orc, o)
        c.step(1)
        o.step(1)
        after = c.get_state()
        np.testing.assert_array_equal(after["id"], o.id)
        np.testing.assert_array_equal(after["r"], o.r)  # new radii bit for bit
        _compare_states(after, o)
        assert c.dt()[0] == o.last_dt  # Eqs. 9 and 10 joined Eq. 7, bit for bit
        np.testing.assert_array_equal(c.binaries(), o.A)  # axes moved with the stars
        took.append(o.last_dt == min(tbb, tbs))
    # the axes are still those set, star by star
    byid = np.empty(n)
    byid[after["id"]] = c.binaries()
    np.testing.assert_array_equal(byid[d["id"]], A)
    if dominates is not None:
        assert all(took) if dominates else not any(took)


def test_mixed_mode_takes_the_same_timestep(g_stage, orc):
    """Mixed mode draws its orbits with its own envelope, but the timestep
    is FP64 in both modes: the same dt, the axes still with their stars."""
    g = g_stage
    n = 8000
    d = ic.plummer(n, seed=2)
    A = _axes(d, 4, 0.02)
    c = _cluster(g, d, 2, A=A, precision=1)
    o = _orc(orc, c, 2)
    c.step(1)
    o.step(1)
    assert c.dt()[0] == o.last_dt
    st = c.get_state()
    byid = np.empty(n)
    byid[st["id"]] = c.binaries()
    np.testing.assert_array_equal(byid[d["id"]], A)


def test_binaries_with_collisions(g_stage, orc):
    """Radii and semi-major axes together: Eqs. 8, 9 and 10 all join Eq. 7's
    minimum, mergers as in the collision tests, both attributes permuted."""
    g = g_stage
    n = 6000
    d = ic.plummer(n, seed=9)
    c = _cluster(g, d, 9, A=_axes(d, 5, 1e-3), R=np.full(n, 1e-4), precision=0)
    for step in range(3):
        o = _orc(orc, c, 9)
        c.step(1)
        o.step(1)
        after = c.get_state()
        np.testing.assert_array_equal(after["id"], o.id)
        np.testing.assert_array_equal(after["r"], o.r)
        np.testing.assert_array_equal(after["m"], o.m)
        _compare_states(after, o)
        assert c.dt()[0] == o.last_dt
        np.testing.assert_array_equal(c.binaries(), o.A)
        np.testing.assert_array_equal(c.radii()[: o.nb], o.R[: o.nb])


def test_dt_cap_bounds_the_step(g_stage, orc):
    """An outside bound shorter than every other timestep is the step (the
    oracle with the same bound gives the same radii); 0 removes it."""
    g = g_stage
    n = 10_000
    d = ic.plummer(n, seed=4)
    c = _cluster(g, d, 4, precision=0)
    o = _orc(orc, c, 4)
    c.step(1)
    o.step(1)
    own = c.dt()[0]
    assert own == o.last_dt
    cap = orc.tse(1.0, own, 0.004)  # 0.25 of the last step
    c.set_dt_cap(cap)
    for _ in range(2):
        o = _orc(orc, c, 4)
        o.dt_cap = cap
        c.step(1)
        o.step(1)
        assert c.dt()[0] == o.last_dt == cap
        np.testing.assert_array_equal(c.get_state()["r"], o.r)
        _compare_states(c.get_state(), o)
    c.set_dt_cap(0.0)
    o = _orc(orc, c, 4)
    c.step(1)
    o.step(1)
    assert c.dt()[0] == o.last_dt > cap
    # a bound longer than the step changes nothing
    c.set_dt_cap(1e3)
    o = _orc(orc, c, 4)
    c.step(1)
    o.step(1)
    assert c.dt()[0] == o.last_dt < 1e3


SIZES = [3, 4097, 2, 9000]


def test_ensemble_caps_and_binaries_per_cluster(g_stage, orc):
    """Clusters of ragged sizes, each with its own cap (none, short, long)
    and binaries in some: each cluster's step and state are its own
    oracle's."""
    g = g_stage
    seeds = [70 + i for i in range(len(SIZES))]
    parts = [ic.plummer(n, s) for n, s in zip(SIZES, seeds)]
    cat = {k: np.concatenate([p[k] for p in parts]) for k in ("r", "vr", "vt", "m", "id")}
    ens = g.Cluster(cat, seeds, sizes=SIZES, precision=0, binaries=1)
    off = np.concatenate([[0], np.cumsum(SIZES)])
    st = ens.get_state()
    A = np.zeros(off[-1])
    A[off[1]:off[2]:3] = 0.01  # binaries in the second cluster
    A[off[3]:off[4]:5] = 2e-3  # and in the fourth
    ens.set_binaries(A)
    ens.step(1)
    dts = ens.dt().copy()
    caps = np.array([0.0, 0.5 * dts[1], 1e3, 0.25 * dts[3]])
    ens.set_dt_cap(caps)
    for step in range(2):
        st = ens.get_state()
        esc = ens.escaped()
        Ab = ens.binaries()
        orcs = []
        for i, sd in enumerate(seeds):
            sl = slice(off[i], off[i + 1])
            o = _oracle_from(orc, {k: st[k][sl] for k in ("r", "vr", "vt", "m", "id", "phi")},
                             sd, st["step"], esc[i])
            o.A = Ab[sl].copy()
            o.dt_cap = caps[i]
            orcs.append(o)
        ens.step(1)
        after = ens.get_state()
        for i, o in enumerate(orcs):
            o.step(1)
            sl = slice(off[i], off[i + 1])
            assert ens.dt()[i] == o.last_dt, (step, i)
            np.testing.assert_array_equal(after["r"][sl], o.r)
            np.testing.assert_array_equal(ens.binaries()[sl], o.A)
        assert ens.dt()[1] == caps[1] and ens.dt()[3] <= caps[3]


def test_binaries_arguments(g_stage):
    g = g_stage
    d = ic.plummer(100, seed=1)
    state = {k: d[k] for k in ("r", "vr", "vt", "m", "id")}
    plain = g.Cluster(state, [1])
    with pytest.raises(g.CMCError):
        plain.set_binaries(np.zeros(100))
    with pytest.raises(g.CMCError):
        plain.binaries()
    c = g.Cluster(state, [1], binaries=1)
    assert np.all(c.binaries() == 0.0)
    bad = np.zeros(100)
    bad[3] = -1.0
    with pytest.raises(g.CMCError):
        c.set_binaries(bad)
    bad[3] = np.inf
    with pytest.raises(g.CMCError):
        c.set_binaries(bad)
    c.set_binaries(np.full(100, 1e-3))
    c.step(1)
    # a new state drops the axes
    c.set_state(state, 0)
    assert np.all(c.binaries() == 0.0)
    for cap in (-1.0, np.nan, np.inf):
        with pytest.raises(g.CMCError):
            c.set_dt_cap(cap)
    for kw in ({"binaries": 2}, {"binaries": 1, "x_bb": 0.0}, {"binaries": 1, "x_bs": -1.0},
               {"x_bb": np.inf}):
        with pytest.raises(g.CMCError):
            g.Cluster(state, [1], **kw)
