"""Stellar collisions on the GPU (configuration collisions = 1): Eq. 8's
collision timestep and sticky-sphere mergers of relaxation pairs (section
2.1 steps 2 and 3(iii)) against the oracle.

Before each step the oracle takes the GPU's state, potential and radii (as
in test_gpu_parity_steps.py); the collision decisions, merged masses, radii
and new positions must then be the oracle's bit for bit, the booked change
of K + W the oracle's to rounding (fixed-point against FP64 sums)."""
import numpy as np
import pytest

import initial_conditions as ic
from test_golden import paper_values
from test_gpu_parity_steps import _oracle_from
from test_gpu_step import _compare_states

pytestmark = pytest.mark.gpu

E62 = 2.0 ** -62


def _cluster(g, d, seed, R, **cfg):
    c = g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [seed], collisions=1, **cfg)
    # radii belong to the sorted order the context keeps: map them by id
    st = c.get_state()
    byid = np.empty(len(d["id"]))
    byid[d["id"]] = R
    c.set_radii(byid[st["id"]])
    return c


def _orc_with_radii(orc, c, seed):
    st = c.get_state()
    o = _oracle_from(orc, st, seed, st["step"], c.escaped()[0])
    o.R = c.radii().copy()
    return o, st


@pytest.mark.parametrize("n,rad", [(5000, 1e-4), (20_011, 3e-5)])
def test_fp64_steps_with_collisions_match_oracle(g_stage, orc, n, rad):
    g = g_stage
    d = ic.plummer(n, seed=n)
    c = _cluster(g, d, 3, np.full(n, rad), precision=0)
    prev = {"collisions": 0, "collision_energy": 0, "escaped": 0}
    merged_total = 0
    for step in range(4):
        o, st = _orc_with_radii(orc, c, 3)
        c.step(1)
        o.step(1)
        after = c.get_state()
        np.testing.assert_array_equal(after["id"], o.id)
        np.testing.assert_array_equal(after["r"], o.r)  # new radii bit for bit
        np.testing.assert_array_equal(after["m"], o.m)  # merged masses
        np.testing.assert_array_equal(c.radii()[: o.nb], o.R[: o.nb])  # merged radii
        _compare_states(after, o)
        assert c.dt()[0] == o.last_dt  # Eq. 8 joined Eq. 7, bit for bit
        s = c.stats()[0]
        n_col = s["collisions"] - prev["collisions"]
        assert n_col == o.collisions[0]
        e_col = (s["collision_energy"] - prev["collision_energy"]) * E62
        assert abs(e_col - o.collisions[1]) <= 1e-10 * max(abs(o.collisions[1]), 1e-30)
        assert s["escaped"] - prev["escaped"] == o.last_stats["escaped"]
        prev = {k: s[k] for k in prev}
        merged_total += n_col
    assert merged_total > 0


def test_mixed_mode_merges_the_same_pairs(g_stage, orc):
    """Mixed mode draws its orbits with its own envelope, but relaxation and
    the collision decisions are FP64 in both modes: the same pairs merge,
    with the same masses and radii, and the same stars leave."""
    g = g_stage
    n = 8000
    d = ic.plummer(n, seed=2)
    c = _cluster(g, d, 2, np.full(n, 1e-4), precision=1)
    o, st = _orc_with_radii(orc, c, 2)
    c.step(1)
    o.step(1)
    after = c.get_state()
    ia, ib = np.argsort(after["id"]), np.argsort(o.id)
    np.testing.assert_array_equal(after["m"][ia], o.m[ib])
    np.testing.assert_array_equal(np.isfinite(after["r"][ia]), np.isfinite(o.r[ib]))
    np.testing.assert_array_equal(c.radii()[ia], o.R[ib])
    assert c.stats()[0]["collisions"] == o.collisions[0] > 0


@pytest.mark.parametrize("precision", [0, 1])
def test_energy_budget_with_collisions(g_stage, precision):
    """N = 10^5 over 50 steps with radii that make a few hundred stars
    merge: K + W + E_esc, less what the mergers changed of K + W, stays
    within the paper's bound; the mass of the bound stars plus what left
    is conserved."""
    g = g_stage
    n = 100_000
    d = ic.plummer(n, seed=5)
    c = _cluster(g, d, 5, np.full(n, 5e-6), precision=precision)
    E0 = c.total_energy()[0]
    M0 = d["m"].sum()
    c.step(50)
    s = c.stats()[0]
    assert s["collisions"] > 50
    budget = c.total_energy()[0] - s["collision_energy"] * E62
    assert abs(budget / E0 - 1) < paper_values()["energy_drift_bound"]
    st = c.get_state()
    nb = int(c.nbound()[0])
    assert abs(st["m"][:nb].sum() + c.escaped()[0][0] - M0) < 1e-12
    assert s["escaped"] + s["collisions"] == n - nb


def test_radii_arguments(g_stage):
    g = g_stage
    d = ic.plummer(100, seed=1)
    plain = g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [1])
    with pytest.raises(g.CMCError):
        plain.set_radii(np.zeros(100))
    c = g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [1], collisions=1)
    assert np.all(c.radii() == 0.0)
    bad = np.zeros(100)
    bad[3] = -1.0
    with pytest.raises(g.CMCError):
        c.set_radii(bad)
    bad[3] = np.nan
    with pytest.raises(g.CMCError):
        c.set_radii(bad)
    c.set_radii(np.full(100, 1e-3))
    c.step(1)
    with pytest.raises(g.CMCError):
        g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [1], collisions=2)
