"""Whole timesteps in the default (Philox counter) mode against the oracle,
step after step along a trajectory.

Before each step the oracle takes the GPU's state: the sorted stars and
their potential Phi.  The two potential scans differ in the last bits
(tree against double-double), and over several steps such differences grow
through the orbits.  With the same Phi going in, the orbit step has identical
inputs on both sides, so the new radii must be equal bit for bit.  Only the
potential of the new order and the energy correction that uses it may
differ, by rounding (within 1e-12).

* Plummer N = 10^4, FP64, 10 steps (section 2.1's timestep, section 3.3's
  order).
* Plummer N = 10^5, FP64, the first 5 steps.
* An ensemble of clusters of ragged sizes, 2 steps.  Each cluster is
  compared with its own oracle cluster, in FP64, and star by star with the
  oracle's orbit step in mixed mode (there the oracle takes the mixed
  sampler's own rejection envelope, so that no accept decision may differ).
"""
import numpy as np
import pytest

import initial_conditions as ic
from gpu_util import dev, host
from test_gpu_step import _compare_states

pytestmark = pytest.mark.gpu

STATS = ("escaped", "degenerate", "cap_hits", "trials", "violations", "clamps")


def _oracle_from(orc, st, seed, step, escaped):
    """An oracle cluster holding the GPU's state: same stars in the same
    sorted slots, the GPU's Phi (checked first against the oracle's own
    double-double potential of that state to 1e-12), same step counter
    and escaper budget."""
    o = orc.Cluster(st["r"], st["vr"], st["vt"], st["m"], st["id"], seed=seed, pot_mode="dd")
    np.testing.assert_array_equal(o.id, st["id"])
    nb = o.nb
    if nb:
        assert np.max(np.abs(st["phi"][:nb] / o.phi[:nb] - 1)) < 1e-12
    o.phi[:] = st["phi"]
    o.step_no = int(step)
    o.escaped[:] = escaped
    return o


def _fp64_step_matches(c, o, ci=0, sl=None):
    """After one step from the same state: new radii bit for bit, the rest
    within 1e-12, same timestep, statistics and escapers."""
    st = c.get_state()
    if sl is not None:
        st = {k: (v[sl] if isinstance(v, np.ndarray) else v) for k, v in st.items()}
    np.testing.assert_array_equal(st["r"], o.r)
    _compare_states(st, o)
    assert int(c.nbound()[ci]) == o.nb
    assert c.dt()[ci] == o.last_dt
    s = c.stats()[ci]
    # the statistics accumulate over the run on the GPU and per step in the
    # oracle: compare the increments
    return s, st


@pytest.mark.parametrize("n,steps", [(10_000, 10), (100_000, 5)])
def test_fp64_trajectory_reinjected_each_step(g_stage, orc, n, steps):
    g = g_stage
    d = ic.plummer(n, seed=1)
    c = g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [1], precision=0)
    prev = {k: 0 for k in STATS}
    for step in range(steps):
        st = c.get_state()
        o = _oracle_from(orc, st, 1, st["step"], c.escaped()[0])
        c.step(1)
        o.step(1)
        s, _ = _fp64_step_matches(c, o)
        for k in STATS:
            assert s[k] - prev[k] == o.last_stats[k], (step, k)
        prev = {k: s[k] for k in STATS}
        np.testing.assert_allclose(c.escaped()[0], o.escaped, rtol=1e-13, atol=0)
    # the stars did move: the trajectory left its initial order
    assert not np.array_equal(c.get_state()["id"][:100], np.sort(c.get_state()["id"][:100]))


SIZES = [1, 3, 20, 4097, 9000, 2, 12_289]


@pytest.fixture(scope="module")
def ragged():
    seeds = [1000 + i for i in range(len(SIZES))]
    parts = [ic.plummer(n, s) for n, s in zip(SIZES, seeds)]
    cat = {k: np.concatenate([p[k] for p in parts]) for k in ("r", "vr", "vt", "m", "id")}
    return cat, seeds


def test_ensemble_fp64_each_cluster_matches_its_oracle(g_stage, orc, ragged):
    g = g_stage
    cat, seeds = ragged
    ens = g.Cluster(cat, seeds, sizes=SIZES, precision=0)
    off = np.concatenate([[0], np.cumsum(SIZES)])
    prev = [{k: 0 for k in STATS} for _ in SIZES]
    for step in range(2):
        st = ens.get_state()
        esc = ens.escaped()
        orcs = []
        for i, sd in enumerate(seeds):
            sl = slice(off[i], off[i + 1])
            orcs.append(_oracle_from(orc, {k: st[k][sl] for k in ("r", "vr", "vt", "m", "id",
                                                                  "phi")},
                                     sd, st["step"], esc[i]))
        ens.step(1)
        for i, o in enumerate(orcs):
            o.step(1)
            s, _ = _fp64_step_matches(ens, o, ci=i, sl=slice(off[i], off[i + 1]))
            for k in STATS:
                assert s[k] - prev[i][k] == o.last_stats[k], (step, i, k)
            prev[i] = {k: s[k] for k in STATS}
            np.testing.assert_allclose(ens.escaped()[i], o.escaped, rtol=1e-13, atol=0)


def test_ensemble_mixed_each_cluster_matches_its_oracle(g_stage, orc, ragged):
    """Mixed mode against the FP64 oracle, cluster by cluster, star by star.
    The mixed sampler bounds g(s) with an FP32 envelope F of its own; its
    FP32 accept tests are certified against the FP64 test with that F (the
    undecidable ones are redone in FP64).  So for each cluster, from the
    ensemble's state: the oracle's bins and relaxation give the velocities
    the orbit step starts from (bit-exact on the GPU); the single-cluster
    mixed orbit stage on them must equal the oracle's orbit step run with
    the stage's own F (same code, same r_new bit for bit, velocities and
    Phi(r_new) to 1e-12); and the ensemble's mixed timestep must have put
    every star at exactly that r_new.  No flipped star is allowed."""
    g = g_stage
    cat, seeds = ragged
    ens = g.Cluster(cat, seeds, sizes=SIZES, precision=1)
    off = np.concatenate([[0], np.cumsum(SIZES)])
    moved = 0
    for step in range(2):
        st = ens.get_state()
        stepno = int(st["step"])
        nbs = ens.nbound()
        expect = []
        for i, sd in enumerate(seeds):
            sl = slice(off[i], off[i + 1])
            nb = int(nbs[i])
            c = {k: st[k][sl][:nb].copy() for k in ("r", "vr", "vt", "m", "id", "phi")}
            lnL = orc.coulomb_log(SIZES[i])
            r_new = {}
            if nb >= 1:
                dt, nbin = orc.timestep(c["r"], c["vr"], c["vt"], c["m"], lnL)
                vr1, vt1, _ = orc.relax(c["vr"], c["vt"], c["m"], c["id"], nbin, dt, lnL, sd,
                                        stepno)
                out = g.stage_orbit(dev(c["r"]), dev(c["phi"]), dev(vr1), dev(vt1),
                                    dev(c["id"]), sd, stepno, precision=1)
                got = {k: host(v) for k, v in out.items()}
                scale = abs(c["phi"][0])
                for k in range(nb):
                    F = got["F"][k] if got["code"][k] == 0 else None
                    o = orc.orbit_star(k, c["r"], c["phi"], vr1[k], vt1[k], int(c["id"][k]),
                                       sd, stepno, F=F)
                    assert got["code"][k] == o["code"], (i, k)
                    assert got["r_new"][k] == o["r_new"], (i, k)
                    if o["code"] == 0:
                        assert got["rmin"][k] == o["rmin"] and got["rmax"][k] == o["rmax"]
                        assert abs(got["vr"][k] ** 2 - o["vr"] ** 2) < 1e-12 * scale
                        assert abs(got["vt"][k] / o["vt"] - 1) < 1e-12 if o["vt"] > 0 else \
                            got["vt"][k] == 0.0
                        assert abs(got["phi_new"][k] / o["phi_new"] - 1) < 1e-12
                        moved += 1
                    r_new[int(c["id"][k])] = o["r_new"]
            expect.append(r_new)
        ens.step(1)
        after = ens.get_state()
        for i in range(len(seeds)):
            sl = slice(off[i], off[i + 1])
            ids, r = after["id"][sl], after["r"][sl]
            for ident, rr in zip(ids.tolist(), r.tolist()):
                if ident in expect[i]:
                    assert rr == expect[i][ident], (step, i, ident)
    assert moved > 0.9 * 2 * sum(SIZES[3:5] + SIZES[6:])


def test_many_escapers_take_the_radix_sort(g_stage, orc):
    """A step with more escapers in one cluster than the shell sort lists
    (4096) is sorted by the radix passes instead: the same state as the
    oracle's, new radii bit for bit, escapers in id order at the end."""
    g = g_stage
    n = 30_000
    d = ic.plummer(n, seed=9)
    fast = np.random.default_rng(9).choice(n, 5000, replace=False)
    d["vr"][fast] *= 10.0
    d["vt"][fast] *= 10.0
    c = g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [9], precision=0)
    for step in range(2):
        st = c.get_state()
        o = _oracle_from(orc, st, 9, st["step"], c.escaped()[0])
        c.step(1)
        o.step(1)
        _fp64_step_matches(c, o)
    assert c.stats()[0]["escaped"] > 4096
