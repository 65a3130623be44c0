"""Parity at the benchmark's size: Plummer N = 10^7 (equal masses, seed 1),
the launch configuration bench.py times.  Where the oracle is fast enough
it runs on every star (sort, potential, timestep, relaxation); the orbit
step is checked bit for bit on sampled stars, each computed one by one by
the oracle against the full 10^7-node table."""
import numpy as np
import pytest

import initial_conditions as ic
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

N = 10_000_000


@pytest.fixture(scope="module")
def big(orc):
    import paper_1206_5878_gb300 as g
    d = ic.plummer(N, seed=1)
    c = g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [1], precision=1)
    st = c.get_state()
    yield d, c, st
    c.close()


def test_init_sort_and_potential_full_size(orc, big):
    d, c, st = big
    perm = orc.sort_perm(d["r"], d["id"])
    np.testing.assert_array_equal(st["id"], d["id"][perm])
    np.testing.assert_array_equal(st["r"], d["r"][perm])
    ref = orc.potential(st["r"], st["m"], "dd")
    assert np.max(np.abs(st["phi"] / ref - 1)) < 1e-12
    E = c.energy()[0]
    Eo = orc.energy(st["r"], st["vr"], st["vt"], st["m"])
    # the oracle sums its 10^7 terms one after another: its own rounding
    # is bounded by N eps ~ 1e-9 relative (the GPU sums in a tree)
    assert np.max(np.abs(E - Eo)) < 1e-9 * abs(Eo[2])
    assert abs(E[2] + 0.25) < 1e-3  # Plummer model in Henon units


def test_timestep_and_relaxation_full_size(g_stage, orc, big):
    g = g_stage
    _, _, st = big
    lnL = orc.coulomb_log(N)
    dt, nbin = g.stage_timestep(dev(st["r"]), dev(st["vr"]), dev(st["vt"]), dev(st["m"]), lnL)
    dto, nbo = orc.timestep(st["r"], st["vr"], st["vt"], st["m"], lnL)
    np.testing.assert_array_equal(host(nbin), nbo)
    assert host(dt)[0] == dto
    vr, vt = g.stage_relax(dev(st["vr"]), dev(st["vt"]), dev(st["m"]), dev(st["id"]), dev(nbo),
                           dto, lnL, 1, 0)
    vro, vto, _ = orc.relax(st["vr"], st["vt"], st["m"], st["id"], nbo, dto, lnL, 1, 0)
    np.testing.assert_array_equal(host(vr), vro)
    np.testing.assert_array_equal(host(vt), vto)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_orbit_sampled_full_size(g_stage, orc, big, precision):
    g = g_stage
    _, _, st = big
    out = g.stage_orbit(dev(st["r"]), dev(st["phi"]), dev(st["vr"]), dev(st["vt"]),
                        dev(st["id"]), 1, 0, precision=precision)
    got = {k: host(v) for k, v in out.items()}
    rng = np.random.default_rng(7)
    ks = np.concatenate([[0, 1, N - 2, N - 1], rng.choice(N, 1500, replace=False)])
    flips = 0
    for k in ks:
        o = orc.orbit_star(int(k), st["r"], st["phi"], st["vr"][k], st["vt"][k],
                           int(st["id"][k]), 1, 0)
        assert got["code"][k] == o["code"]
        if precision != 1:
            for key in ("r_new", "vr", "vt", "phi_new", "rmin", "rmax", "F"):
                assert got[key][k] == o[key], (k, key)
        else:
            # turning points bit for bit; with the mixed sampler's own
            # envelope F the oracle accepts the same trial: r_new bit for bit
            assert got["rmin"][k] == o["rmin"] and got["rmax"][k] == o["rmax"], k
            if o["code"] == 0:
                oF = orc.orbit_star(int(k), st["r"], st["phi"], st["vr"][k], st["vt"][k],
                                    int(st["id"][k]), 1, 0, F=got["F"][k])
                assert got["r_new"][k] == oF["r_new"], k
                assert abs(got["vt"][k] - oF["vt"]) <= 1e-12 * oF["vt"]
                assert abs(got["phi_new"][k] / oF["phi_new"] - 1) <= 1e-12
                if got["r_new"][k] != o["r_new"]:
                    flips += 1  # the envelope changed the accepted trial
    assert flips <= 3


def test_mixed_turning_points_equal_fp64_on_every_star(g_stage, big):
    """The sampled step's r_min and r_max (float-pair bracket walks,
    certified or walked again in FP64) equal the FP64 bisection's bit for
    bit on all 10^7 stars, at the start and after three mixed steps; about
    250 stars a step take the walks' fallback (an FP32 bisection), so that
    path is covered too.  And the two FP64 paths (precision 0: FP32
    screening with FP64 decisions; 2: bisection on the FP64 table) give the
    same new orbit, envelope and code on every star."""
    g = g_stage
    d, _, st0 = big
    c = g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [1], precision=1,
                  autotune=0)
    try:
        c.step(3)
        states = [(st0, N), (c.get_state(), int(c.nbound()[0]))]
    finally:
        c.close()
    for st, nb in states:
        cut = {k: st[k][:nb] for k in ("r", "phi", "vr", "vt", "id")}
        o = {p: {k: host(v) for k, v in
                 g.stage_orbit(dev(cut["r"]), dev(cut["phi"]), dev(cut["vr"]), dev(cut["vt"]),
                               dev(cut["id"]), 1, 5, precision=p).items()}
             for p in (2, 1, 0)}
        for key in ("rmin", "rmax"):
            a, b = o[2][key], o[1][key]
            bad = np.nonzero(a.view(np.int64) != b.view(np.int64))[0]
            assert bad.size == 0, (key, bad[:5], a[bad[:5]], b[bad[:5]])
        np.testing.assert_array_equal(o[0]["code"], o[2]["code"])
        for key in ("rmin", "rmax", "F", "r_new", "vr", "vt", "phi_new"):
            a, b = o[0][key], o[2][key]
            bad = np.nonzero(a.view(np.int64) != b.view(np.int64))[0]
            assert bad.size == 0, (key, bad[:5], a[bad[:5]], b[bad[:5]])


def test_one_mixed_step_full_size(big):
    _, c, st = big
    c.step(1)
    s1 = c.get_state()
    assert np.all(np.diff(s1["r"][np.isfinite(s1["r"])]) >= 0)
    assert sorted(s1["id"][:1000].tolist()) != list(range(1000))  # stars moved
    assert np.array_equal(np.sort(s1["id"]), np.arange(N, dtype=np.uint32))
    assert c.stats()[0]["cap_hits"] == 0
