"""Whole timesteps through the C ABI (cmc_init / cmc_step / cmc_energy /
cmc_lagrange_radii / cmc_get_state / cmc_set_state) against the oracle, and
the reproducibility properties of the design: batched = unbatched,
resumed = uninterrupted, result independent of launch shape."""
import math

import numpy as np
import pytest

import initial_conditions as ic
from gpu_util import dev, host
from test_golden import paper_values

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    assert torch.cuda.is_available()
    import paper_1206_5878_gb300 as lib
    lib.load()
    return lib


def _cluster(g, d, seed, **cfg):
    return g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [seed], **cfg)


def _phi_scale(st):
    nb = np.isfinite(st["r"]).sum()
    return abs(st["phi"][0]) if nb else 1.0


def _compare_states(st, orc_cluster, rtol=1e-12):
    """Same ids at the same sorted slots; r, v_t and Phi within rtol; v_r^2
    within rtol of the energy scale |Phi_0| (v_r = sqrt(Q) magnifies the
    rounding of Q near a turning point)."""
    o = orc_cluster
    np.testing.assert_array_equal(st["id"], o.id)
    fin = np.isfinite(o.r)
    np.testing.assert_array_equal(np.isfinite(st["r"]), fin)
    assert np.all(np.isfinite(st["vr"])) and np.all(np.isfinite(st["vt"]))
    if not fin.any():
        return
    assert np.max(np.abs(st["r"][fin] / o.r[fin] - 1)) < rtol
    scale = _phi_scale(st)
    assert np.max(np.abs(st["vr"] ** 2 - o.vr ** 2)) < rtol * scale
    assert np.all(np.sign(st["vr"]) == np.sign(o.vr))
    assert np.max(np.abs(st["vt"] - o.vt) / (np.abs(o.vt) + 1e-300)) < rtol or \
        np.max(np.abs(st["vt"] ** 2 - o.vt ** 2)) < rtol * scale
    assert np.max(np.abs(st["phi"][fin] / o.phi[fin] - 1)) < rtol


@pytest.mark.parametrize("n,masses", [(1, "equal"), (2, "equal"), (21, "equal"),
                                      (10_000, "equal"), (30_011, "salpeter")])
def test_init_energy_and_lagrange(g, orc, n, masses):
    d = ic.plummer(n, seed=1, masses=masses)
    c = _cluster(g, d, 1)
    o = orc.Cluster(d["r"], d["vr"], d["vt"], d["m"], d["id"], seed=1, pot_mode="dd")
    st = c.get_state()
    np.testing.assert_array_equal(st["id"], o.id)
    np.testing.assert_array_equal(st["r"], o.r)
    assert np.max(np.abs(st["phi"] / o.phi - 1)) < 1e-12
    E = c.energy()[0]
    Eo = o.energy()
    assert np.max(np.abs(E - Eo) / np.abs(Eo).max()) < 1e-12
    fr = [0.0, 0.1, 0.5, 0.9, 1.0]
    lr = c.lagrange_radii(fr)[0]
    lro = o.lagrange_radii(fr)
    # the enclosed-mass threshold is a floating-point decision: the GPU's
    # star is the oracle's or its neighbour where M_k sits at f M_b +- 1e-12
    for a, b in zip(lr, lro):
        if a != b:
            ka, kb = np.searchsorted(o.r, a), np.searchsorted(o.r, b)
            assert abs(ka - kb) == 1
    assert c.nbound()[0] == n and c.kernels_per_step() > 10


@pytest.mark.parametrize("n", [2, 3, 41, 4097, 10_000])
def test_one_step_matches_oracle(g, orc, n):
    d = ic.plummer(n, seed=n)
    c = _cluster(g, d, 7)
    o = orc.Cluster(d["r"], d["vr"], d["vt"], d["m"], d["id"], seed=7, pot_mode="dd")
    c.step(1)
    o.step(1)
    _compare_states(c.get_state(), o)
    assert c.nbound()[0] == o.nb
    assert c.dt()[0] == o.last_dt  # same bins, same stars, same order
    # escaper budget: same stars, same per-star energy, other summation order
    np.testing.assert_allclose(c.escaped()[0], o.escaped, rtol=1e-13, atol=0)
    s = c.stats()[0]
    for k in ("escaped", "degenerate", "cap_hits", "trials", "violations", "clamps"):
        assert s[k] == o.last_stats[k], k


def test_ten_steps_plummer_1e4_fp64(g, orc):
    """Plummer N = 10^4, FP64, 10 steps against the oracle: total energy
    (bound stars plus what the escapers took) conserved to the paper's
    bound on both sides and the same statistics.
    Here each side runs its own trajectory: the potentials of the two sides
    differ in the last bits (other summation order), which the orbits
    amplify step by step.  Star-by-star agreement along the same 10 steps,
    with the state handed to the oracle before each step, is
    test_gpu_parity_steps.py's."""
    d = ic.plummer(10_000, seed=1)
    c = _cluster(g, d, 1)
    o = orc.Cluster(d["r"], d["vr"], d["vt"], d["m"], d["id"], seed=1, pot_mode="dd")
    E0 = c.total_energy()[0]
    bound = paper_values()["energy_drift_bound"]
    for step in range(10):
        c.step(1)
        o.step(1)
        # the near-circular tail grows by about a decade per step and,
        # through Phi, lifts the bulk; an accept decision that flips on
        # last-bit differences moves one star and shifts Phi for all by
        # ~m/r, which moves every turning point and flips more decisions:
        # within a few steps the trajectories decorrelate star by star and
        # agree only statistically (energy, mass profile, escapers)
        assert abs(int(c.nbound()[0]) - o.nb) <= 5
        assert abs(c.total_energy()[0] / E0 - 1) < bound
        assert abs(o.total_energy() / E0 - 1) < bound
        assert abs(c.total_energy()[0] / o.total_energy() - 1) < 2 * bound
        # Lagrangian radii within a few times the sampling noise of 10^4 stars
        np.testing.assert_allclose(c.lagrange_radii([0.1, 0.5, 0.9])[0],
                                   o.lagrange_radii([0.1, 0.5, 0.9]), rtol=0.08)


def test_ensemble_equals_separate_runs(g):
    sizes = [1, 3, 4096, 4097, 9000, 20]
    seeds = [1000 + c for c in range(len(sizes))]
    parts = [ic.plummer(n, s) for n, s in zip(sizes, seeds)]
    cat = {k: np.concatenate([p[k] for p in parts]) for k in ("r", "vr", "vt", "m", "id")}
    ens = g.Cluster(cat, seeds, sizes=sizes)
    ens.step(4)
    est = ens.get_state()
    off = np.concatenate([[0], np.cumsum(sizes)])
    for i, (p, s) in enumerate(zip(parts, seeds)):
        one = _cluster(g, p, s)
        one.step(4)
        st = one.get_state()
        sl = slice(off[i], off[i + 1])
        for k in ("r", "vr", "vt", "m", "id", "phi"):
            np.testing.assert_array_equal(est[k][sl], st[k], err_msg="%d %s" % (i, k))
        assert ens.dt()[i] == one.dt()[0]
        assert ens.stats()[i] == one.stats()[0]
        np.testing.assert_array_equal(ens.energy()[i], one.energy()[0])
        np.testing.assert_array_equal(ens.escaped()[i], one.escaped()[0])


@pytest.mark.parametrize("precision", [0, 1])
def test_step_potential_equals_the_potential_entry_point(g, precision):
    """After a timestep the potential of the bound stars (its per-tile sums
    taken by the post-sort gather) equals, bit for bit, cmc_potential on
    the same sorted radii and masses (the sums read back from memory), for
    every cluster of an ensemble whose sizes leave ragged last tiles."""
    sizes = [4097, 30_000, 12_289]
    seeds = [7 + c for c in range(len(sizes))]
    parts = [ic.plummer(n, s) for n, s in zip(sizes, seeds)]
    cat = {k: np.concatenate([p[k] for p in parts]) for k in ("r", "vr", "vt", "m", "id")}
    ens = g.Cluster(cat, seeds, sizes=sizes, precision=precision)
    ens.step(3)
    st = ens.get_state()
    nb = ens.nbound()
    off = np.concatenate([[0], np.cumsum(sizes)])
    for c in range(len(sizes)):
        sl = slice(off[c], off[c] + int(nb[c]))
        phi, M = g.stage_potential(dev(st["r"][sl]), dev(st["m"][sl]), want_M=True)
        np.testing.assert_array_equal(host(phi), st["phi"][sl], err_msg=str(c))
    assert int(nb.sum()) < sum(sizes)  # escapers were left out of the sums


def test_resume_is_bit_identical(g):
    d = ic.plummer(12_345, seed=3, masses="salpeter")
    a = _cluster(g, d, 3)
    a.step(6)
    b = _cluster(g, d, 3)
    b.step(3)
    mid = b.get_state()
    c = _cluster(g, d, 3)
    c.set_state(mid, mid["step"])
    c.set_escaped(b.escaped())
    c.step(3)
    sa, sc = a.get_state(), c.get_state()
    for k in ("r", "vr", "vt", "m", "id", "phi"):
        np.testing.assert_array_equal(sa[k], sc[k], err_msg=k)
    assert sc["step"] == 6
    np.testing.assert_array_equal(a.escaped(), c.escaped())


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_launch_shape_does_not_change_bits(g, precision):
    d = ic.plummer(20_000, seed=4)
    outs = []
    shapes = [(32, 0, 0), (128, 0, 1), (256, 0, 2)]
    if precision != 2:
        shapes += [(64, v, v % 3) for v in range(1, 7)]
    for blk, var, rv in shapes:
        c = _cluster(g, d, 4, orbit_block=blk, precision=precision, orbit_variant=var,
                     relax_variant=rv, autotune=0)
        assert c.tuning()["orbit_variant"] == var and c.tuning()["relax_variant"] == rv
        c.step(2)
        outs.append((c.get_state(), c.stats()))
    for o, st in outs[1:]:
        for k in ("r", "vr", "vt", "phi"):
            np.testing.assert_array_equal(o[k], outs[0][0][k])
        assert st == outs[0][1]


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_autotuned_shapes_do_not_change_bits(g, precision):
    d = ic.plummer(30_001, seed=6, masses="salpeter")
    a = _cluster(g, d, 6, autotune=0, precision=precision)
    b = _cluster(g, d, 6, autotune=1, precision=precision)
    ta, tb = a.tuning(), b.tuning()
    assert ta == {"orbit_block": 64, "sort_keys_per_thread": 16, "sort_multisplit": "match",
                  "orbit_variant": 0, "relax_variant": 0}
    assert tb["relax_variant"] in (0, 1, 2)
    assert tb["orbit_block"] in (64, 128, 256)
    assert tb["sort_keys_per_thread"] in (8, 16, 24, 32)  # 24 and 32: packed keys only
    assert b.stats()[0]["trials"] == 0  # the tuner's dry run left no trace
    a.step(3)
    b.step(3)
    sa, sb = a.get_state(), b.get_state()
    for k in ("r", "vr", "vt", "m", "id", "phi"):
        np.testing.assert_array_equal(sa[k], sb[k])
    assert a.stats() == b.stats()


def test_host_and_device_inputs_agree(g):
    import torch
    d = ic.plummer(5000, seed=8)
    a = _cluster(g, d, 8)
    b = g.Cluster({k: dev(d[k]) for k in ("r", "vr", "vt", "m", "id")}, [8])
    a.step(2)
    b.step(2)
    sa, sb = a.get_state(), b.get_state()
    out = {k: torch.empty(5000, dtype=torch.float64, device="cuda") for k in ("r", "vr", "vt",
                                                                              "m", "phi")}
    out["id"] = torch.empty(5000, dtype=torch.int32, device="cuda")
    b.get_state(out)
    for k in ("r", "vr", "vt", "m", "id", "phi"):
        np.testing.assert_array_equal(sa[k], sb[k])
        np.testing.assert_array_equal(sa[k], host(out[k]))


def test_mixed_precision_plummer_1e4(g, orc):
    """Mixed mode: energy within the paper's bound; per step, the radii
    advanced from the same FP64 state match the FP64 path to rounding
    (turning points from the enclosed-mass slopes) except for the stars
    whose FP32 accept decision flipped."""
    d = ic.plummer(10_000, seed=2)
    c = _cluster(g, d, 2, precision=1)
    E0 = c.total_energy()[0]
    for _ in range(10):
        c.step(1)
        assert abs(c.total_energy()[0] / E0 - 1) < paper_values()["energy_drift_bound"]
    st = c.get_state()
    f64 = _cluster(g, d, 2)
    f32 = _cluster(g, d, 2, precision=1)
    f64.set_state(st, st["step"])
    f32.set_state(st, st["step"])
    f64.step(1)
    f32.step(1)
    a, b = f64.get_state(), f32.get_state()
    same = np.isin(a["id"], b["id"])
    assert same.all()
    ia, ib = np.argsort(a["id"]), np.argsort(b["id"])
    fin = np.isfinite(a["r"][ia]) & np.isfinite(b["r"][ib])
    rel = np.abs(a["r"][ia][fin] / b["r"][ib][fin] - 1)
    assert (rel < 1e-9).mean() > 0.99


def test_invalid_inputs_are_rejected(g):
    d = ic.plummer(100, seed=1)
    for bad in ("neg_r", "nan_v", "dup_id", "neg_vt", "neg_m"):
        e = {k: d[k].copy() for k in ("r", "vr", "vt", "m", "id")}
        if bad == "neg_r":
            e["r"][5] = -1.0
        elif bad == "nan_v":
            e["vr"][7] = np.nan
        elif bad == "dup_id":
            e["id"][3] = e["id"][4]
        elif bad == "neg_vt":
            e["vt"][2] = -0.1
        else:
            e["m"][9] = -1e-3
        with pytest.raises(g.CMCError) as ei:
            _cluster(g, e, 1)
        assert ei.value.status == 1  # CMC_EINVAL
    for bad_cfg in ({"orbit_variant": 7}, {"orbit_variant": -2}, {"orbit_block": 48},
                    {"relax_variant": 3}, {"relax_variant": -2}):
        with pytest.raises(g.CMCError):
            _cluster(g, d, 1, **bad_cfg)
    c = _cluster(g, d, 1)
    with pytest.raises(g.CMCError):
        c.step(-1)
    with pytest.raises(g.CMCError):
        c.lagrange_radii([1.5])
    with pytest.raises(g.CMCError):
        c.set_escaped([0.0, np.nan])
    c.step(1)  # the context is still usable


def test_set_state_in_order_and_shuffled(g):
    """A state read back is set again in place (its order and ids checked
    without sorting); the same stars shuffled go through the sorts and give
    the same state; an ordered state with a duplicated id is rejected."""
    d = ic.plummer(30_000, seed=6)
    a = _cluster(g, d, 6)
    a.step(2)
    st = a.get_state()
    b = _cluster(g, d, 6)
    b.set_state(st, st["step"])
    rng = np.random.default_rng(1)
    perm = rng.permutation(30_000)
    c = _cluster(g, d, 6)
    c.set_state({k: st[k][perm] for k in ("r", "vr", "vt", "m", "id")}, st["step"])
    sb, sc = b.get_state(), c.get_state()
    for k in ("r", "vr", "vt", "m", "id", "phi"):
        np.testing.assert_array_equal(sb[k], st[k], err_msg=k)
        np.testing.assert_array_equal(sc[k], st[k], err_msg=k)
    b.step(2)
    c.step(2)
    a.step(2)
    for k in ("r", "vr", "vt", "id", "phi"):
        np.testing.assert_array_equal(b.get_state()[k], a.get_state()[k], err_msg=k)
        np.testing.assert_array_equal(c.get_state()[k], a.get_state()[k], err_msg=k)
    dup = {k: st[k].copy() for k in ("r", "vr", "vt", "m", "id")}
    dup["id"][10] = dup["id"][20000]  # still in (r, id) order
    with pytest.raises(g.CMCError) as ei:
        b.set_state(dup, 0)
    assert ei.value.status == 1  # CMC_EINVAL


@pytest.mark.parametrize("n,masses,rng", [(30_011, "equal", "philox"),
                                          (50_000, "salpeter", "philox"),
                                          (20_000, "equal", "taus113")])
def test_fp64_paths_agree_over_steps(g, n, masses, rng):
    """FP64 mode through the certified FP32 screening (precision 0) and by
    bisection on the FP64 table (precision 2) are the same method: over
    five timesteps the states, the statistics and the escapers' budget are
    identical bit for bit."""
    d = ic.plummer(n, seed=12, masses=masses)
    a = _cluster(g, d, 12, precision=0, rng=1 if rng == "taus113" else 0)
    b = _cluster(g, d, 12, precision=2, rng=1 if rng == "taus113" else 0)
    a.step(5)
    b.step(5)
    sa, sb = a.get_state(), b.get_state()
    for k in ("r", "vr", "vt", "m", "id", "phi"):
        np.testing.assert_array_equal(sa[k], sb[k], err_msg=k)
    sta, stb = a.stats()[0], b.stats()[0]
    for k in sta:
        if k not in ("fp64_trials", "envelope_fp64"):  # the screened path's own counts
            assert sta[k] == stb[k], k
    np.testing.assert_array_equal(a.escaped(), b.escaped())


@pytest.mark.parametrize("precision", [0, 1])
def test_packed_sort_keys_change_nothing(g_stage, precision):
    """The timestep's sort on packed keys (each key's low 24 bits, which the
    radix passes leave to the tie fix, carrying the star's index) against
    the keys-and-values sort: the same states, bit for bit, after several
    steps of one cluster and of a ragged ensemble (escapers included)."""
    g = g_stage
    sizes = [1, 3, 20, 4097, 9000, 2, 12_289]
    seeds = [500 + i for i in range(len(sizes))]
    parts = [ic.plummer(n, s) for n, s in zip(sizes, seeds)]
    ens = {k: np.concatenate([p[k] for p in parts]) for k in ("r", "vr", "vt", "m", "id")}
    d = ic.plummer(50_000, seed=6)
    one = {k: d[k] for k in ("r", "vr", "vt", "m", "id")}
    for state, sd, sz in ((one, [6], None), (ens, seeds, sizes)):
        a = g.Cluster(state, sd, sizes=sz, precision=precision, sort_packed=1)
        b = g.Cluster(state, sd, sizes=sz, precision=precision, sort_packed=0)
        a.step(6)
        b.step(6)
        sa, sb = a.get_state(), b.get_state()
        for k in ("r", "vr", "vt", "m", "id", "phi"):
            np.testing.assert_array_equal(sa[k], sb[k], err_msg=k)
        np.testing.assert_array_equal(a.nbound(), b.nbound())
        assert a.stats() == b.stats()
        a.close()
        b.close()


def test_unsorted_state_after_the_tuned_sort_shape(g):
    """A new state in no particular order is ordered by the keys-and-values
    sort, which takes tiles of 16 keys per thread whatever shape the tuner
    chose for the timestep's packed keys (24 or 32 at large N), and puts the
    tuned shape back: the same sorted state, bit for bit, and steps go on."""
    d = ic.plummer(2_000_000, seed=12)
    c = _cluster(g, d, 12)
    tuned = c.tuning()
    c.step(1)
    st = c.get_state()
    perm = np.random.default_rng(1).permutation(len(st["r"]))
    c.set_state({k: np.ascontiguousarray(st[k][perm]) for k in ("r", "vr", "vt", "m", "id")},
                st["step"])
    again = c.get_state()
    for k in ("r", "vr", "vt", "m", "id", "phi"):
        np.testing.assert_array_equal(again[k], st[k], err_msg=k)
    assert c.tuning() == tuned
    c.step(2)
    assert np.all(np.isfinite(c.get_state()["r"][: int(c.nbound()[0])]))
