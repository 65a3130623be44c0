"""Stage parity: each CUDA kernel of the hot path against the oracle on the
same seeded inputs, through the C ABI.  RNG, sort, timestep, relaxation,
orbit (FP64) and energy correction are bit-exact; the potential scan sums
in another order and is held to 1e-12 relative of the double-double
oracle (about 30 ulp of headroom over the error of a tree of 2^24 sums)."""
import math

import numpy as np
import pytest

import initial_conditions as ic
from gpu_util import dev, host, sorted_plummer

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 19, 20, 21, 4095, 4096, 4097, 3 * 4096 + 17, 100_003]


@pytest.fixture(scope="module")
def g():
    import torch
    assert torch.cuda.is_available()
    import paper_1206_5878_gb300 as lib
    lib.load()
    return lib


def test_philox_bit_exact(g, orc):
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2**32, size=(200_000, 4), dtype=np.uint64).astype(np.uint32)
    for seed in (0, 1, 0xDEADBEEF12345678):
        out = host(g.stage_philox(dev(ctr), seed).view(-1)).reshape(-1, 4)
        np.testing.assert_array_equal(out, orc.philox(ctr, seed))


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("case", ["random", "ties", "short_ties", "near_ties", "escapers"])
def test_sort_permutation_bit_exact(g, orc, n, case):
    rng = np.random.default_rng(n)
    r = rng.lognormal(0.0, 1.5, n)
    ids = rng.permutation(n).astype(np.uint32)
    if case == "near_ties":
        # radii that differ only in the lowest mantissa bits (equal in the
        # bits the radix passes sort on), some exactly equal, shuffled
        base = np.repeat(rng.lognormal(0.0, 1.5, (n + 3) // 4), 4)[:n]
        r = base * (1.0 + rng.integers(0, 8, n) * 2.0 ** -50)
        r = r[rng.permutation(n)]
    elif case == "ties":
        r = np.round(r, 1) + 0.05  # long runs of equal radii in scrambled id order
    elif case == "short_ties":
        r = np.round(r, 5) + 1e-6  # pairs and triples of equal radii
    elif case == "escapers":
        r[rng.random(n) < 0.1] = np.inf
    perm = host(g.stage_sort_radius(dev(r), dev(ids)))
    np.testing.assert_array_equal(perm.astype(np.int64), orc.sort_perm(r, ids))


def test_sort_all_equal_and_presorted(g, orc):
    n = 50_000
    ids = np.random.default_rng(1).permutation(n).astype(np.uint32)
    for r in (np.full(n, 0.5), np.linspace(0.1, 5, n), np.linspace(5, 0.1, n)):
        perm = host(g.stage_sort_radius(dev(r), dev(ids)))
        np.testing.assert_array_equal(perm.astype(np.int64), orc.sort_perm(r, ids))


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("masses", ["equal", "salpeter"])
def test_potential_within_1e12(g, orc, n, masses):
    s = sorted_plummer(n, seed=n, masses=masses)
    phi, M = g.stage_potential(dev(s["r"]), dev(s["m"]), want_M=True)
    ref = orc.potential(s["r"], s["m"], "dd")
    assert np.max(np.abs(host(phi) / ref - 1)) < 1e-12
    Mref = np.cumsum(s["m"].astype(np.longdouble))  # wider than double on x86 and Arm
    assert np.max(np.abs(host(M) / Mref - 1)) < 1e-12


@pytest.mark.parametrize("n", [2, 3, 20, 21, 41, 4097, 100_003])
def test_timestep_bit_exact(g, orc, n):
    s = sorted_plummer(n, seed=7, masses="salpeter")
    lnL = orc.coulomb_log(n)
    dt, nbin = g.stage_timestep(dev(s["r"]), dev(s["vr"]), dev(s["vt"]), dev(s["m"]), lnL)
    dto, nbo = orc.timestep(s["r"], s["vr"], s["vt"], s["m"], lnL)
    np.testing.assert_array_equal(host(nbin), nbo)
    assert host(dt)[0] == dto


@pytest.mark.parametrize("n", [2, 3, 21, 4097, 100_003])
@pytest.mark.parametrize("step", [0, 5])
def test_relax_bit_exact(g, orc, n, step):
    s = sorted_plummer(n, seed=11, masses="salpeter")
    lnL = orc.coulomb_log(n)
    dto, nbo = orc.timestep(s["r"], s["vr"], s["vt"], s["m"], lnL)
    vr, vt = g.stage_relax(dev(s["vr"]), dev(s["vt"]), dev(s["m"]), dev(s["id"]), dev(nbo),
                           dto, lnL, 99, step)
    vro, vto, fails = orc.relax(s["vr"], s["vt"], s["m"], s["id"], nbo, dto, lnL, 99, step)
    assert fails == 0
    np.testing.assert_array_equal(host(vr), vro)
    np.testing.assert_array_equal(host(vt), vto)


def _orbit_inputs(n, seed, masses="equal"):
    import oracle
    s = sorted_plummer(n, seed=seed, masses=masses)
    s["phi"] = oracle.potential(s["r"], s["m"], "dd")
    return s


# precision 0: FP64 through the certified FP32 screening (float-pair
# brackets, FP32 envelope bounds and accept tests, FP64 where undecided);
# precision 2: FP64 bisection on the FP64 table.  Both are the oracle's
# FP64 method, bit for bit.
@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("n", [1, 2, 3, 21, 4097, 30_001])
@pytest.mark.parametrize("masses", ["equal", "salpeter"])
def test_orbit_fp64_bit_exact(g, orc, n, masses, precision):
    s = _orbit_inputs(n, seed=n + 1, masses=masses)
    out = g.stage_orbit(dev(s["r"]), dev(s["phi"]), dev(s["vr"]), dev(s["vt"]), dev(s["id"]),
                        1234, 3, precision=precision)
    ref = orc.orbit_all(s["r"], s["phi"], s["vr"], s["vt"], s["id"], 1234, 3)
    np.testing.assert_array_equal(host(out["code"]), ref["code"])
    for k in ("r_new", "vr", "vt", "phi_new", "rmin", "rmax", "F"):
        np.testing.assert_array_equal(host(out[k]), ref[k], err_msg=k)


@pytest.mark.parametrize("precision", [0, 2])
def test_orbit_special_stars_bit_exact(g, orc, precision):
    """Escapers (E >= 0), radial orbits (J = 0), a trial cap of 1."""
    s = _orbit_inputs(5000, seed=3)
    vr, vt = s["vr"].copy(), s["vt"].copy()
    vesc = np.sqrt(-2 * s["phi"])
    vr[::7] = 1.01 * vesc[::7]
    vt[::7] = 0.0
    vt[1::7] = 0.0
    for trials in (1, 1000):
        out = g.stage_orbit(dev(s["r"]), dev(s["phi"]), dev(vr), dev(vt), dev(s["id"]), 5, 0,
                            max_trials=trials, precision=precision)
        ref = orc.orbit_all(s["r"], s["phi"], vr, vt, s["id"], 5, 0, max_trials=trials)
        np.testing.assert_array_equal(host(out["code"]), ref["code"])
        for k in ("r_new", "vr", "vt", "phi_new", "rmin", "rmax", "F"):
            np.testing.assert_array_equal(host(out[k]), ref[k], err_msg=k)
    assert (ref["code"] == 1).sum() > 0


@pytest.mark.parametrize("n", [4097, 100_003])
def test_orbit_mixed_against_fp64(g, orc, n):
    """Mixed precision: turning points are the FP64 shell roots; the new
    orbit equals the FP64 one unless an FP32 accept decision flips."""
    s = _orbit_inputs(n, seed=5)
    ref = orc.orbit_all(s["r"], s["phi"], s["vr"], s["vt"], s["id"], 77, 1)
    out = g.stage_orbit(dev(s["r"]), dev(s["phi"]), dev(s["vr"]), dev(s["vt"]), dev(s["id"]),
                        77, 1, precision=1)
    code = host(out["code"])
    np.testing.assert_array_equal(code, ref["code"])
    ok = code == 0
    # turning points: FP64 shell roots (the slope of each shell here comes
    # from the same division as in FP64 mode)
    np.testing.assert_array_equal(host(out["rmin"]), ref["rmin"])
    np.testing.assert_array_equal(host(out["rmax"]), ref["rmax"])
    same = ok & (host(out["r_new"]) == ref["r_new"])
    flips = ok.sum() - same.sum()
    assert flips <= max(3, 1e-3 * ok.sum())
    # the accepted orbit is recomputed in FP64 with Phi = Phi_j + M_j (x_j -
    # 1/r) and v_t = J (1/r): a few roundings away from the FP64 path
    scale = np.abs(s["phi"][0])
    a, b = host(out["vr"])[same], ref["vr"][same]
    assert np.max(np.abs(a * a - b * b)) < 1e-12 * scale
    for k in ("vt", "phi_new"):
        a, b = host(out[k])[same], ref[k][same]
        assert np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)) < 1e-13, k
    # F is a sampled bound: g(s) = (dr/ds)/sqrt(Q) with Q = 2(E - Phi) - L^2
    # cancels in FP32 (E and Phi carry 2^-24 relative error each), so the
    # FP32 samples agree with FP64 to ~1e-5 typically, worse where Q is small
    rel = np.abs(host(out["F"])[ok] / ref["F"][ok] - 1)
    assert np.median(rel) < 1e-4 and np.quantile(rel, 0.99) < 1e-2


@pytest.mark.parametrize("n", [3, 4097, 100_003])
def test_energy_correction_bit_exact(g, orc, n):
    s = _orbit_inputs(n, seed=9, masses="salpeter")
    rng = np.random.default_rng(0)
    r_old = s["r"] * rng.uniform(0.5, 2.0, n)
    c = rng.normal(0, 1e-3, n)
    vr, vt = g.stage_energy_correction(dev(s["r"]), dev(s["phi"]), dev(s["vr"]), dev(s["vt"]),
                                       dev(r_old), dev(c))
    vro, vto, _ = orc.energy_correction(s["r"], s["phi"], s["vr"], s["vt"], r_old, c)
    np.testing.assert_array_equal(host(vr), vro)
    np.testing.assert_array_equal(host(vt), vto)
