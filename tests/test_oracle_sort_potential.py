"""Pins for the oracle's sort (section 2.1 step 6), shell potential (Eqs. 1-6)
and diagnostics, against independent brute force and Plummer closed forms."""
import math

import numpy as np
import pytest

import initial_conditions as ic

A = ic.PLUMMER_A


def _py_order(r, ids):
    return sorted(range(len(r)), key=lambda i: (math.isinf(r[i]), 0.0 if math.isinf(r[i])
                                                else r[i], int(ids[i])))


@pytest.mark.parametrize("case", ["random", "equal", "one", "two", "odd", "twovals",
                                  "sorted", "reversed", "escapers", "tiny"])
def test_sort_is_the_r_then_id_order(orc, case):
    g = np.random.default_rng(5)
    n = {"one": 1, "two": 2, "odd": 999}.get(case, 1000)
    r = g.random(n) + 0.1
    ids = g.permutation(n).astype(np.uint32)
    if case == "equal":
        r[:] = 0.7
    elif case == "twovals":
        r = np.where(g.random(n) < 0.5, 0.3, 0.9)
    elif case == "sorted":
        r = np.sort(r)
    elif case == "reversed":
        r = np.sort(r)[::-1].copy()
    elif case == "escapers":
        r[g.random(n) < 0.2] = np.inf
    elif case == "tiny":
        r = r * 1e-300
    perm = orc.sort_perm(r, ids)
    assert sorted(perm.tolist()) == list(range(n))  # a permutation
    assert perm.tolist() == _py_order(r.tolist(), ids)
    rs = r[perm]
    fin = np.isfinite(rs)
    assert np.all(np.diff(rs[fin]) >= 0)
    assert np.all(fin[: fin.sum()])  # escapers last


def _brute_phi(r, m, rq):
    """Eq. 1 at arbitrary radii: -sum_i m_i / max(r, r_i), exactly rounded sum."""
    return np.array([-math.fsum((m / np.maximum(q, r)).tolist()) for q in rq])


@pytest.fixture(scope="module")
def small_cluster():
    d = ic.plummer(1000, seed=3, masses="salpeter")
    perm = np.lexsort((d["id"], d["r"]))
    return {k: v[perm] for k, v in d.items()}


def test_potential_against_brute_force(orc, small_cluster):
    r, m = small_cluster["r"], small_cluster["m"]
    ref = _brute_phi(r, m, r)
    dd = orc.potential(r, m, "dd")
    rec = orc.potential(r, m, "recursion")
    bru = orc.potential(r, m, "brute")
    assert np.max(np.abs(dd / ref - 1)) < 4e-16
    assert np.max(np.abs(rec / ref - 1)) < 1000 * 2.3e-16
    assert np.max(np.abs(bru / ref - 1)) < 1000 * 2.3e-16


def test_potential_energy_identity(orc, small_cluster):
    """1/2 sum m_k Phi_k = W_pair - (G/2) sum m_k^2 / r_k (own mass in M_k)."""
    r, m = small_cluster["r"], small_cluster["m"]
    phi = orc.potential(r, m, "dd")
    n = len(r)
    W = -math.fsum((np.triu(np.outer(m, m) / np.maximum.outer(r, r), 1)).ravel().tolist())
    lhs = 0.5 * math.fsum((m * phi).tolist())
    rhs = W - 0.5 * math.fsum((m * m / r).tolist())
    assert abs(lhs / rhs - 1) < 1e-14
    K, Wo, E = orc.energy(r, small_cluster["vr"], small_cluster["vt"], m)
    assert abs(Wo / W - 1) < n * 2.3e-16
    assert abs(orc.energy_W_brute(r, m) / W - 1) < n * 2.3e-16
    Kref = 0.5 * math.fsum((m * (small_cluster["vr"] ** 2 + small_cluster["vt"] ** 2)).tolist())
    assert abs(K / Kref - 1) < n * 2.3e-16 and E == K + Wo


def test_phi_of_r_is_eq1_between_stars(orc, small_cluster):
    """Eq. 6 interpolation equals Eq. 1 at any radius: inside r_0, on nodes,
    between nodes, beyond the last star."""
    r, m = small_cluster["r"], small_cluster["m"]
    phi = orc.potential(r, m, "dd")
    g = np.random.default_rng(1)
    rq = np.concatenate([[r[0] * 0.5, r[0], r[-1], r[-1] * 3.0], r[[5, 100, 999]],
                         np.exp(g.uniform(np.log(r[0]), np.log(r[-1]), 200))])
    got = np.array([orc.phi_of_r(r, phi, q) for q in rq])
    ref = _brute_phi(r, m, rq)
    assert np.max(np.abs(got / ref - 1)) < 1e-13


@pytest.mark.parametrize("n", [1000, 10_000, 100_000, 1_000_000])
def test_quantile_plummer_potential_converges(orc, n):
    """On the quantile Plummer model (r_k at enclosed-mass fraction
    (k + 1/2)/N, equal masses) the shell potential approaches the closed form
    -GM/sqrt(r^2 + a^2) at first order in 1/N: N r_k |Phi_k - Phi(r_k)| stays
    below 0.2 for every star and every N (its maximum, at the innermost star,
    tends to 1/6).  Dropping the star's own mass from M_k, or counting it
    twice, moves that maximum to about 1/3."""
    r = ic.quantile_plummer(n)
    m = np.full(n, 1.0 / n)
    phi = orc.potential(r, m, "dd")
    werr = n * r * np.abs(phi + 1.0 / np.sqrt(r * r + A * A))
    assert werr.max() < 0.17
    assert werr.max() > 0.16
    # away from the centre the error is O(1/N) without the r weight
    outer = r > A
    assert n * np.max(np.abs(phi[outer] + 1.0 / np.sqrt(r[outer] ** 2 + A * A))) < 0.5


def test_plummer_sample_energy_and_lagrange_radii(orc):
    n = 200_000
    d = ic.plummer(n, seed=11)
    perm = orc.sort_perm(d["r"], d["id"])
    r, vr, vt, m = (d[k][perm] for k in ("r", "vr", "vt", "m"))
    K, W, E = orc.energy(r, vr, vt, m)
    assert abs(E + 0.25) < 10 / math.sqrt(n)  # E = -3 pi G M^2 / (64 a) = -1/4
    assert abs(2 * K + W) < 10 / math.sqrt(n)  # virial equilibrium
    fr = np.array([0.1, 0.5, 0.9])
    lr = orc.lagrange_radii(r, m, fr)
    ana = A / np.sqrt(fr ** (-2.0 / 3.0) - 1.0)
    np.testing.assert_allclose(ana, [0.3087, 0.7686, 2.1837], atol=6e-4)
    assert np.all(np.abs(lr / ana - 1) < 0.03)


def test_lagrange_radii_brute(orc, small_cluster):
    r, m = small_cluster["r"], small_cluster["m"]
    fr = [0.0, 0.01, 0.1, 0.5, 0.9, 1.0]
    got = orc.lagrange_radii(r, m, fr)
    Mb = math.fsum(m.tolist())
    for f, gv in zip(fr, got):
        acc, want = 0.0, r[-1]
        for k in range(len(r)):
            acc += m[k]
            if acc >= f * Mb:
                want = r[k]
                break
        assert gv == want
