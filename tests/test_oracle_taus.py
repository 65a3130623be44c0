"""Pins of the oracle's combined Tausworthe generator (the paper's PRNG,
section 3.6: L'Ecuyer 1999, period ~2^113) and of its jump functions:

- each LFSR component has the maximal period 2^k - 1 on its k state bits:
  T^(2^k - 1) is the identity there and T^((2^k - 1)/p) is not, for every
  prime p dividing 2^k - 1 (factorised by sympy), which a wrong shift or
  mask parameter would break;
- the low 32 - k bits of a word never reach its state bits;
- jumping by matrix powers equals stepping, for several displacements;
- streams are D = 2^80 apart: each starts at T^(2^80) of the one before;
- outputs are uniform bit by bit and as fractions of 2^32.
"""
import numpy as np
import pytest

import oracle

K = (31, 29, 28, 25)


def _mask(k):
    return (0xFFFFFFFF << (32 - k)) & 0xFFFFFFFF


@pytest.mark.parametrize("j", range(4))
def test_components_have_maximal_period(j):
    sympy = pytest.importorskip("sympy")
    k = K[j]
    m = _mask(k)
    period = (1 << k) - 1
    T = oracle.taus_pow(j, period)
    for i in range(32 - k, 32):
        assert oracle.gf2_apply(T, 1 << i) & m == 1 << i
    for p in sympy.factorint(period):
        T = oracle.taus_pow(j, period // p)
        assert any(oracle.gf2_apply(T, 1 << i) & m != 1 << i for i in range(32 - k, 32)), p


@pytest.mark.parametrize("j", range(4))
def test_low_bits_never_reach_the_state(j):
    k = K[j]
    T = oracle.taus_pow(j, 1)
    for i in range(32 - k):
        assert oracle.gf2_apply(T, 1 << i) & _mask(k) == 0


@pytest.mark.parametrize("D", [1, 7, 1000, 123457])
def test_jump_equals_stepping(D):
    z0 = oracle.taus_seed(11)
    z = z0.copy()
    oracle.taus_next(z, D)
    for j in range(4):
        assert oracle.gf2_apply(oracle.taus_pow(j, D), int(z0[j])) == int(z[j])


def test_streams_are_2_to_80_apart():
    t = oracle.taus_streams(5, 6).reshape(6, 4)
    np.testing.assert_array_equal(t[0], oracle.taus_seed(5))
    J = [oracle.taus_pow2(j, 80) for j in range(4)]
    for i in range(5):
        nxt = [oracle.gf2_apply(J[j], int(t[i, j])) for j in range(4)]
        assert nxt == [int(x) for x in t[i + 1]]
    # two squarings of T^(2^79) give the same matrix as 80 squarings of T
    J79 = oracle.taus_pow2(0, 79)
    sq = np.array([oracle.gf2_apply(J79, int(c)) for c in J79], dtype=np.uint32)
    np.testing.assert_array_equal(sq, J[0])


def test_seed_words_and_uniformity():
    z = oracle.taus_seed(3)
    assert np.all(z >= np.uint32(0x80000000))
    assert not np.array_equal(z, oracle.taus_seed(4))
    n = 1 << 18
    out = oracle.taus_next(z, n).astype(np.float64)
    u = out / 2.0 ** 32
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / n)
    bits = ((oracle.taus_next(z, n)[:, None] >> np.arange(32, dtype=np.uint32)) & 1).mean(0)
    assert np.all(np.abs(bits - 0.5) < 5 * 0.5 / np.sqrt(n))


def test_orbit_draws_one_block_per_trial_and_one_for_the_sign():
    """With the streams bound, a star's orbit step takes one block of four
    outputs per rejection trial and, once accepted, one for the sign of v_r;
    an escaper takes none."""
    import initial_conditions as ic
    d = ic.plummer(3000, seed=2)
    perm = oracle.sort_perm(d["r"], d["id"])
    r, m = d["r"][perm], d["m"][perm]
    vr, vt, ids = d["vr"][perm], d["vt"][perm], d["id"][perm]
    phi = oracle.potential(r, m)
    table = oracle.taus_streams(9, 3000)
    seen = set()
    for k in (0, 1, 17, 1500, 2999):
        vr_k = vr[k] if k != 2999 else 10.0  # the last star made unbound
        t0 = table.copy()
        with oracle.taus_bound(table):
            o = oracle.orbit_star(k, r, phi, vr_k, vt[k], int(ids[k]), 9, 0)
        seen.add(o["code"])
        i = int(ids[k])
        blocks = 0 if o["code"] in (1, 2) else o["trials"] + (1 if o["code"] == 0 else 0)
        z = t0[4 * i: 4 * i + 4].copy()
        oracle.taus_next(z, 4 * blocks)
        np.testing.assert_array_equal(table[4 * i: 4 * i + 4], z)
        others = np.ones(3000, dtype=bool)
        others[i] = False
        np.testing.assert_array_equal(table.reshape(-1, 4)[others], t0.reshape(-1, 4)[others])
    assert {0, 1} <= seen


def test_cluster_steps_with_streams_are_deterministic_and_differ_from_philox():
    import initial_conditions as ic
    d = ic.plummer(4000, seed=3)
    args = (d["r"], d["vr"], d["vt"], d["m"], d["id"])
    a = oracle.Cluster(*args, seed=4, rng="taus113").step(3)
    b = oracle.Cluster(*args, seed=4, rng="taus113").step(3)
    c = oracle.Cluster(*args, seed=4).step(3)
    np.testing.assert_array_equal(a.r, b.r)
    np.testing.assert_array_equal(a.taus, b.taus)
    assert not np.array_equal(a.r, c.r)
    assert a.last_stats["angle_fails"] == 0 and a.last_stats["cap_hits"] == 0
