"""Core diagnostics on the GPU (cmc_core: the 6th-order radial density
estimator, Eq. 19's rho_c and the density-weighted core radius) against the
oracle's: the per-star estimates are the same expressions, so only the
summation order differs (rho_c, r_c within 1e-12 relative; the number of
estimates exact).  Initial Plummer and Salpeter clusters, a state after
mixed steps, every cluster of an ensemble, and clusters too small for an
estimate."""
import numpy as np
import pytest

import initial_conditions as ic

pytestmark = pytest.mark.gpu


def _cluster(g, d, seeds=(1,), sizes=None, **cfg):
    return g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, list(seeds), sizes=sizes,
                     **cfg)


def _check(got, r, m, orc):
    rho_c, r_c, n_est = orc.core(r, m)
    assert int(got[2]) == n_est
    if n_est == 0:
        assert got[0] == 0.0 and got[1] == 0.0
        return
    assert abs(got[0] / rho_c - 1) < 1e-12
    assert abs(got[1] / r_c - 1) < 1e-12


@pytest.mark.parametrize("masses", ["equal", "salpeter"])
def test_core_matches_oracle_initial(orc, masses):
    import paper_1206_5878_gb300 as g
    d = ic.plummer(100_000, seed=3, masses=masses)
    with _cluster(g, d) as c:
        st = c.get_state()
        nb = int(c.nbound()[0])
        _check(c.core()[0], st["r"][:nb], st["m"][:nb], orc)


def test_core_matches_oracle_after_steps(orc):
    import paper_1206_5878_gb300 as g
    d = ic.plummer(200_000, seed=5)
    with _cluster(g, d, precision=1) as c:
        c.step(4)
        st = c.get_state()
        nb = int(c.nbound()[0])
        _check(c.core()[0], st["r"][:nb], st["m"][:nb], orc)


def test_core_per_cluster_of_an_ensemble(orc):
    import paper_1206_5878_gb300 as g
    cat, sizes, seeds = ic.ensemble(6, seed=2)
    sizes = [int(x) for x in sizes]
    with g.Cluster(cat, [int(x) for x in seeds], sizes=sizes) as c:
        c.step(2)
        st = c.get_state()
        nbs = c.nbound()
        got = c.core()
        off = np.concatenate([[0], np.cumsum(sizes)])
        for i in range(len(sizes)):
            sl = slice(off[i], off[i] + int(nbs[i]))
            _check(got[i], st["r"][sl], st["m"][sl], orc)


@pytest.mark.parametrize("n", [1, 6, 7, 8])
def test_core_small_clusters(orc, n):
    import paper_1206_5878_gb300 as g
    d = ic.plummer(n, seed=1)
    with _cluster(g, d) as c:
        st = c.get_state()
        _check(c.core()[0], st["r"][:n], st["m"][:n], orc)
