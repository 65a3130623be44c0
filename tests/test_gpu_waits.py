"""The sort's bounded device waits run out, on purpose, without faulting or
hanging anything: with a look-back limit of one poll, a timestep whose many
escapers hand its sort to the radix passes gives up on earlier tiles,
reports CMC_ETIMEOUT and poisons its context (later calls return
CMC_EPOISONED), while another context on the device is unaffected; with a tie-fix limit of a few moves the stage sort of a run of
equal radii falls back to sorting by id, then by radius, and still returns
the (r, id) order.  Every wait bound is host-set (cmc_set_wait_limits) and
restored to its default afterwards."""
import numpy as np
import pytest

import initial_conditions as ic
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1206_5878_gb300 as lib
    lib.load()
    return lib


def _cluster(g, n, seed):
    d = ic.plummer(n, seed=seed)
    return g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [seed], autotune=0)


def _unbound(n, seed, n_fast):
    """A Plummer sample with n_fast stars sent out at ten times their
    speed (E > 0: they escape in the first step)."""
    d = ic.plummer(n, seed=seed)
    fast = np.random.default_rng(seed).choice(n, n_fast, replace=False)
    d["vr"][fast] *= 10.0
    d["vt"][fast] *= 10.0
    return d


def test_lookback_limit_times_out_and_poisons(g):
    """More escapers in one step than the shell sort lists hand the step to
    the radix sort, whose look-back then runs out."""
    other = _cluster(g, 50_000, 2)  # built before the limit: unaffected later
    d = _unbound(2_000_000, 1, 6000)  # 489 sort tiles, > 4096 escapers
    c = g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [1], autotune=0)
    try:
        g.set_wait_limits(lookback_polls=1)
        with pytest.raises(g.CMCError) as ei:
            c.step(1)
        assert ei.value.status == 5  # CMC_ETIMEOUT
        assert "look-back" in str(ei.value)
        with pytest.raises(g.CMCError) as ei:
            c.energy()
        assert ei.value.status == 6  # CMC_EPOISONED
    finally:
        g.set_wait_limits()
        c.close()
    other.step(2)  # defaults again: a full-size wait budget
    st = other.get_state()
    fin = np.isfinite(st["r"])
    assert np.all(np.diff(st["r"][fin]) >= 0)


def test_stage_sort_reports_the_timeout(g):
    d = ic.plummer(2_000_000, seed=4)
    try:
        g.set_wait_limits(lookback_polls=1)
        with pytest.raises(g.CMCError) as ei:
            g.stage_sort_radius(dev(d["r"]), dev(d["id"]))
        assert ei.value.status == 5
    finally:
        g.set_wait_limits()
    perm = host(g.stage_sort_radius(dev(d["r"]), dev(d["id"])))
    assert np.all(np.diff(d["r"][perm.astype(np.int64)]) >= 0)


def test_tie_move_limit_falls_back_and_keeps_the_order(g, orc):
    n = 20_000
    r = np.full(n, 0.7)
    r[::7] = 0.3  # two long runs of equal radii
    ids = np.random.default_rng(3).permutation(n).astype(np.uint32)
    try:
        g.set_wait_limits(tie_moves=8)
        perm = host(g.stage_sort_radius(dev(r), dev(ids)))
    finally:
        g.set_wait_limits()
    np.testing.assert_array_equal(perm.astype(np.int64), orc.sort_perm(r, ids))


def test_wait_limit_arguments(g):
    g.set_wait_limits(0, 0)
    g.set_wait_limits(-5, -1)  # non-positive: the defaults
