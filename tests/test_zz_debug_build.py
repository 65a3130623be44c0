"""The debug build (libcmc_debug.so, -DCMC_DEBUG): the same kernels with
device-side index checks at every table probe and scatter that a wrong
bracket, bucket or segment offset would send out of range.  On the
workloads below no check fails, and the checked build gives the release
build's bits, in every precision, with the Tausworthe streams and with
collisions.  (Built on first use; collected last.)"""
import numpy as np
import pytest

import initial_conditions as ic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbg():
    from paper_1206_5878_gb300 import _build, _native
    _build.build(debug=True)
    lib = _native.load(debug=True)
    assert lib.cmc_is_debug_build() == 1
    return lib


def _site(lib):
    import ctypes
    v = ctypes.c_uint32(0)
    assert lib.cmc_debug_check(ctypes.byref(v)) == 0
    return v.value


@pytest.mark.parametrize("precision,rng,collisions", [(0, "philox", 0), (1, "philox", 0),
                                                      (2, "philox", 0), (1, "taus113", 0),
                                                      (0, "philox", 1)])
def test_debug_build_matches_release_with_no_failed_check(g_stage, dbg, precision, rng,
                                                          collisions):
    g = g_stage
    cat, sizes, seeds = ic.ensemble(4, seed=2)
    sizes = [int(x) for x in sizes]
    seeds = [int(x) for x in seeds]
    st = {k: cat[k] for k in ("r", "vr", "vt", "m", "id")}
    runs = []
    assert _site(dbg) == 0
    for debug in (False, True):
        c = g.Cluster(st, seeds, sizes=sizes, precision=precision, rng=rng,
                      collisions=collisions, debug=debug)
        if collisions:
            c.set_radii(np.full(sum(sizes), 3e-5))
        c.step(4)
        runs.append((c.get_state(), c.stats()))
        c.close()
    assert _site(dbg) == 0
    (a, sa), (b, sb) = runs
    for k in ("r", "vr", "vt", "m", "id", "phi"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert sa == sb


def test_release_build_reports_no_checks(g_stage):
    from paper_1206_5878_gb300 import _native
    lib = _native.load()
    assert lib.cmc_is_debug_build() == 0
    assert _site(lib) == 0
