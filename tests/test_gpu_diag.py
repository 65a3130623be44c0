"""The per-step diagnostics ring (cmc_config.diag_ring): records written on
the device at every step end hold what the host calls report after that
step, the ring keeps the newest records in order when it wraps, and it
changes nothing of the trajectory."""
import numpy as np
import pytest

import initial_conditions as ic

pytestmark = pytest.mark.gpu


def _cluster(g, d, seeds, sizes=None, **cfg):
    return g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, seeds, sizes=sizes, **cfg)


@pytest.mark.parametrize("precision", [0, 1])
def test_ring_records_match_host_calls(g_stage, precision):
    g = g_stage
    import paper_1206_5878_gb300._native as nat
    F = {k: i for i, k in enumerate(nat.DIAG_FIELDS)}
    cat, sizes, seeds = ic.ensemble(3, seed=4)
    sizes = [int(x) for x in sizes]
    seeds = [int(x) for x in seeds]
    cap, steps = 4, 7
    c = _cluster(g, cat, seeds, sizes, precision=precision, diag_ring=cap)
    assert c.diagnostics().shape == (3, 0, len(nat.DIAG_FIELDS))
    seen = []
    for _ in range(steps):
        c.step(1)
        e = c.energy()
        seen.append({"dt": c.dt().copy(), "nb": c.nbound().copy(), "K": e[:, 0].copy(),
                     "W": e[:, 1].copy(), "esc": c.escaped().copy(),
                     "trials": np.array([s["trials"] for s in c.stats()])})
    rec = c.diagnostics()
    assert rec.shape == (3, cap, len(nat.DIAG_FIELDS))
    for i in range(cap):
        h = seen[steps - cap + i]
        np.testing.assert_array_equal(rec[:, i, F["step"]], steps - cap + i + 1)
        np.testing.assert_array_equal(rec[:, i, F["dt"]], h["dt"])
        np.testing.assert_array_equal(rec[:, i, F["nbound"]], h["nb"])
        np.testing.assert_array_equal(rec[:, i, F["K"]], h["K"])
        np.testing.assert_array_equal(rec[:, i, F["W"]], h["W"])
        np.testing.assert_array_equal(rec[:, i, F["M_esc"]], h["esc"][:, 0])
        np.testing.assert_array_equal(rec[:, i, F["E_esc"]], h["esc"][:, 1])
        np.testing.assert_array_equal(rec[:, i, F["E_total"]],
                                      (h["K"] + h["W"]) + h["esc"][:, 1])
        np.testing.assert_array_equal(rec[:, i, F["trials"]], h["trials"])
        np.testing.assert_array_equal(rec[:, i, F["err"]], 0)


def test_ring_changes_nothing_and_is_off_by_default(g_stage):
    g = g_stage
    d = ic.plummer(20_000, seed=9)
    a = _cluster(g, d, [9], precision=1)
    b = _cluster(g, d, [9], precision=1, diag_ring=3)
    assert b.kernels_per_step() == a.kernels_per_step() + 4
    a.step(4)
    b.step(4)
    sa, sb = a.get_state(), b.get_state()
    for k in ("r", "vr", "vt", "m", "id", "phi"):
        np.testing.assert_array_equal(sa[k], sb[k])
    assert a.stats() == b.stats()
    with pytest.raises(g.CMCError):
        a.diagnostics()
    with pytest.raises(g.CMCError):
        _cluster(g, d, [9], diag_ring=-1)
