"""The paper's generator as the alternative draw mode (rng = taus113: the
combined Tausworthe generator, one stream per star id, 2^80 apart) through
the C ABI, against the oracle's streams: the starting states, whole FP64
timesteps (the states and the stream tables after every step, so every
block a kernel draws is the oracle's), mixed mode, checkpoints and the
argument checks."""
import numpy as np
import pytest

import initial_conditions as ic
from test_golden import paper_values
from test_gpu_step import _compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1206_5878_gb300 as lib
    lib.load()
    return lib


def _cluster(g, d, seed, **cfg):
    return g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [seed], rng="taus113",
                     **cfg)


def test_starting_streams_are_the_oracles(g, orc):
    d = ic.plummer(5000, seed=2)
    with _cluster(g, d, 7) as c:
        np.testing.assert_array_equal(c.rng_state(), orc.taus_streams(7, 5000))
    cat, sizes, seeds = ic.ensemble(4, seed=3, sizes=[700, 1200, 333, 2000])
    with g.Cluster(cat, [int(x) for x in seeds], sizes=[int(x) for x in sizes],
                   rng="taus113") as c:
        got = c.rng_state()
        off = 0
        for nc, sd in zip(sizes, seeds):
            want = orc.taus_streams(int(sd), int(nc))
            np.testing.assert_array_equal(got[off: off + want.shape[0]], want)
            off += want.shape[0]
        assert off == got.shape[0]


@pytest.mark.parametrize("n", [3, 41, 4097])
def test_one_fp64_step_matches_oracle(g, orc, n):
    d = ic.plummer(n, seed=n)
    c = _cluster(g, d, 5)
    o = orc.Cluster(d["r"], d["vr"], d["vt"], d["m"], d["id"], seed=5, pot_mode="dd",
                    rng="taus113")
    c.step(1)
    o.step(1)
    _compare_states(c.get_state(), o)
    np.testing.assert_array_equal(c.rng_state(), o.taus)
    s = c.stats()[0]
    for k in ("escaped", "degenerate", "cap_hits", "trials", "violations", "clamps"):
        assert s[k] == o.last_stats[k], k


def test_fp64_steps_from_the_same_state_match_oracle(g, orc):
    """Six FP64 steps at N = 10^4; before each, the oracle takes the GPU's
    state and stream table (the two potentials differ in the last bits, so
    trajectories decorrelate star by star over several steps, as in the
    counter mode): after each step the states agree and the stream tables
    are equal, so every block each kernel drew was the oracle's, escapers,
    degenerate orbits and relaxation pairs included."""
    d = ic.plummer(10_000, seed=1)
    c = _cluster(g, d, 1)
    E0 = c.total_energy()[0]
    for step in range(6):
        st = c.get_state()
        o = orc.Cluster(st["r"], st["vr"], st["vt"], st["m"], st["id"], seed=1, pot_mode="dd",
                        rng="taus113")
        o.taus[:] = c.rng_state()
        o.step_no = step
        c.step(1)
        o.step(1)
        _compare_states(c.get_state(), o)
        np.testing.assert_array_equal(c.rng_state(), o.taus)
    assert abs(c.total_energy()[0] / E0 - 1) < paper_values()["energy_drift_bound"]


def test_mixed_mode_is_deterministic_and_conserves_energy(g):
    d = ic.plummer(100_000, seed=4)
    a = _cluster(g, d, 4, precision=1)
    b = _cluster(g, d, 4, precision=1, autotune=0)
    E0 = a.total_energy()[0]
    a.step(5)
    b.step(5)
    for k in ("r", "vr", "vt", "id"):
        np.testing.assert_array_equal(a.get_state()[k], b.get_state()[k], err_msg=k)
    np.testing.assert_array_equal(a.rng_state(), b.rng_state())
    assert abs(a.total_energy()[0] / E0 - 1) < paper_values()["energy_drift_bound"]
    st = a.stats()[0]
    assert st["cap_hits"] == 0 and st["angle_fails"] == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_resumes_bit_for_bit(g, precision):
    d = ic.plummer(20_000, seed=8)
    a = _cluster(g, d, 8, precision=precision)
    a.step(6)
    b = _cluster(g, d, 8, precision=precision)
    b.step(3)
    mid, words, esc = b.get_state(), b.rng_state(), b.escaped()
    c = _cluster(g, d, 8, precision=precision)
    c.set_state(mid, mid["step"])
    c.set_rng_state(words)
    c.set_escaped(esc)
    c.step(3)
    sa, sc = a.get_state(), c.get_state()
    for k in ("r", "vr", "vt", "m", "id", "phi"):
        np.testing.assert_array_equal(sa[k], sc[k], err_msg=k)
    np.testing.assert_array_equal(a.rng_state(), c.rng_state())


def test_stream_mode_argument_checks(g):
    d = ic.plummer(100, seed=1)
    e = {k: v.copy() for k, v in d.items()}
    e["id"][5] = 4 * 100 + 64  # beyond the stream slots
    with pytest.raises(g.CMCError) as ei:
        _cluster(g, e, 1)
    assert ei.value.status == 1
    with g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [1]) as c:
        with pytest.raises(g.CMCError):
            c.rng_state()
    with _cluster(g, d, 1) as c:
        with pytest.raises(g.CMCError):
            c.set_rng_state(np.zeros(3, dtype=np.uint32))
        with pytest.raises(g.CMCError):
            g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [1], rng=2)
