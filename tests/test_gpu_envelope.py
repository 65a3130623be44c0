"""FP64 mode's envelope F = 1.2 max_j g(s_j) on its rare path (section 2.1
step 5, Eqs. 13-15).

The screening kernel bounds g at the 21 samples in FP32 and lists the
(star, sample) pairs that may hold the maximum; a second kernel evaluates
them in FP64.  On nearly circular orbits g is flat, FP32 bounds cannot rank
the samples, and most of the 21 are evaluated: more pairs than the list
holds (2N + 1024), so that stars find it full and go to the spill list,
whose pairs the evaluation kernel pools per warp.  The step must still be
the oracle's, star by star."""
import numpy as np
import pytest

import initial_conditions as ic
from test_gpu_parity_steps import _oracle_from
from test_gpu_step import _compare_states

pytestmark = pytest.mark.gpu


def _near_circular(n, seed, spread=1e-3):
    """Plummer positions; v_t the circular speed sqrt(M_k / r_k) of the
    shell model (M_k with the star's own mass), both components perturbed
    by `spread` of it."""
    d = ic.plummer(n, seed=seed)
    rng = np.random.default_rng(seed)
    order = np.argsort(d["r"], kind="stable")
    M = np.empty(n)
    M[order] = np.cumsum(d["m"][order])
    vc = np.sqrt(M / d["r"])
    d["vt"] = vc * (1.0 + spread * rng.standard_normal(n))
    d["vr"] = spread * vc * rng.standard_normal(n)
    return d


@pytest.mark.parametrize("n", [3000, 20_011])
def test_fp64_envelope_spill_path_matches_oracle(g_stage, orc, n):
    g = g_stage
    d = _near_circular(n, seed=11)
    c = g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [11], precision=0)
    for step in range(2):
        before = c.stats()[0]["envelope_fp64"]
        st = c.get_state()
        o = _oracle_from(orc, st, 11, st["step"], c.escaped()[0])
        c.step(1)
        o.step(1)
        # more FP64 evaluations than the pair list holds: the spill path ran
        assert c.stats()[0]["envelope_fp64"] - before > 2 * n + 1024, step
        after = c.get_state()
        np.testing.assert_array_equal(after["id"], o.id)
        np.testing.assert_array_equal(after["r"], o.r)  # new radii bit for bit
        _compare_states(after, o)
        assert c.dt()[0] == o.last_dt
