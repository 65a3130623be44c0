"""Long run to core collapse (section 4.2): a Plummer sphere of 10^5 equal
masses, mixed precision, advanced until its core density (Eq. 19) has grown
ten-thousandfold.

- The time at which rho_c has grown a thousandfold, in units of the initial
  half-mass relaxation time (Eq. 20), is the method's calibration as a whole
  (the relaxation rate, the Eq. 7 timestep, the orbit sampling, the
  potential): the paper finds 17.4 t_rh at this N and cites 15 to 18 t_rh
  from the literature.
- Self-similar collapse makes rho_c a power of r_c: the paper fits a slope
  d ln rho_c / d ln r_c near -2.24 close to collapse (-2.23 in the
  literature it cites), after about -2.5 earlier on.  Here the slope is
  fitted while rho_c grows from 10^2 to 10^4 times its initial value (r_c
  falling about sevenfold).
- The energy budget at collapse.  The potential of Eqs. 1-5 counts each
  star's own mass (M_k includes m_k), so the step conserves
  K + W - S with S = 1/2 sum m_k^2 / r_k, not K + W; and the energy
  correction's clamps of T' < 0 to 0 add energy (counted by the library,
  clamp_energy).  The total K + W + E_esc drifts by about -1.2e-3 of |E_0|
  by the collapse at this N, beyond the paper's 0.04% (its models start at
  N = 10^5 too); what remains after the change of S and the clamp energy
  is taken out stays inside the paper's bound."""
import numpy as np
import pytest

import initial_conditions as ic
from test_golden import paper_values

pytestmark = pytest.mark.gpu


def test_plummer_1e5_core_collapse_time_and_slope(orc):
    import paper_1206_5878_gb300 as g
    n = 100_000
    d = ic.plummer(n, seed=1)
    with g.Cluster({k: d[k] for k in ("r", "vr", "vt", "m", "id")}, [1], precision=1) as c:
        t_rh = orc.half_mass_relaxation_time(n, c.lagrange_radii([0.5])[0][0])
        rho0 = c.core()[0][0]
        E0 = c.total_energy()[0]

        def self_term():
            st = c.get_state()
            nb = int(c.nbound()[0])
            return 0.5 * float(np.sum(st["m"][:nb] ** 2 / st["r"][:nb]))

        S0 = self_term()
        t, t_cc = 0.0, None
        late = []  # (r_c, rho_c) once rho_c > 100 rho_c0
        for step in range(1, 40_001):
            c.step(1)
            t += float(c.dt()[0])
            if step % 20 == 0:
                rho_c, r_c, _ = c.core()[0]
                if t_cc is None and rho_c > 1e3 * rho0:
                    t_cc = t
                    # at a thousandfold about 2.3% of the stars have escaped
                    # and the drift is about -1.2e-3, 90% of it the clamps'
                    # energy; without the change of S and the clamps, what
                    # is left was measured at 3e-5
                    assert c.nbound()[0] > 0.95 * n
                    E = c.total_energy()[0]
                    e_clamp = c.stats()[0]["clamp_energy"] * 2.0 ** -62
                    assert abs(E / E0 - 1) < 2e-3
                    rest = (E - e_clamp - (self_term() - S0)) / E0 - 1
                    assert abs(rest) < paper_values()["energy_drift_bound"], rest
                if rho_c > 1e2 * rho0:
                    late.append((r_c, rho_c))
                if rho_c > 1e4 * rho0:
                    break
            assert t < 25 * t_rh, "no collapse by 25 t_rh"
        assert t_cc is not None and late and late[-1][1] > 1e4 * rho0
        assert 15.0 <= t_cc / t_rh <= 19.0, t_cc / t_rh
        rc, rho = np.array(late).T
        beta = np.polyfit(np.log(rc), np.log(rho), 1)[0]
        # the paper: about -2.5 early in the collapse, -2.24 deep in it;
        # measured -2.31 to -2.33 over seeds 1-3 and N = 10^5, 10^6
        assert -2.5 < beta < -2.2, beta
