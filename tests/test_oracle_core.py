"""Pins of the oracle's core diagnostics (section 4.2, Eq. 19): the radial
6th-order density estimator, rho_c = sum rho_i^2 / sum rho_i and the
density-weighted core radius, against what geometry and probability fix:

- a uniform sphere sampled on its volume quantiles (every shell between
  neighbours i - 3 and i + 3 spans exactly 6 / N of the volume and holds 5
  stars): every estimate is 5/6 of the true density, and r_c is the mean
  radius 3R/4;
- a Poisson sample of a uniform sphere: the shell spans 6 exponential volume
  gaps, so the estimate's mean is the true density and its second moment
  25/20 of the density squared, giving rho_c = 1.25 rho;
- a Plummer sphere on its mass quantiles: rho_c and r_c converge to
  (5/6) rho_0 B(3/2, 6) / B(3/2, 7/2) and a (1/24) / (15 pi / 768) = 32 a / (15 pi),
  the continuum integrals int rho^3 dV / int rho^2 dV and
  int rho^2 r dV / int rho^2 dV (the Beta functions from scipy).
"""
import math

import numpy as np
import pytest
from scipy.special import beta

import oracle

A = 3 * math.pi / 16  # Plummer scale of the Henon-unit model (E = -1/4)


def uniform_lattice(n, R):
    return R * ((np.arange(n) + 0.5) / n) ** (1.0 / 3.0), np.full(n, 1.0 / n)


def test_uniform_lattice_density_and_radius():
    n, R = 20_000, 2.0
    r, m = uniform_lattice(n, R)
    rho_true = 3.0 / (4.0 * math.pi * R ** 3)
    rho = oracle.core_rho(r, m)
    inner = rho[3:n - 3]
    assert np.all(rho[:3] == 0) and np.all(rho[n - 3:] == 0)
    np.testing.assert_allclose(inner, 5.0 / 6.0 * rho_true, rtol=1e-11)
    rho_c, r_c, cnt = oracle.core(r, m)
    assert cnt == n - 6
    assert abs(rho_c / (5.0 / 6.0 * rho_true) - 1) < 1e-11
    assert abs(r_c / (0.75 * R) - 1) < 2e-3


def test_poisson_uniform_sphere_moments():
    n, R = 200_000, 1.0
    rng = np.random.default_rng(11)
    r = np.sort(R * rng.random(n) ** (1.0 / 3.0))
    m = np.full(n, 1.0 / n)
    rho_true = 3.0 / (4.0 * math.pi * R ** 3)
    rho = oracle.core_rho(r, m)[3:n - 3]
    # one estimate's relative standard deviation is 1/2; neighbouring
    # estimates share gaps, leaving ~n/6 independent ones: sigma ~ 0.003
    assert abs(rho.mean() / rho_true - 1) < 0.015
    rho_c, _, _ = oracle.core(r, m)
    assert abs(rho_c / rho_true - 1.25) < 0.03


def plummer_quantiles(n, a=A):
    q = (np.arange(n) + 0.5) / n
    return a / np.sqrt(q ** (-2.0 / 3.0) - 1.0), np.full(n, 1.0 / n)


def test_plummer_quantiles_converge_to_the_continuum():
    rho0 = 3.0 / (4.0 * math.pi * A ** 3)
    rho_c_inf = 5.0 / 6.0 * rho0 * beta(1.5, 6.0) / beta(1.5, 3.5)
    r_c_inf = 32.0 * A / (15.0 * math.pi)
    errs = []
    for n in (10_000, 100_000, 1_000_000):
        r, m = plummer_quantiles(n)
        rho_c, r_c, _ = oracle.core(r, m)
        errs.append((abs(rho_c / rho_c_inf - 1), abs(r_c / r_c_inf - 1)))
    assert errs[-1][0] < 5e-5 and errs[-1][1] < 5e-5
    # the errors fall as 1/N (discreteness at the centre and in the tail)
    assert errs[0][0] > 50 * errs[2][0] and errs[0][1] > 50 * errs[2][1]


def test_core_degenerate_inputs():
    # fewer than 7 stars: no estimate
    r, m = uniform_lattice(6, 1.0)
    assert oracle.core(r, m) == (0.0, 0.0, 0)
    # equal radii give shells of no volume: skipped
    r = np.ones(20)
    m = np.full(20, 0.05)
    assert oracle.core(r, m)[2] == 0


def test_half_mass_relaxation_time_scales_as_eq20():
    # Eq. 20: t_rh grows as N / ln(0.1 N) at fixed r_h and as r_h^(3/2)
    t1 = oracle.half_mass_relaxation_time(10 ** 5, 0.8)
    t2 = oracle.half_mass_relaxation_time(10 ** 6, 0.8)
    assert t2 / t1 == pytest.approx(10 * math.log(1e4) / math.log(1e5), rel=1e-12)
    t3 = oracle.half_mass_relaxation_time(10 ** 5, 1.6)
    assert t3 / t1 == pytest.approx(2 ** 1.5, rel=1e-12)
