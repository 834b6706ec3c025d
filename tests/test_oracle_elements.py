"""Pins of the oracle's element sampling and libration detector (section 3), no GPU.

* elements invert the input generator's element -> Cartesian conversion
  (independent code) and the exact hyperbolic orbit (mpmath);
* the barycentre makes the total momentum of star and planets zero;
* the resonant argument of a constructed configuration;
* physics: particles placed in Neptune's 3:2 resonance (phi = 180 deg) librate
  (phi never within 10 deg of 0) over 2e4 yr, particles at 45-50 AU circulate.
"""
import numpy as np
import pytest

import glisse_inputs as gi
import pins


def _ang(x, y):
    return np.abs(np.mod(np.asarray(x) - np.asarray(y) + np.pi, 2 * np.pi) - np.pi)


def test_elements_invert_the_generator(orc):
    rng = np.random.default_rng(0)
    n = 3000
    a = rng.uniform(1.0, 100.0, n)
    e = rng.uniform(0.01, 0.95, n)
    inc = rng.uniform(0.02, 3.12, n)
    ang = rng.uniform(0.0, 2 * np.pi, (3, n))
    st = gi.elements_to_cartesian(gi.G, a, e, inc, *ang)
    el = orc.elements(gi.G, st)
    # omega and M lose ~1/e of their accuracy for small e; Omega ~1/sin i for small i
    assert np.abs(el[:, 0] / a - 1).max() < 1e-12
    assert np.abs(el[:, 1] - e).max() < 1e-13
    assert np.abs(el[:, 2] - inc).max() < 1e-13
    assert (_ang(el[:, 3], ang[0]) * np.sin(inc)).max() < 1e-13
    assert (_ang(el[:, 4], ang[1]) * e * np.sin(inc)).max() < 1e-12
    assert (_ang(el[:, 5], ang[2]) * e).max() < 1e-12
    # the sums that stay defined as e, i -> 0: longitude of pericentre and mean longitude
    varpi, lam = ang[0] + ang[1], ang[0] + ang[1] + ang[2]
    assert (_ang(el[:, 3] + el[:, 4], varpi) * e).max() < 1e-12
    assert _ang(el[:, 3] + el[:, 4] + el[:, 5], lam).max() < 1e-11


def test_elements_of_an_exact_hyperbola(orc):
    pytest.importorskip("mpmath")
    a, e, inc, Om, om, M = -25.0, 1.5, 0.3, 1.1, 2.2, 0.7
    st = pins.analytic_state(gi.G, 25.0, e, inc, Om, om, M)  # |a| = 25 AU
    el = orc.elements(gi.G, st[None])[0]
    assert abs(el[0] / a - 1) < 1e-13 and abs(el[1] - e) < 1e-14
    assert _ang(el[2], inc) < 1e-14 and _ang(el[3], Om) < 1e-14 and _ang(el[4], om) < 1e-13
    assert abs(el[5] - M) < 1e-13


def test_circular_equatorial_orbit(orc):
    r = 7.0
    st = np.array([[r, 0.0, 0.0, 0.0, np.sqrt(gi.G / r), 0.0]])
    el = orc.elements(gi.G, st)[0]
    assert abs(el[0] - r) < 1e-13 * r and el[1] < 1e-15 and el[2] == 0.0
    assert el[3] == 0.0 and el[4] == 0.0 and abs(el[5]) < 1e-15


def test_barycentre_has_zero_momentum(orc):
    w = gi.make("tiny", n=1)
    pl = w["planets"]
    R = orc.barycentre(1.0, pl[:, 0], pl[:, 1:])
    # star at the heliocentric origin at rest; momenta about the barycentre sum to zero
    p = 1.0 * (np.zeros(6) - R) + np.sum(pl[:, 0, None] * (pl[:, 1:] - R), axis=0)
    scale = np.sum(np.abs(pl[:, 0, None] * pl[:, 1:]), axis=0)
    assert np.all(np.abs(p) < 1e-15 * scale), (p, scale)
    assert np.abs(R[:3]).max() > 1e-4  # not trivially zero


def test_resonant_argument_of_a_constructed_configuration(orc):
    """Particle at pericentre (M = 0) with varpi = 0.4, planet with mean longitude 1.3:
    phi31 = 3 lambda - lambda_N - 2 varpi = 3 (0.4) - 1.3 - 2 (0.4) = -0.9 -> 2 pi - 0.9."""
    pm = np.array([1e-4])
    mu_pl = gi.G * (1.0 + pm[0])
    planet = gi.elements_to_cartesian(mu_pl, 30.0, 0.01, 0.02, 0.5, 0.3, 0.5)  # lambda_N = 1.3
    part = gi.elements_to_cartesian(gi.G, 62.6, 0.2, 0.05, 0.1, 0.3, 0.0)      # varpi = 0.4, lambda = 0.4
    import ctypes as C

    el = np.empty((1, 6))
    ph = np.empty(1)
    n0, n1, cnt = np.zeros(1, np.uint8), np.zeros(1, np.uint8), np.zeros(1, np.int32)
    live = np.ones(1, np.uint8)
    st = np.ascontiguousarray(part[None])
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    u8 = lambda a: a.ctypes.data_as(C.POINTER(C.c_uint8))
    rc = orc.lib().orc_sample(1.0, 1, dp(pm), dp(np.ascontiguousarray(planet[None])), 0, 0, 3, 1,
                              np.radians(10.0), dp(st), u8(live), 1, dp(el), dp(ph), u8(n0), u8(n1),
                              cnt.ctypes.data_as(C.POINTER(C.c_int32)))
    assert rc == 0
    assert abs(ph[0] - (2 * np.pi - 0.9)) < 1e-12
    assert cnt[0] == 1 and n0[0] == 0 and n1[0] == 0


def _resonant_and_circulating(orc):
    w = gi.make("tiny", n=1)
    pl = w["planets"]
    elN = orc.elements(gi.G * (1 + pl[3, 0]), pl[3:4, 1:])[0]
    lamN = elN[3] + elN[4] + elN[5]
    rng = np.random.default_rng(0)
    rows = []
    for _ in range(6):
        varpi = rng.uniform(0, 2 * np.pi)
        lam = (np.pi + 2 * lamN + varpi) / 3  # phi32 = 180 deg
        rows.append(gi.elements_to_cartesian(gi.G, elN[0] * 1.5 ** (2 / 3), 0.25, np.radians(3), 0.3,
                                             varpi - 0.3, lam - varpi))
    for k in range(6):
        rows.append(gi.elements_to_cartesian(gi.G, 45.0 + k, 0.05, np.radians(3), 0.3,
                                             *rng.uniform(0, 2 * np.pi, 2)))
    return pl, np.array(rows)


def test_resonant_particles_librate_and_others_circulate(orc):
    """Samples every 5 yr: phi32 of the circulating particles turns by at most ~6 deg per
    sample (period >= 300 yr), less than the 20 deg window around 0, so no crossing is missed."""
    pl, pa = _resonant_and_circulating(orc)
    out = orc.run_sampled(1.0, pl, pa, 0.5, 40000, 10, frame=0, res_planet=3, res_p=3, res_q=2)
    assert np.all(out["removal_step"] < 0)
    assert np.all(out["count"] == 4000)
    librating = (out["near0"] == 0) | (out["near180"] == 0)
    assert librating[:6].all() and not librating[6:].any(), (out["near0"], out["near180"])
    # the barycentric frame gives the same classification
    outb = orc.run_sampled(1.0, pl, pa, 0.5, 40000, 10, frame=1, res_planet=3, res_p=3, res_q=2)
    np.testing.assert_array_equal((outb["near0"] == 0) | (outb["near180"] == 0), librating)
