"""Pins of the oracle against numbers the paper prints (tests/golden/paper_values.txt), no GPU.

The paper prints no particle states, but it does print where mean-motion
resonances sit and how the 3:1 resonance with Neptune looks in the resonant
argument.  Both follow from the map the oracle integrates (the drift's
mean motions and the planets' kicks), from its element conversion and from
its libration test, so they pin those parts against the paper itself:

* resonance locations (Section 3.3): circular particles started at the
  printed locations, integrated with the four planets, have mean motions whose
  ratio to the planet's, measured from the unwrapped mean longitudes, puts the
  exact commensurability within the printed variation of the printed location;
* the 3:1 resonance (Section 4.2.1): particles with phi_31 = 180 deg scanned
  across a librate (by the paper's 10 deg criterion) in one interval that
  contains the printed centre, is no wider than the printed width, and lies in
  the printed initial box; particles farther out circulate.

The synthetic planets stand in for the real ones (same semimajor axes and
masses to the digits the paper's application uses), so agreement is at the
level the paper's own footnote states: a few tenths of an au.
"""
import numpy as np
import pytest

import glisse_inputs as gi
import pins

PLANET_INDEX = {"uranus": 2, "neptune": 3}


def _lam(el):
    return el[..., 3] + el[..., 4] + el[..., 5]


def test_printed_resonance_locations(orc):
    vals = pins.paper_values("resonance_locations")
    variation = float(vals.pop("variation"))
    res = [v.split() for v in vals.values()]
    w = gi.make("tiny", n=1)
    planets = w["planets"].copy()
    rng = np.random.default_rng(5)
    a0 = np.array([float(r[3]) for r in res])
    particles = np.array([gi.elements_to_cartesian(gi.G, a, 0.0, 0.0, 0.0, 0.0, ph)
                          for a, ph in zip(a0, rng.uniform(0.0, 2 * np.pi, len(res)))])
    dt, every, n_samples = 0.5, 20, 400  # 10 yr between samples, 4000 yr in all
    run = orc.ParticleRun(1.0, np.ascontiguousarray(planets[:, 0]), particles, orc.rcrit(1.0, planets, 0, 1.0), 1000.0)
    lam_p, lam_pl = [], []
    for _ in range(n_samples):
        planets, log, _ = orc.planet_wh(1.0, planets, dt, every)
        run.advance(log, dt)
        lam_p.append(_lam(orc.elements(gi.G, run.state)))
        lam_pl.append([_lam(orc.elements(gi.G * (1.0 + planets[j, 0]), planets[j:j + 1, 1:])[0]) for j in (2, 3)])
    assert np.all(run.removal_step < 0)
    t = np.arange(1, n_samples + 1) * every * dt
    # Uranus and Neptune move by at most 0.12 of a turn between samples, the particles less
    n_p = np.polyfit(t, np.unwrap(np.array(lam_p), axis=0), 1)[0]
    n_pl = np.polyfit(t, np.unwrap(np.array(lam_pl), axis=0), 1)[0]
    for k, (planet, m, n, _) in enumerate(res):
        ratio = n_p[k] / n_pl[PLANET_INDEX[planet] - 2]
        nominal = int(m) / int(n)
        # where the ratio would be exactly m/n, by Kepler's third law about the particle's own orbit
        a_exact = a0[k] * (ratio / nominal) ** (2.0 / 3.0)
        assert abs(a_exact - a0[k]) <= variation, (planet, m, n, a_exact)


def test_three_to_one_resonance_at_the_printed_centre(orc):
    v = pins.paper_values("resonance_3_1")
    j = PLANET_INDEX[v["planet"]]
    m, n = int(v["m"]), int(v["n"])
    centre, width = float(v["centre"]), float(v["width"])
    box = (float(v["box_min"]), float(v["box_max"]))
    w = gi.make("tiny", n=1)
    planets = w["planets"]
    pm = planets[:, 0]
    mt = 1.0 + pm.sum()
    # the paper's elements are barycentric: start the particles from barycentric elements
    R = orc.barycentre(1.0, pm, planets[:, 1:])
    el_pl = orc.elements(gi.G * mt, (planets[j, 1:] - R)[None])[0]
    lam_pl = _lam(el_pl)
    step = 0.1
    a_scan = np.round(np.arange(centre - 1.6, centre + 1.6 + step / 2, step), 6)
    rng = np.random.default_rng(1)
    rows = []
    for a in a_scan:
        varpi = rng.uniform(0.0, 2 * np.pi)
        node = rng.uniform(0.0, 2 * np.pi)
        lam = (np.pi + n * lam_pl + (m - n) * varpi) / m  # phi = m lam - n lam_N - (m - n) varpi = 180 deg
        rows.append(gi.elements_to_cartesian(gi.G * mt, a, 0.4, np.radians(5.0), node, varpi - node, lam - varpi) + R)
    # 4e4 yr sampled every 5 yr: outside the resonance phi turns by < 1 deg per sample
    out = orc.run_sampled(1.0, planets, np.array(rows), 0.5, 80000, 10, frame=1, res_planet=j, res_p=m, res_q=n,
                          avoid_deg=float(v["window_deg"]))
    assert np.all(out["removal_step"] < 0)
    assert np.all(out["count"] == 8000)
    librating = (out["near0"] == 0) | (out["near180"] == 0)
    inside = a_scan[librating]
    assert inside.size > 0
    lo, hi = inside.min(), inside.max()
    # one interval, containing the printed centre, no wider than the printed width, within the printed box
    assert np.all(librating[(a_scan >= lo) & (a_scan <= hi)]), a_scan[librating]
    assert lo <= centre <= hi, (lo, hi)
    assert hi - lo <= width + step / 2, (lo, hi)
    assert box[0] <= lo and hi <= box[1], (lo, hi)
    # and circulation on both sides
    assert (~librating[a_scan < lo]).all() and (a_scan < lo).any()
    assert (~librating[a_scan > hi]).all() and (a_scan > hi).any()
