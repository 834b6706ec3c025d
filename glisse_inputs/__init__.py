"""Seeded synthetic workloads for the GLISSE test-particle map.

This module is the one thing the CUDA path and the CPU oracle share: it draws
initial conditions and nothing else.  It holds none of the map's arithmetic
(no kick, drift, removal test or planet integrator); the orbital-element to
Cartesian conversion below only places bodies on their starting orbits.

Workload shapes follow the paper's experiments (section 3: belts of test
particles between and beyond the giant planets, drawn uniformly in a, e and
with small inclinations) and the synthetic configurations used to measure
this implementation:

  tiny      1024 particles, a in U[21, 28] AU, e in U[0, 0.05], sigma_i = 1 deg,
            dt = 0.5 yr, 1e4 steps, seed 0 (parity workload)
  longrun   131072 particles, a in U[20, 29], e in U[0, 0.1], sigma_i = 2 deg,
            2e6 steps in chunks of 1024, seed 1 (headline throughput)
  belt      1048576 particles, a in U[40, 50], e in U[0, 0.4], sigma_i = 5 deg,
            1e6 steps, seed 2 (resonant belt, frequent removal)
  diff      65536 particles, a in U[22, 28], e in U[0, 0.05], sigma_i = 1 deg,
            1e4 steps, seed 3
  eccentric 131072 particles, a in U[20, 29], e in U[0, 0.9], sigma_i = 2 deg,
            seed 5 (mixed solve costs: the sorting option's workload)

All share the 4-planet system below: star of 1 M_sun; planets at
a = 5.2, 9.55, 19.2, 30.1 AU with m = 9.5e-4, 2.9e-4, 4.4e-5, 5.2e-5 M_sun,
near-circular, near-coplanar (e, i fixed close to the real giants), and
Omega, omega, M drawn from the seeded generator.

Random draw order (numpy PCG64(seed)): for each planet in index order its
Omega, omega, M; then the particle arrays a, e, i, Omega, omega, M, each drawn
vectorised over all N.  Inclinations are Rayleigh: i = sigma sqrt(-2 ln(1-U)).
Units: AU, yr, M_sun, G = 4 pi^2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

G = 4.0 * math.pi * math.pi

PLANET_A = (5.2, 9.55, 19.2, 30.1)
PLANET_M = (9.5e-4, 2.9e-4, 4.4e-5, 5.2e-5)
PLANET_E = (0.048, 0.054, 0.047, 0.009)
PLANET_I_DEG = (1.3, 2.5, 0.8, 1.8)


@dataclass
class Workload:
    name: str
    n: int
    a_range: tuple
    e_range: tuple
    sigma_i_deg: float
    dt: float
    n_steps: int
    seed: int
    chunk: int = 1024
    resync: int = 1
    k_hill: float = 1.0
    r_max: float = 1000.0
    star_mass: float = 1.0
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    "tiny": Workload("tiny", 1024, (21.0, 28.0), (0.0, 0.05), 1.0, 0.5, 10_000, 0),
    "longrun": Workload("longrun", 131072, (20.0, 29.0), (0.0, 0.1), 2.0, 0.5, 2_000_000, 1),
    "belt": Workload("belt", 1048576, (40.0, 50.0), (0.0, 0.4), 5.0, 0.5, 1_000_000, 2),
    "diff": Workload("diff", 65536, (22.0, 28.0), (0.0, 0.05), 1.0, 0.5, 10_000, 3),
    "eccentric": Workload("eccentric", 131072, (20.0, 29.0), (0.0, 0.9), 2.0, 0.5, 2_000_000, 5),
}


def solve_kepler_mean_to_eccentric(M, e):
    """E with E - e sin E = M for 0 <= e < 1 (vectorised Newton, fixed 40 iterations)."""
    M = np.asarray(M, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    E = np.where(e < 0.8, M, np.pi * np.ones_like(M))
    for _ in range(40):
        E = E - (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
    return E


def elements_to_cartesian(mu, a, e, inc, node, peri, mean_anom):
    """Heliocentric Cartesian state [..., 6] from elliptic elements (angles in radians)."""
    a, e, inc, node, peri, mean_anom = (np.asarray(v, dtype=np.float64) for v in (a, e, inc, node, peri, mean_anom))
    mu = np.asarray(mu, dtype=np.float64)
    E = solve_kepler_mean_to_eccentric(np.mod(mean_anom, 2 * np.pi), e)
    cE, sE = np.cos(E), np.sin(E)
    b = np.sqrt(1.0 - e * e)
    n = np.sqrt(mu / a**3)
    xo = a * (cE - e)
    yo = a * b * sE
    den = 1.0 - e * cE
    vxo = -n * a * sE / den
    vyo = n * a * b * cE / den
    cO, sO = np.cos(node), np.sin(node)
    cw, sw = np.cos(peri), np.sin(peri)
    ci, si = np.cos(inc), np.sin(inc)
    # rotation Rz(node) Rx(inc) Rz(peri)
    p11 = cO * cw - sO * sw * ci
    p12 = -cO * sw - sO * cw * ci
    p21 = sO * cw + cO * sw * ci
    p22 = -sO * sw + cO * cw * ci
    p31 = sw * si
    p32 = cw * si
    x = p11 * xo + p12 * yo
    y = p21 * xo + p22 * yo
    z = p31 * xo + p32 * yo
    vx = p11 * vxo + p12 * vyo
    vy = p21 * vxo + p22 * vyo
    vz = p31 * vxo + p32 * vyo
    return np.stack([x, y, z, vx, vy, vz], axis=-1)


def planet_system(rng: np.random.Generator, star_mass: float = 1.0):
    """[4][7] heliocentric (m, x, y, z, vx, vy, vz) of the 4-planet system."""
    rows = []
    for j in range(4):
        node = rng.uniform(0.0, 2 * np.pi)
        peri = rng.uniform(0.0, 2 * np.pi)
        mean = rng.uniform(0.0, 2 * np.pi)
        mu = G * (star_mass + PLANET_M[j])
        st = elements_to_cartesian(mu, PLANET_A[j], PLANET_E[j], math.radians(PLANET_I_DEG[j]), node, peri, mean)
        rows.append(np.concatenate([[PLANET_M[j]], st]))
    return np.array(rows, dtype=np.float64)


def particle_belt(rng: np.random.Generator, n: int, a_range, e_range, sigma_i_deg: float, star_mass: float = 1.0):
    """[n][6] heliocentric particle states drawn as documented in the module docstring."""
    a = rng.uniform(a_range[0], a_range[1], n)
    e = rng.uniform(e_range[0], e_range[1], n)
    u = rng.uniform(0.0, 1.0, n)
    inc = math.radians(sigma_i_deg) * np.sqrt(-2.0 * np.log1p(-u))
    node = rng.uniform(0.0, 2 * np.pi, n)
    peri = rng.uniform(0.0, 2 * np.pi, n)
    mean = rng.uniform(0.0, 2 * np.pi, n)
    return elements_to_cartesian(G * star_mass, a, e, inc, node, peri, mean)


def make(name: str, n: int | None = None):
    """Build a workload by name.  ``n`` truncates the particle set to its first n
    ids (the generator still draws the full set so ids are stable)."""
    w = WORKLOADS[name]
    rng = np.random.Generator(np.random.PCG64(w.seed))
    planets = planet_system(rng, w.star_mass)
    particles = particle_belt(rng, w.n, w.a_range, w.e_range, w.sigma_i_deg, w.star_mass)
    if n is not None:
        particles = particles[:n]
    return {
        "workload": w,
        "star_mass": w.star_mass,
        "planets": np.ascontiguousarray(planets),
        "particles": np.ascontiguousarray(particles),
        "dt": w.dt,
    }


def make_batched(seed: int = 4, n_systems: int = 256, n_min: int = 512, n_max: int = 65536, star_mass: float = 1.0):
    """Many independent systems (the batched workload).

    Per system, drawn in this order from PCG64(seed): the planet count N_p
    uniform in {2..8}; planet masses log-uniform in [1e-5, 1e-3] M_sun; the
    innermost semi-major axis uniform in [1, 5] AU, each next one at least 10
    mutual Hill radii further out (a_{i+1} = a_i (1 + 5k)/(1 - 5k) (1 + U[0, 0.3]),
    k = ((m_i + m_{i+1}) / 3 m0)^(1/3)); e in U[0, 0.05], i in U[0, 2] deg and
    uniform angles for each planet; then the particle count log-uniform in
    [n_min, n_max]; particles half between the two outermost planets (10% of
    the gap kept clear at each end) and half beyond the outermost one
    (a in U[1.2, 1.6] a_out), e in U[0, 0.05], Rayleigh sigma_i = 1 deg.
    dt is 1/20 of the innermost planet's period.  With the defaults about 4e6
    particles in all.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {"star_mass": [], "n_planets": [], "planets": [], "n_particles": [], "particles": [], "dt": []}
    for _ in range(n_systems):
        npl = int(rng.integers(2, 9))
        m = np.exp(rng.uniform(np.log(1e-5), np.log(1e-3), npl))
        a = np.empty(npl)
        a[0] = rng.uniform(1.0, 5.0)
        for i in range(npl - 1):
            k = ((m[i] + m[i + 1]) / (3.0 * star_mass)) ** (1.0 / 3.0)
            a[i + 1] = a[i] * (1 + 5 * k) / (1 - 5 * k) * (1.0 + rng.uniform(0.0, 0.3))
        e = rng.uniform(0.0, 0.05, npl)
        inc = np.radians(rng.uniform(0.0, 2.0, npl))
        ang = rng.uniform(0.0, 2 * np.pi, (3, npl))
        st = elements_to_cartesian(G * (star_mass + m), a, e, inc, ang[0], ang[1], ang[2])
        planets = np.concatenate([m[:, None], st], axis=1)
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        between = rng.uniform(0.0, 1.0, n) < 0.5
        gap = a[-1] - a[-2]
        pa = np.where(between, rng.uniform(a[-2] + 0.1 * gap, a[-1] - 0.1 * gap, n),
                      a[-1] * rng.uniform(1.2, 1.6, n))
        pe = rng.uniform(0.0, 0.05, n)
        u = rng.uniform(0.0, 1.0, n)
        pinc = np.radians(1.0) * np.sqrt(-2.0 * np.log1p(-u))
        pang = rng.uniform(0.0, 2 * np.pi, (3, n))
        parts = elements_to_cartesian(G * star_mass, pa, pe, pinc, pang[0], pang[1], pang[2])
        period = 2 * np.pi * np.sqrt(a[0] ** 3 / (G * (star_mass + m[0])))
        out["star_mass"].append(star_mass)
        out["n_planets"].append(npl)
        out["planets"].append(planets)
        out["n_particles"].append(n)
        out["particles"].append(parts)
        out["dt"].append(period / 20.0)
    return {
        "star_mass": np.array(out["star_mass"]),
        "n_planets": np.array(out["n_planets"], dtype=np.int32),
        "planets": np.ascontiguousarray(np.concatenate(out["planets"], axis=0)),
        "n_particles": np.array(out["n_particles"], dtype=np.int64),
        "particles": np.ascontiguousarray(np.concatenate(out["particles"], axis=0)),
        "dt": np.array(out["dt"]),
    }


def subset_ids(name: str, k: int):
    """Sorted random subset of k particle ids of a workload (seeded by the workload)."""
    w = WORKLOADS[name]
    rng = np.random.Generator(np.random.PCG64(10_000 + w.seed))
    return np.sort(rng.choice(w.n, size=min(k, w.n), replace=False))
