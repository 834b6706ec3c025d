"""Independent references that pin the oracle (and, through parity, the CUDA path).

Nothing here imports the oracle's arithmetic: each reference is derived from
the mathematics directly.

* ``analytic_state``: the exact two-body orbit in mpmath (40 digits) from
  classical elements, Kepler's equation solved to full precision.
* ``nbody_reference``: the full heliocentric N-body equations of motion of the
  star, planets and massless particles integrated by scipy's DOP853 at tight
  tolerance (a library integrator used as one step of the reference).
* ``jacobi_constant``: the Jacobi integral of the circular restricted
  three-body problem in the rotating barycentric frame.
* ``paper_values``: the numbers the paper prints (``tests/golden/paper_values.txt``,
  each section with the passage it comes from).
"""
from __future__ import annotations

import math
import os

import numpy as np

G = 4.0 * math.pi * math.pi


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_values(section: str) -> dict:
    """One section of ``golden/paper_values.txt`` as a dict of strings."""
    import configparser

    cp = configparser.ConfigParser(inline_comment_prefixes=("#",))
    with open(os.path.join(GOLDEN, "paper_values.txt")) as fh:
        cp.read_file(fh)
    return dict(cp[section])


def _mp():
    import pytest

    return pytest.importorskip("mpmath")


def analytic_state(mu, a, e, inc, node, peri, M, dps=40, as_mp=False):
    """Cartesian state [6] (float64, or mpmath numbers with as_mp) of a two-body orbit; hyperbolic
    orbits take a = |a| and e > 1, with M the hyperbolic mean anomaly e sinh F - F."""
    mp = _mp()
    with mp.workdps(dps):
        mu, a, e, inc, node, peri, M = (mp.mpf(v) for v in (mu, a, e, inc, node, peri, M))
        n = mp.sqrt(mu / a**3)
        if e < 1:
            Mr = M - 2 * mp.pi * mp.floor(M / (2 * mp.pi))
            E = mp.findroot(lambda E: E - e * mp.sin(E) - Mr, (Mr - e - mp.mpf("1e-30"), Mr + e + mp.mpf("1e-30")),
                            solver="anderson")
            den = 1 - e * mp.cos(E)
            b = mp.sqrt(1 - e * e)
            xo, yo = a * (mp.cos(E) - e), a * b * mp.sin(E)
            vxo, vyo = -n * a * mp.sin(E) / den, n * a * b * mp.cos(E) / den
        else:
            # bracket: e sinh F - F >= e F^3 / 6 for F >= 0, so the root lies in [0, (6|M|/e)^(1/3)]
            if M == 0:
                Fh = mp.mpf(0)
            else:
                hi = mp.cbrt(6 * abs(M) / e) * (1 + mp.mpf("1e-30"))
                sg = 1 if M > 0 else -1
                Fh = sg * mp.findroot(lambda F: e * mp.sinh(F) - F - abs(M), (mp.mpf(0), hi), solver="anderson")
            den = e * mp.cosh(Fh) - 1
            b = mp.sqrt(e * e - 1)
            xo, yo = a * (e - mp.cosh(Fh)), a * b * mp.sinh(Fh)
            vxo, vyo = -n * a * mp.sinh(Fh) / den, n * a * b * mp.cosh(Fh) / den
        cO, sO, cw, sw, ci, si = mp.cos(node), mp.sin(node), mp.cos(peri), mp.sin(peri), mp.cos(inc), mp.sin(inc)
        p11 = cO * cw - sO * sw * ci
        p12 = -cO * sw - sO * cw * ci
        p21 = sO * cw + cO * sw * ci
        p22 = -sO * sw + cO * cw * ci
        p31 = sw * si
        p32 = cw * si
        out = [p11 * xo + p12 * yo, p21 * xo + p22 * yo, p31 * xo + p32 * yo,
               p11 * vxo + p12 * vyo, p21 * vxo + p22 * vyo, p31 * vxo + p32 * vyo]
        if as_mp:
            return out
        return np.array([float(v) for v in out])


def state_to_elements(mu, state, dps=40):
    """Classical elements (|a|, e, inc, node, peri, M) of a Cartesian state, computed in mpmath.

    The state is taken as exact (its double values), so the analytic reference
    starts from precisely the input the integrator sees.  Needs inc > 0."""
    mp = _mp()
    with mp.workdps(dps):
        r = [x if isinstance(x, mp.mpf) else mp.mpf(float(x)) for x in state[:3]]
        v = [x if isinstance(x, mp.mpf) else mp.mpf(float(x)) for x in state[3:6]]
        mu = mp.mpf(mu)

        def cross(p, q):
            return [p[1] * q[2] - p[2] * q[1], p[2] * q[0] - p[0] * q[2], p[0] * q[1] - p[1] * q[0]]

        def dot(p, q):
            return p[0] * q[0] + p[1] * q[1] + p[2] * q[2]

        rn = mp.sqrt(dot(r, r))
        h = cross(r, v)
        hn = mp.sqrt(dot(h, h))
        hu = [x / hn for x in h]
        inc = mp.acos(h[2] / hn)
        nv = [-h[1], h[0], mp.mpf(0)]
        vxh = cross(v, h)
        ev = [vxh[i] / mu - r[i] / rn for i in range(3)]
        e = mp.sqrt(dot(ev, ev))
        energy = dot(v, v) / 2 - mu / rn
        a = -mu / (2 * energy)
        node = mp.atan2(nv[1], nv[0])
        peri = mp.atan2(dot(cross(nv, ev), hu), dot(nv, ev))
        nu = mp.atan2(dot(cross(ev, r), hu), dot(ev, r))
        if e < 1:
            E = 2 * mp.atan(mp.sqrt((1 - e) / (1 + e)) * mp.tan(nu / 2))
            M = E - e * mp.sin(E)
        else:
            F = 2 * mp.atanh(mp.sqrt((e - 1) / (e + 1)) * mp.tan(nu / 2))
            M = e * mp.sinh(F) - F
        return (abs(a), e, inc, node, peri, M)


def propagate_exact(mu, state, dt, dps=40):
    """Exact two-body propagation of a double state by dt (elements route, mpmath)."""
    mp = _mp()
    with mp.workdps(dps):
        a, e, inc, node, peri, M = state_to_elements(mu, state, dps)
        n = mp.sqrt(mp.mpf(mu) / a**3)
        return analytic_state(mu, a, e, inc, node, peri, M + n * mp.mpf(dt), dps)


def propagate_exact_mp(mu, state, dt, dps=60):
    """propagate_exact for a state of mpmath numbers (or doubles), returning mpmath numbers."""
    mp = _mp()
    with mp.workdps(dps):
        a, e, inc, node, peri, M = state_to_elements(mu, state, dps)
        n = mp.sqrt(mp.mpf(mu) / a**3)
        return analytic_state(mu, a, e, inc, node, peri, M + n * mp.mpf(dt), dps, as_mp=True)


def condition(mu, state, dt):
    """Rough FP64 condition number of a two-body propagation: the kinetic-to-binding energy ratio
    (cancellation in the energy) times the number of radians of mean motion covered."""
    r = float(np.linalg.norm(state[:3]))
    v2 = float(np.dot(state[3:6], state[3:6]))
    energy = abs(0.5 * v2 - mu / r)
    a = mu / (2 * energy)
    n = math.sqrt(mu / a**3)
    return (0.5 * v2 / energy) * (1.0 + abs(n * dt))


def mean_motion(mu, a):
    return math.sqrt(mu / abs(a) ** 3)


def rel_err(x, ref):
    """max(|dr|/|r|, |dv|/|v|) for states [..., 6]."""
    x = np.asarray(x).reshape(-1, 6)
    ref = np.asarray(ref).reshape(-1, 6)
    er = np.linalg.norm(x[:, :3] - ref[:, :3], axis=1) / np.linalg.norm(ref[:, :3], axis=1)
    ev = np.linalg.norm(x[:, 3:] - ref[:, 3:], axis=1) / np.linalg.norm(ref[:, 3:], axis=1)
    return np.maximum(er, ev)


def nbody_reference(m0, planets, particles, t_end, rtol=1e-13, atol=1e-14):
    """Heliocentric N-body integration of planets (massive) and particles (massless) to t_end.

    Equations of motion (heliocentric, star at the origin):
      planet i:  r_i'' = -G (m0 + m_i) r_i/|r_i|^3 - sum_{j!=i} G m_j [ (r_i - r_j)/|r_i - r_j|^3 + r_j/|r_j|^3 ]
      particle:  r''   = -G m0 r/|r|^3 - sum_j G m_j [ (r - r_j)/|r - r_j|^3 + r_j/|r_j|^3 ]
    Returns (planets_out [np][7], particles_out [n][6])."""
    import pytest

    integrate = pytest.importorskip("scipy.integrate")
    pl = np.asarray(planets, dtype=np.float64)
    pa = np.asarray(particles, dtype=np.float64).reshape(-1, 6)
    m = pl[:, 0]
    npl, npa = len(m), len(pa)
    Gm = G * m

    def rhs(_t, y):
        Y = y.reshape(-1, 6)
        r = Y[:, :3]
        v = Y[:, 3:]
        rp = r[:npl]
        rp3 = np.linalg.norm(rp, axis=1) ** 3
        ind = -(Gm[:, None] * rp / rp3[:, None]).sum(axis=0)  # indirect acceleration of the star's frame
        acc = np.empty_like(r)
        rn3 = np.linalg.norm(r, axis=1) ** 3
        acc[:npl] = -G * (m0 + m)[:, None] * r[:npl] / rn3[:npl, None]
        acc[npl:] = -G * m0 * r[npl:] / rn3[npl:, None]
        for j in range(npl):
            d = r - rp[j]
            d3 = np.linalg.norm(d, axis=1) ** 3
            d3[j] = np.inf  # a planet does not pull itself
            acc -= Gm[j] * d / d3[:, None]
        # indirect term: every body feels -sum_j G m_j r_j/|r_j|^3 except planet j's own term
        acc += ind
        for j in range(npl):
            acc[j] += Gm[j] * rp[j] / rp3[j]
        return np.concatenate([v, acc], axis=1).ravel()

    y0 = np.concatenate([pl[:, 1:7], pa], axis=0).ravel()
    sol = integrate.solve_ivp(rhs, (0.0, t_end), y0, method="DOP853", rtol=rtol, atol=atol)
    assert sol.success
    Y = sol.y[:, -1].reshape(-1, 6)
    plo = np.concatenate([m[:, None], Y[:npl]], axis=1)
    return plo, Y[npl:]


def jacobi_constant(m0, m1, a1, t, r1, v1, state):
    """Jacobi integral E_J = E - n L_z of a massless particle in the circular restricted problem.

    Inputs are heliocentric: planet position r1 and velocity v1 at time t, particle state [..., 6].
    The barycentre sits at R = m1 r1 / (m0 + m1); n = sqrt(G (m0 + m1) / a1^3)."""
    s = np.asarray(state).reshape(-1, 6)
    M = m0 + m1
    n = math.sqrt(G * M / a1**3)
    R = m1 * np.asarray(r1) / M
    V = m1 * np.asarray(v1) / M
    rb = s[:, :3] - R
    vb = s[:, 3:] - V
    star_b = -R
    pl_b = np.asarray(r1) - R
    d0 = np.linalg.norm(rb - star_b, axis=1)
    d1 = np.linalg.norm(rb - pl_b, axis=1)
    E = 0.5 * (vb**2).sum(axis=1) - G * m0 / d0 - G * m1 / d1
    Lz = rb[:, 0] * vb[:, 1] - rb[:, 1] * vb[:, 0]
    return E - n * Lz


def circular_planet(m0, m1, a1, t, phase=0.0):
    """Heliocentric position and velocity of a planet on a circular orbit of radius a1 in the xy plane."""
    n = math.sqrt(G * (m0 + m1) / a1**3)
    th = n * np.asarray(t) + phase
    r = np.stack([a1 * np.cos(th), a1 * np.sin(th), np.zeros_like(th)], axis=-1)
    v = np.stack([-a1 * n * np.sin(th), a1 * n * np.cos(th), np.zeros_like(th)], axis=-1)
    return r, v
