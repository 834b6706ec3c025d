"""Pins of the CPU oracle against the mathematics (no GPU).

Each test checks the oracle against something it does not contain: the exact
two-body orbit (mpmath), exact time reversibility of a symmetric map, the
Jacobi integral of the circular restricted problem, the full N-body equations
integrated by a library integrator, and special cases with known outcomes.
The planted-mistake tests in test_oracle_mutants.py show each class of
mistake is caught by at least one of these.
"""
import math

import numpy as np
import pytest

import pins
from pins import G

M0 = 1.0


# --------------------------------------------------------------------------
# 1. Two-body closed form (the drift, paper section 2.2 Kepler-equation step)
# --------------------------------------------------------------------------
ELEMENTS = [
    # (a, e, inc, node, peri, M0)
    (25.0, 0.0, 0.3, 1.1, 2.2, 0.7),
    (25.0, 0.05, 0.3, 1.1, 2.2, 0.7),
    (25.0, 0.4, 0.3, 1.1, 2.2, 2.9),
    (25.0, 0.9, 0.3, 1.1, 2.2, 0.2),
    (25.0, 0.9995, 0.1, 0.4, 0.5, 0.0),   # at pericentre, nearly radial: universal-variable branch
    (25.0, 1.5, 0.3, 1.1, 2.2, 0.3),      # hyperbolic
    (40.0, 1.0001, 0.2, 0.3, 0.1, 0.01),  # barely hyperbolic
]


def two_body_one_step(orc, elems, dt):
    a, e, inc, node, peri, Mi = elems
    mu = G * M0
    s0 = pins.analytic_state(mu, a, e, inc, node, peri, Mi)
    ref = pins.propagate_exact(mu, s0, dt)
    out, rc, _ = orc.kepler_drift(mu, s0, dt)
    assert rc == 0
    return float(pins.rel_err(out, ref)[0]), pins.condition(mu, s0, dt)


@pytest.mark.parametrize("elems", ELEMENTS)
@pytest.mark.parametrize("dt", [0.5, -0.5, 7.3, 300.0, -1234.5])
def test_two_body_single_drift(orc, elems, dt):
    """One drift equals the exact orbit of the same double state to 1e-14 x the FP64 condition
    number (energy cancellation x radians of mean motion): any e, either sign of dt, dt > period."""
    err, cond = two_body_one_step(orc, elems, dt)
    assert err < 1e-14 * max(cond, 1.0) + 1e-15, (err, cond)


JUPITER_LIKE = (5.2, 0.048, 0.02, 0.3, 0.4, 0.5)


@pytest.mark.parametrize("elems", [ELEMENTS[1], ELEMENTS[2], ELEMENTS[5], JUPITER_LIKE])
def test_two_body_many_steps(orc, elems):
    """10^4 steps of the map with no planets follow the exact orbit within FP64's phase random walk.

    Rounding the stored state every step moves the orbital energy by a few ulp
    at random, so the mean-longitude error after n steps grows like
    eps * dM * n^(3/2) (dM = mean motion x dt).  The bound allows 10 ulp of
    energy noise per step.  A drift that converges short of the root on one
    side shifts the energy by the same sign every step: the error then grows
    like n^2 and the energy trend test below fails."""
    a, e, inc, node, peri, Mi = elems
    mu = G * M0
    dt, n_steps = 0.5, 10_000
    s0 = pins.analytic_state(mu, a, e, inc, node, peri, Mi)
    run = orc.ParticleRun(M0, np.zeros(0), s0[None, :], np.zeros(0), 0.0)
    run.advance(np.zeros((n_steps + 1, 0, 3)), dt)
    ref = pins.propagate_exact(mu, s0, dt * n_steps)
    err = float(pins.rel_err(run.state, ref)[0])
    assert run.removal_step[0] == -1
    dM = pins.mean_motion(mu, a) * dt
    tol = 10 * 2.0**-53 * dM * n_steps**1.5
    assert err < tol, (err, tol)


@pytest.mark.parametrize("elems", [JUPITER_LIKE, ELEMENTS[2], ELEMENTS[5]])
def test_two_body_no_secular_energy_drift(orc, elems):
    """The orbital energy along 10^4 drifts has no trend above 1e-17 per step (unbiased rounding
    gives ~1e-18; a one-sided convergence error gives ~1e-16)."""
    mu = G * M0
    st = pins.analytic_state(mu, *elems)
    energies = []
    for _ in range(50):
        run = orc.ParticleRun(M0, np.zeros(0), st[None, :], np.zeros(0), 0.0)
        run.advance(np.zeros((201, 0, 3)), 0.5)
        st = run.state[0]
        energies.append(0.5 * np.dot(st[3:], st[3:]) - mu / np.linalg.norm(st[:3]))
    en = np.array(energies)
    slope = np.polyfit(np.arange(len(en)) * 200.0, en / abs(en[0]), 1)[0]
    assert abs(slope) < 1e-17, slope


def test_drift_zero_dt_is_identity(orc):
    s0 = pins.analytic_state(G, 25.0, 0.2, 0.1, 0.2, 0.3, 1.0)
    out, rc, _ = orc.kepler_drift(G, s0, 0.0)
    assert rc == 0
    np.testing.assert_allclose(out, s0, rtol=1e-15, atol=0)


# --------------------------------------------------------------------------
# 2. Time reversibility of the symmetric kick-drift-kick map
# --------------------------------------------------------------------------
def _far_particles(k=8, seed=5):
    rng = np.random.default_rng(seed)
    import glisse_inputs as gi

    a = rng.uniform(36.0, 42.0, k)
    e = rng.uniform(0.0, 0.03, k)
    inc = np.radians(rng.uniform(0.0, 3.0, k))
    ang = rng.uniform(0, 2 * np.pi, (3, k))
    return gi.elements_to_cartesian(G * M0, a, e, inc, ang[0], ang[1], ang[2])


def _planets():
    import glisse_inputs as gi

    return gi.make("tiny")["planets"]


@pytest.mark.parametrize("n", [1000, 10_000])
def test_reversibility_particles(orc, n):
    """Forward n steps then back with -dt over the reversed planet log returns the start state.

    Rounding is not undone by the reverse map, so the residue follows the same
    FP64 phase random walk as the two-body test (eps dM (2n)^1.5, 20 ulp of
    energy noise per step); a one-sided or asymmetric step misses by orders."""
    pl = _planets()
    dt = 0.5
    _, log, _ = orc.planet_wh(M0, pl, dt, n)
    p0 = _far_particles()
    run = orc.ParticleRun(M0, pl[:, 0], p0, np.zeros(4), 0.0)
    run.advance(log, dt)
    moved = float(pins.rel_err(run.state, p0).min())
    run.advance(log[::-1], -dt)
    err = float(pins.rel_err(run.state, p0).max())
    assert moved > 1e-3
    dM = pins.mean_motion(G * M0, 36.0) * dt
    tol = 20 * 2.0**-53 * dM * (2 * n) ** 1.5
    assert err < tol, (err, tol)


@pytest.mark.parametrize("n", [1000, 10_000])
def test_reversibility_planets(orc, n):
    pl = _planets()
    dt = 0.5
    pl1, _, _ = orc.planet_wh(M0, pl, dt, n, want_log=False)
    pl2, _, _ = orc.planet_wh(M0, pl1, -dt, n, want_log=False)
    err = float(pins.rel_err(pl2[:, 1:], pl[:, 1:]).max())
    dM = pins.mean_motion(G * M0, 5.2) * dt
    tol = 20 * 2.0**-53 * dM * (2 * n) ** 1.5
    assert err < tol, (err, tol)


# --------------------------------------------------------------------------
# 3. Jacobi constant of the circular restricted three-body problem
# --------------------------------------------------------------------------
def _cr3bp_run(orc, dt, n_steps, k=4):
    m1, a1 = 1e-3, 5.2
    t = np.arange(n_steps + 1) * dt
    r1, v1 = pins.circular_planet(M0, m1, a1, t)
    import glisse_inputs as gi

    # particles outside the planet on near-circular orbits (regular region)
    a = np.linspace(8.0, 9.5, k)
    st0 = gi.elements_to_cartesian(G * M0, a, np.full(k, 0.02), np.zeros(k), np.zeros(k), np.linspace(0, 3, k),
                                   np.linspace(0.5, 5, k))
    run = orc.ParticleRun(M0, np.array([m1]), st0, np.zeros(1), 0.0)
    samples = []
    every = max(1, n_steps // 400)
    for c in range(0, n_steps, every):
        cj = pins.jacobi_constant(M0, m1, a1, t[c], r1[c], v1[c], run.state)
        samples.append((t[c], cj))
        run.advance(r1[c:c + every + 1][:, None, :], dt)
    cj = pins.jacobi_constant(M0, m1, a1, t[n_steps], r1[n_steps], v1[n_steps], run.state)
    samples.append((t[n_steps], cj))
    ts = np.array([s[0] for s in samples])
    cjs = np.array([s[1] for s in samples])
    return ts, cjs


def test_jacobi_constant_cr3bp(orc):
    """E_J error stays bounded (no secular drift) over 10^5 steps and scales as dt^2."""
    ts, cj = _cr3bp_run(orc, 0.5, 100_000)
    rel = (cj - cj[0]) / np.abs(cj[0])
    amp = np.abs(rel).max(axis=0)
    for j in range(rel.shape[1]):
        slope = np.polyfit(ts, rel[:, j], 1)[0]
        drift = abs(slope) * (ts[-1] - ts[0])
        assert drift < 0.5 * amp[j] + 1e-13, (j, drift, amp[j])
    assert amp.max() < 1e-4  # ~ (m1/m0) (2 pi dt / P)^2 for these orbits
    ts2, cj2 = _cr3bp_run(orc, 0.25, 200_000)
    amp2 = np.abs((cj2 - cj2[0]) / np.abs(cj2[0])).max(axis=0)
    ratio = amp / amp2
    assert np.all((ratio > 3.2) & (ratio < 4.8)), ratio


# --------------------------------------------------------------------------
# 4. Brute force: full N-body equations (library integrator) vs the map
# --------------------------------------------------------------------------
def _brute_errors(orc, dts, t_end=100.0):
    pl = _planets()
    rng = np.random.default_rng(11)
    import glisse_inputs as gi

    k = 8
    a = np.concatenate([rng.uniform(36, 44, k - 2), [23.0, 25.5]])
    e = rng.uniform(0.0, 0.05, k)
    inc = np.radians(rng.uniform(0, 4, k))
    ang = rng.uniform(0, 2 * np.pi, (3, k))
    p0 = gi.elements_to_cartesian(G * M0, a, e, inc, ang[0], ang[1], ang[2])
    pl_ref, pa_ref = pins.nbody_reference(M0, pl, p0, t_end)
    out = []
    for dt in dts:
        n = int(round(t_end / dt))
        pl1, log, _ = orc.planet_wh(M0, pl, dt, n)
        run = orc.ParticleRun(M0, pl[:, 0], p0, np.zeros(4), 0.0)
        run.advance(log, dt)
        ep = np.abs(pl1[:, 1:4] - pl_ref[:, 1:4]).max()
        ea = np.abs(run.state[:, :3] - pa_ref[:, :3]).max()
        out.append((ep, ea))
    return np.array(out)


@pytest.mark.slow
def test_brute_force_second_order(orc):
    """The map's error against the exact N-body solution at t = 100 yr falls as dt^2."""
    errs = _brute_errors(orc, [0.5, 0.25, 0.125])
    for col in range(2):
        e = errs[:, col]
        orders = np.log2(e[:-1] / e[1:])
        assert np.all((orders > 1.8) & (orders < 2.2)), (col, e, orders)
    assert errs[0].max() < 2e-2  # AU at dt = 0.5 yr; the order test above is the pin


# --------------------------------------------------------------------------
# 5. Planet energy: bounded, no secular drift, error ~ dt^2
# --------------------------------------------------------------------------
def test_planet_energy(orc):
    pl = _planets()

    def amp(dt, n):
        _, _, en = orc.planet_wh(M0, pl, dt, n, want_log=False, want_energy=True)
        rel = (en - en[0]) / abs(en[0])
        t = np.arange(n + 1) * dt
        slope = np.polyfit(t[::50], rel[::50], 1)[0]
        return np.abs(rel).max(), abs(slope) * t[-1]

    a1, d1 = amp(0.5, 100_000)
    a2, d2 = amp(0.25, 200_000)
    assert a1 < 1e-5
    assert d1 < 0.5 * a1 and d2 < 0.5 * a2
    assert 3.2 < a1 / a2 < 4.8, (a1, a2)


def _barycentric_angular_momentum(m0, pl):
    """Total angular momentum about the barycentre of the star (at the heliocentric origin,
    at rest there) and planets [np][7] (m, heliocentric position and velocity)."""
    m = np.concatenate([[m0], pl[:, 0]])
    r = np.vstack([np.zeros(3), pl[:, 1:4]])
    v = np.vstack([np.zeros(3), pl[:, 4:7]])
    R = (m[:, None] * r).sum(axis=0) / m.sum()
    V = (m[:, None] * v).sum(axis=0) / m.sum()
    return (m[:, None] * np.cross(r - R, v - V)).sum(axis=0)


def test_planet_angular_momentum(orc):
    """The planets' total angular momentum, the other conserved quantity the paper watches
    when it chooses a time step (section 2.2), is an exact invariant of the map: every Kepler
    drift is a central-force flow and the interaction kick comes from a rotation-invariant
    potential.  Over 10^5 steps it may change by rounding only, where the energy error is
    ~1e-6."""
    pl = _planets()
    L0 = _barycentric_angular_momentum(M0, pl)
    worst = 0.0
    for _ in range(100):
        pl, _, _ = orc.planet_wh(M0, pl, 0.5, 1000, want_log=False)
        L = _barycentric_angular_momentum(M0, pl)
        worst = max(worst, np.linalg.norm(L - L0) / np.linalg.norm(L0))
    assert worst < 1e-12, worst


# --------------------------------------------------------------------------
# 6. Special cases
# --------------------------------------------------------------------------
def test_massless_planets_are_pure_kepler(orc):
    """With m_j = 0 the planets and particles all follow their own two-body orbits about m0
    (to FP64's phase random walk; any leftover interaction term would be orders larger)."""
    els = [(6.0, 0.05, 0.02, 0.3, 0.4, 0.5), (12.0, 0.1, 0.03, 1.3, 2.4, 1.5)]
    pl = np.array([[0.0, *pins.analytic_state(G * M0, *e)] for e in els])
    dt, n = 0.5, 2000

    def tol(a):
        return 100 * 2.0**-53 * pins.mean_motion(G * M0, a) * dt * n**1.5

    pl1, log, _ = orc.planet_wh(M0, pl, dt, n)
    for j, e in enumerate(els):
        ref = pins.propagate_exact(G * M0, pl[j, 1:], dt * n)
        assert pins.rel_err(pl1[j, 1:], ref)[0] < tol(e[0])
    pe = (25.0, 0.2, 0.1, 0.2, 0.3, 0.4)
    s0 = pins.analytic_state(G * M0, *pe)
    run = orc.ParticleRun(M0, pl[:, 0], s0[None], np.zeros(2), 0.0)
    run.advance(log, dt)
    ref = pins.propagate_exact(G * M0, s0, dt * n)
    assert pins.rel_err(run.state, ref)[0] < tol(pe[0])


def test_removal_at_t0_inside_rcrit(orc):
    pl = _planets()
    rc = orc.rcrit(M0, pl, 0, 1.0)
    # particles placed at 0.5 R_crit from planets 2 and 4 (1-based reason codes)
    p = np.zeros((3, 6))
    for row, j in enumerate([1, 3]):
        p[row, :3] = pl[j, 1:4] + np.array([0.5 * rc[j], 0, 0])
        p[row, 3:] = pl[j, 4:7]
    p[2] = pins.analytic_state(G, 25.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    _, log, _ = orc.planet_wh(M0, pl, 0.5, 3)
    run = orc.ParticleRun(M0, pl[:, 0], p, rc, 1000.0)
    run.advance(log, 0.5)
    assert list(run.removal_step[:2]) == [0, 0]
    assert list(run.reason[:2]) == [2, 4]
    np.testing.assert_array_equal(run.state[:2], p[:2])  # frozen at the encounter
    assert run.removal_step[2] == -1


def test_hill_radius_definition(orc):
    """R_H = a_p (m_p / 3 m0)^(1/3) with a_p the initial osculating semi-major axis."""
    els = (10.0, 0.3, 0.1, 0.2, 0.3, 2.0)
    m = 1e-4
    pl = np.array([[m, *pins.analytic_state(G * (M0 + m), *els)]])
    rc = orc.rcrit(M0, pl, 0, 2.0)
    assert abs(rc[0] - 2.0 * 10.0 * (m / 3.0) ** (1 / 3)) < 1e-12
    assert orc.rcrit(M0, pl, 1, 0.5)[0] == 0.5


def test_escape_step_matches_analytic_crossing(orc):
    """A hyperbolic particle with no planets is removed at the first step where r > r_max."""
    mu = G * M0
    a, e = 20.0, 1.3
    Mh0 = 0.0
    n = pins.mean_motion(mu, a)
    r_max = 150.0
    # r = a (e cosh F - 1)  =>  F at the crossing, t = (e sinh F - F - Mh0) / n
    Fc = math.acosh((r_max / a + 1.0) / e)
    t_cross = (e * math.sinh(Fc) - Fc - Mh0) / n
    dt = 0.5
    k_expected = math.ceil(t_cross / dt)
    assert abs(t_cross / dt - round(t_cross / dt)) > 1e-3  # not on a step boundary
    s0 = pins.analytic_state(mu, a, e, 0.2, 0.1, 0.3, Mh0)
    run = orc.ParticleRun(M0, np.zeros(0), s0[None], np.zeros(0), r_max)
    run.advance(np.zeros((k_expected + 50, 0, 3)), dt)
    assert run.reason[0] == -1
    assert run.removal_step[0] == k_expected
    r_final = np.linalg.norm(run.state[0, :3])
    assert r_final > r_max  # frozen just after crossing


def test_tie_breaks(orc):
    """Lowest planet index wins; an encounter wins over escape."""
    pl = _planets()
    _, log, _ = orc.planet_wh(M0, pl, 0.5, 2)
    mid = 0.5 * (pl[2, 1:4] + pl[3, 1:4])
    p = np.zeros((2, 6))
    p[0, :3] = mid
    p[1, :3] = pl[3, 1:4] + np.array([0.1, 0, 0])
    rc = np.full(4, 1e3)  # fixed-distance mode with a huge radius: every planet fires
    run = orc.ParticleRun(M0, pl[:, 0], p, rc, 1.0)  # r_max = 1 AU also fires
    run.advance(log, 0.5)
    assert list(run.reason) == [1, 1]
    rc2 = np.array([0.0, 0.0, 0.0, 0.5])
    run2 = orc.ParticleRun(M0, pl[:, 0], p[1:], rc2, 1.0)
    run2.advance(log, 0.5)
    assert run2.reason[0] == 4  # encounter beats escape
    run3 = orc.ParticleRun(M0, pl[:, 0], p[1:], np.zeros(4), 1.0)
    run3.advance(log, 0.5)
    assert run3.reason[0] == -1


def test_nonfinite_state_is_deactivated(orc):
    pl = _planets()
    _, log, _ = orc.planet_wh(M0, pl, 0.5, 3)
    p = np.array([[np.nan, 25.0, 0, 0, 1.2, 0], [25.0, 0, 0, 0, 1.25, 0]])
    run = orc.ParticleRun(M0, pl[:, 0], p, np.zeros(4), 1000.0)
    run.advance(log, 0.5)
    assert run.reason[0] == -3 and run.removal_step[0] == 1
    assert run.reason[1] == 0 and run.removal_step[1] == -1


def test_split_invariance_exact(orc):
    """advance(a) + advance(b) is bitwise advance(a + b) in the oracle (it never merges kicks)."""
    w = __import__("glisse_inputs").make("tiny", n=64)
    pl = w["planets"]
    rc = orc.rcrit(M0, pl)
    _, log, _ = orc.planet_wh(M0, pl, 0.5, 600)
    r1 = orc.ParticleRun(M0, pl[:, 0], w["particles"], rc, 1000.0).advance(log, 0.5)
    r2 = orc.ParticleRun(M0, pl[:, 0], w["particles"], rc, 1000.0)
    r2.advance(log[:251], 0.5).advance(log[250:], 0.5)
    np.testing.assert_array_equal(r1.state, r2.state)
    np.testing.assert_array_equal(r1.removal_step, r2.removal_step)
