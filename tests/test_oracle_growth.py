"""Pins of the oracle's tangent-growth gradient (no GPU).

The oracle's gradient of g = log(|J t0| / |t0|) with respect to the initial
state, t0 held fixed, is a Richardson-extrapolated central difference of its
complex-step growth.  Checked here:
* with no planets, against the exact two-body flow differentiated twice by
  central differences in 60-digit arithmetic (mpmath);
* the second derivative of the map is symmetric, d(J b)/dx [a] = d(J a)/dx [b];
* the per-coordinate gradient reproduces a directional difference along a
  random direction;
* the gradient does not change when the seed is rescaled.
"""
import numpy as np

import glisse_inputs as gi
import pins

M0 = 1.0


def _setup(orc, n=6, steps=400):
    w = gi.make("diff", n=64)
    pl = w["planets"]
    _, log, _ = orc.planet_wh(M0, pl, w["dt"], steps)
    return w, pl, log, orc.rcrit(M0, pl), w["particles"][:n]


def _seed(s0):
    r = s0[:, :3] / np.linalg.norm(s0[:, :3], axis=1, keepdims=True)
    v = s0[:, 3:] / np.linalg.norm(s0[:, 3:], axis=1, keepdims=True)
    return np.hstack([r, v]) / 2**0.5


def test_growth_gradient_two_body_matches_exact_flow(orc):
    mp = pins._mp()
    mu = pins.G * M0
    els = [(25.0, 0.05, 0.3, 1.1, 2.2, 0.7), (22.0, 0.4, 0.2, 0.4, 1.3, 2.9)]
    s0 = np.array([pins.analytic_state(mu, *e) for e in els])
    t0 = _seed(s0)
    n, dt = 200, 0.5
    log = np.zeros((n + 1, 0, 3))
    got, err, ok = orc.growth_gradient(M0, np.zeros(0), log, dt, s0, t0, np.zeros(0), 0.0)
    assert ok.all()
    dps = 60
    with mp.workdps(dps):
        he, hg = mp.mpf("1e-22"), mp.mpf("1e-14")

        def growth_exact(x):
            xp = [x[k] + he * t0[p][k] for k in range(6)]
            xm = [x[k] - he * t0[p][k] for k in range(6)]
            fp = pins.propagate_exact_mp(mu, xp, dt * n, dps)
            fm = pins.propagate_exact_mp(mu, xm, dt * n, dps)
            jt = [(fp[k] - fm[k]) / (2 * he) for k in range(6)]
            return mp.log(mp.fsum(v * v for v in jt) / mp.fsum(mp.mpf(float(v)) ** 2 for v in t0[p])) / 2

        for p in range(len(els)):
            x0 = [mp.mpf(float(v)) for v in s0[p]]
            ref = np.empty(6)
            for c in range(6):
                xp = list(x0)
                xm = list(x0)
                xp[c] += hg
                xm[c] -= hg
                ref[c] = float((growth_exact(xp) - growth_exact(xm)) / (2 * hg))
            rel = np.abs(got[p] - ref).max() / np.abs(ref).max()
            assert rel < 1e-7, (p, rel, got[p], ref)


def test_second_derivative_is_symmetric(orc):
    w, pl, log, rc, s0 = _setup(orc, n=4, steps=300)
    rng = np.random.default_rng(3)
    a = rng.normal(size=s0.shape) * [1e-2, 1e-2, 1e-2, 1e-3, 1e-3, 1e-3]
    b = rng.normal(size=s0.shape) * [1e-2, 1e-2, 1e-2, 1e-3, 1e-3, 1e-3]
    h = 1e-3  # along the scaled directions: ~1e-5 AU, ~1e-6 AU/yr

    def djv(x, u, v):
        """d(J(x) v)/dx [u], central difference of the complex-step tangent."""
        _, jp, _, _ = orc.particles_jvp(M0, pl[:, 0], log, w["dt"], x + h * u, v, rc, 1000.0)
        _, jm, _, _ = orc.particles_jvp(M0, pl[:, 0], log, w["dt"], x - h * u, v, rc, 1000.0)
        return (jp - jm) / (2 * h)

    ab = djv(s0, a, b)
    ba = djv(s0, b, a)
    rel = np.abs(ab - ba).max(axis=1) / np.abs(ab).max(axis=1)
    assert rel.max() < 1e-6, rel


def test_gradient_gives_the_directional_derivative(orc):
    w, pl, log, rc, s0 = _setup(orc, n=4, steps=400)
    t0 = _seed(s0)
    grad, err, ok = orc.growth_gradient(M0, pl[:, 0], log, w["dt"], s0, t0, rc, 1000.0)
    assert ok.all()
    a = np.random.default_rng(4).normal(size=s0.shape) * [1e-5, 1e-5, 1e-5, 1e-6, 1e-6, 1e-6]
    d = []
    for hh in (1.0, 0.5):
        gp, _ = orc.growth(M0, pl[:, 0], log, w["dt"], s0 + hh * a, t0, rc, 1000.0)
        gm, _ = orc.growth(M0, pl[:, 0], log, w["dt"], s0 - hh * a, t0, rc, 1000.0)
        d.append((gp - gm) / (2 * hh))
    fd = (4 * d[1] - d[0]) / 3
    pred = (grad * a).sum(axis=1)
    assert np.abs(pred - fd).max() < 1e-7 * np.abs(fd).max(), (pred, fd)


def test_gradient_is_invariant_under_seed_scale(orc):
    w, pl, log, rc, s0 = _setup(orc, n=3, steps=300)
    t0 = _seed(s0)
    g1, _, _ = orc.growth_gradient(M0, pl[:, 0], log, w["dt"], s0, t0, rc, 1000.0)
    g2, _, _ = orc.growth_gradient(M0, pl[:, 0], log, w["dt"], s0, 3.0 * t0, rc, 1000.0)
    assert np.abs(g1 - g2).max() < 1e-7 * np.abs(g1).max()  # the difference quotients' rounding floor
