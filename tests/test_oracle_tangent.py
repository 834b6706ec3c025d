"""Pins of the oracle's tangent map (complex-step derivative of the map), no GPU.

* the Jacobian of a symplectic map is symplectic: J^T Omega J = Omega;
* it agrees with central finite differences of the pinned oracle;
* with no planets it agrees with the derivative of the exact two-body orbit
  (mpmath, 40 digits);
* the Jacobian of the map run backwards is the inverse of the forward one.
"""
import numpy as np
import pytest

import glisse_inputs as gi
import pins

M0 = 1.0
OMEGA = np.block([[np.zeros((3, 3)), np.eye(3)], [-np.eye(3), np.zeros((3, 3))]])


def _setup(orc, n=12, steps=1000):
    w = gi.make("tiny", n=n)
    pl = w["planets"]
    _, log, _ = orc.planet_wh(M0, pl, w["dt"], steps)
    return w, pl, log, orc.rcrit(M0, pl)


def test_tangent_is_symplectic(orc):
    w, pl, log, rc = _setup(orc)
    J = orc.particles_jacobian(M0, pl[:, 0], log, w["dt"], w["particles"], rc, 1000.0)
    for p in range(J.shape[0]):
        M = J[p].T @ OMEGA @ J[p]
        scale = max(1.0, np.abs(J[p]).max() ** 2)
        assert np.abs(M - OMEGA).max() < 1e-13 * scale, (p, np.abs(M - OMEGA).max(), scale)


def test_tangent_matches_central_differences(orc):
    w, pl, log, rc = _setup(orc, n=8, steps=400)
    s0 = w["particles"]
    J = orc.particles_jacobian(M0, pl[:, 0], log, w["dt"], s0, rc, 1000.0)
    h = 1e-7  # AU in positions, AU/yr in velocities
    for c in range(6):
        e = np.zeros_like(s0)
        e[:, c] = h
        sp = orc.ParticleRun(M0, pl[:, 0], s0 + e, rc, 1000.0).advance(log, w["dt"]).state
        sm = orc.ParticleRun(M0, pl[:, 0], s0 - e, rc, 1000.0).advance(log, w["dt"]).state
        fd = (sp - sm) / (2 * h)
        # FD round-off is ~eps |state| / h in absolute terms: measure against the Jacobian scale
        err = np.abs(fd - J[:, :, c]).max(axis=1) / np.abs(J).max(axis=(1, 2))
        assert err.max() < 1e-5, (c, err.max())


def test_tangent_two_body_matches_exact_orbit(orc):
    pytest.importorskip("mpmath")
    mu = pins.G * M0
    els = [(25.0, 0.05, 0.3, 1.1, 2.2, 0.7), (25.0, 0.4, 0.3, 1.1, 2.2, 2.9), (25.0, 1.5, 0.3, 1.1, 2.2, 0.3)]
    s0 = np.array([pins.analytic_state(mu, *e) for e in els])
    n, dt = 50, 0.5
    log = np.zeros((n + 1, 0, 3))
    J = orc.particles_jacobian(M0, np.zeros(0), log, dt, s0, np.zeros(0), 0.0)
    h = 1e-6
    for p in range(len(els)):
        for c in range(6):
            e = np.zeros(6)
            e[c] = h * (np.linalg.norm(s0[p, :3]) if c < 3 else np.linalg.norm(s0[p, 3:]))
            fp = pins.propagate_exact(mu, s0[p] + e, dt * n, dps=50)
            fm = pins.propagate_exact(mu, s0[p] - e, dt * n, dps=50)
            # central difference of the exact flow; h^2 truncation ~1e-12 at this h
            fd = (fp - fm) / (2 * e[c])
            err = np.abs(fd - J[p, :, c]).max() / np.abs(J[p]).max()
            assert err < 1e-9, (p, c, err)


def test_backward_jacobian_is_the_inverse(orc):
    w, pl, log, rc = _setup(orc, n=8, steps=500)
    s0 = w["particles"]
    J = orc.particles_jacobian(M0, pl[:, 0], log, w["dt"], s0, np.zeros(4), 0.0)
    s1 = orc.ParticleRun(M0, pl[:, 0], s0, np.zeros(4), 0.0).advance(log, w["dt"]).state
    Jb = orc.particles_jacobian(M0, pl[:, 0], log[::-1], -w["dt"], s1, np.zeros(4), 0.0)
    for p in range(len(s0)):
        P = Jb[p] @ J[p]
        assert np.abs(P - np.eye(6)).max() < 1e-9 * max(1.0, np.abs(J[p]).max() ** 2), p
