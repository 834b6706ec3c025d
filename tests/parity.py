"""Comparison of the CUDA path with the oracle on the same seeded inputs.

The map is chaotic for particles that pass near a planet: a close pass
multiplies any rounding difference by a large factor, so two correct FP64
implementations that round differently drift apart on those particles.  The
acceptance criteria therefore measure each particle's own conditioning with
the oracle: it is rerun from inputs changed by one ulp (perturbed_inputs:
eight patterns of +-2^-52 relative changes of the particles' coordinates;
perturbed_planets: the planets' coordinates, where the path under test
integrates the planets itself), and ``sens`` is the largest relative state
change this causes.

  * removal step and reason agree exactly for every particle whose removal
    metric stayed at least 1e-9 away from its threshold at every test in the
    oracle's run, and whose removal step every 1-ulp rerun reproduces (both
    exclusions are listed, not counted);
  * regular particles (sens <= 3e-12 (n / 10^4)^1.5, i.e. orbits a one-ulp
    change barely moves, that never came within 5 R_crit of a planet: a
    close pass can start a divergence that the reruns have not yet shown)
    agree in position and velocity to 1e-10 relative
    after 10^4 steps, scaled by (n / 10^4)^1.5 (FP64 phase noise grows as
    n^1.5, see the oracle's two-body pins);
  * where the step is a different fraction of the orbit than on the 1024- and
    131072-particle workloads (the batched systems, dt = P_inner / 20), the
    same bounds are applied per particle in terms of the mean anomaly phi it
    advances: the rounding of every step random-walks the orbital energy
    (~ sqrt(n)), which turns into a phase error ~ phi sqrt(n), so
    (n / 10^4)^1.5 becomes (phi / PHASE_REF) (n / 10^4)^0.5 with PHASE_REF
    the phase of a = 25 AU over 10^4 steps of 0.5 yr (equal to the step law
    when phi grows like n, as on those workloads);
  * for eccentric orbits the same bounds are multiplied by 1 / (1 - e) of the
    initial osculating orbit (e capped at 0.99): near the pericentre the FP64
    noise of every drift is amplified by the Kepler equation's condition
    number 1 / (1 - e cos E), in the oracle as on the GPU.  On two-body orbits
    with e in [0.3, 0.95] (no planets, exact solution in 40 digits) the oracle
    is off by up to 6e-11 after 2000 steps and the GPU by up to 1.3e-11;
  * every other particle live in both agrees to within sens_factor(n) x sens
    (or the regular bound, whichever is larger), sens_factor(n) = 10 sqrt(n).
    Derivation: a second correct FP64 implementation differs from the oracle
    by rounding at every step, by at most ~10 ulp of the orbit's energy per
    step (the bound the oracle's own two-body runs meet).  The offset made at
    step k reaches step n multiplied by the same growth factor that carries a
    one-ulp change of the input from step 0 (linear phase shear on a regular
    orbit, exponential growth on a chaotic one, and no faster than that from a
    later start); offsets of independent steps add in quadrature, so after n
    steps the difference is at most ~10 sqrt(n) times the one-ulp divergence.
    ``sens`` is the largest of N_PERTURB = 8 one-ulp reruns (all coordinates
    up; velocities down; six seeded random sign patterns), so that one lucky
    rerun does not understate a particle's conditioning.  The law is checked
    on the CPU against a differently rounded build of the oracle
    (tests/test_parity_criteria.py) as well as by the GPU tests.
"""
from __future__ import annotations

import numpy as np

BAND = 1e-9
N_PERTURB = 8
ULP_PER_STEP = 10.0


def sens_factor(n_steps: int) -> float:
    """Largest ratio of a differently rounded FP64 run's difference to the one-ulp sensitivity
    after n_steps: ULP_PER_STEP ulp per step, added in quadrature (see the module docstring)."""
    return ULP_PER_STEP * np.sqrt(max(int(n_steps), 1))


def rel_err(a, b):
    a = np.asarray(a).reshape(-1, 6)
    b = np.asarray(b).reshape(-1, 6)
    er = np.linalg.norm(a[:, :3] - b[:, :3], axis=1) / np.linalg.norm(b[:, :3], axis=1)
    ev = np.linalg.norm(a[:, 3:] - b[:, 3:], axis=1) / np.linalg.norm(b[:, 3:], axis=1)
    return np.maximum(er, ev)


def state_tol(n_steps: int, base: float = 1e-10) -> float:
    return max(base * (max(n_steps, 1) / 1e4) ** 1.5, 1e-13)


def regular_limit(n_steps: int) -> float:
    return 3e-12 * (max(n_steps, 1) / 1e4) ** 1.5


# mean anomaly advanced at a = 25 AU around 1 M_sun over 10^4 steps of 0.5 yr (G = 4 pi^2)
PHASE_REF = 1e4 * 0.5 * 2.0 * np.pi / 25.0**1.5


def phase_advance(state0, mu, dt, n_steps):
    """Mean anomaly each particle advances over n_steps on its initial osculating orbit
    (unbound orbits: the circular rate at their initial distance)."""
    s = np.asarray(state0, dtype=np.float64).reshape(-1, 6)
    r = np.linalg.norm(s[:, :3], axis=1)
    alpha = 2.0 / r - np.sum(s[:, 3:] ** 2, axis=1) / mu
    rate = np.where(alpha > 0, np.sqrt(mu * np.abs(alpha) ** 3), np.sqrt(mu / r**3))
    return rate * abs(dt) * n_steps


def eccentricity(states, mu):
    """Osculating eccentricity of heliocentric states [n][6] about mu (test-side helper)."""
    s = np.asarray(states, dtype=np.float64).reshape(-1, 6)
    r = np.linalg.norm(s[:, :3], axis=1)
    v2 = np.sum(s[:, 3:] ** 2, axis=1)
    rv = np.sum(s[:, :3] * s[:, 3:], axis=1)
    ev = ((v2 - mu / r)[:, None] * s[:, :3] - rv[:, None] * s[:, 3:]) / mu
    return np.linalg.norm(ev, axis=1)


def perturbed_inputs(particles, k: int = N_PERTURB):
    """The one-ulp perturbations of a particle set used to measure sensitivity: every
    coordinate scaled by 1 + 2^-52; the velocities by 1 - 2^-52; then k - 2 patterns
    that scale each coordinate by 1 + s 2^-52 with s in {-1, 0, 1} drawn from a seeded
    generator (the same patterns on every call)."""
    p = np.asarray(particles, dtype=np.float64).reshape(-1, 6)
    up = p * (1.0 + 2.0**-52)
    vm = p.copy()
    vm[:, 3:] *= (1.0 - 2.0**-52)
    out = [up, vm]
    rng = np.random.default_rng(20110348)
    for _ in range(max(k - 2, 0)):
        sgn = rng.integers(-1, 2, size=p.shape)
        out.append(p * (1.0 + sgn * 2.0**-52))
    return out[:k]


def perturbed_planets(planets):
    """The planets with every heliocentric coordinate scaled by 1 + 2^-52 (masses unchanged): the
    rerun that measures a particle's sensitivity to the planets' own rounding.  The GPU integrates
    the planets itself, so its planet positions differ from the oracle's by their FP64 phase noise;
    a slow particle can be far more sensitive to that than to its own initial state."""
    pl = np.array(planets, dtype=np.float64).reshape(-1, 7)
    pl[:, 1:] *= 1.0 + 2.0**-52
    return pl


def sensitivity(base: dict, runs: list) -> tuple:
    """Per-particle sensitivity and the mask of particles whose removal step a 1-ulp change alters."""
    sens = np.zeros(len(base["removal_step"]))
    unstable = np.zeros(len(base["removal_step"]), dtype=bool)
    for r in runs:
        unstable |= r["removal_step"] != base["removal_step"]
        sens = np.maximum(sens, rel_err(r["state"], base["state"]))
    return sens, unstable


def compare(gpu: dict, orc: dict, n_steps: int, sens=None, unstable=None, phase=None, ecc=None) -> dict:
    """Returns a report dict; callers assert on its fields (see assert_parity).
    phase: optional per-particle mean anomaly advanced (phase_advance) for the phase-scaled bounds;
    ecc: optional initial eccentricities for the eccentricity-scaled bounds."""
    n = len(orc["removal_step"])
    if phase is None:
        tol = state_tol(n_steps)
        reg_lim = regular_limit(n_steps)
    else:
        scale = (np.asarray(phase, dtype=np.float64) / PHASE_REF) * (max(n_steps, 1) / 1e4) ** 0.5
        tol = np.maximum(1e-10 * scale, 1e-13)
        reg_lim = 3e-12 * scale
    if ecc is not None:
        amp = 1.0 / (1.0 - np.minimum(np.asarray(ecc, dtype=np.float64), 0.99))
        tol = tol * amp
        reg_lim = reg_lim * amp
    border = orc["margin"] < BAND
    if unstable is not None:
        border = border | unstable
    step_bad = (gpu["removal_step"] != orc["removal_step"]) & ~border
    rsn_bad = (gpu["removal_reason"] != orc["reason"]) & ~border
    both_alive = gpu["alive"] & (orc["removal_step"] < 0) & ~border
    e = rel_err(gpu["state"], orc["state"])
    if sens is None:
        # without reruns: only particles that never came within 5 R_crit count as regular
        regular = both_alive & (orc["closest"] >= 25.0)
        bound = np.where(regular, tol, np.inf)
    else:
        # insensitive to a one-ulp change AND never within 5 R_crit of a planet: a chaotic orbit
        # whose divergence has not yet shown in its reruns still counts as "other"
        regular = both_alive & (sens <= reg_lim) & (orc["closest"] >= 25.0)
        bound = np.maximum(tol, sens_factor(n_steps) * sens)
    tolv = np.broadcast_to(tol, (n,))
    over = both_alive & (e > bound)
    removed_same = (~gpu["alive"]) & (gpu["removal_step"] == orc["removal_step"]) & ~border
    return {
        "n": n,
        "excluded": int(border.sum()),
        "step_mismatch": int(step_bad.sum()),
        "reason_mismatch": int(rsn_bad.sum()),
        "removed": int((~gpu["alive"]).sum()),
        "regular": int(regular.sum()),
        "regular_max_err": float(e[regular].max()) if regular.any() else 0.0,
        "regular_over_tol": int((e[regular] > tolv[regular]).sum()),
        "over_bound": int(over.sum()),
        "alive_max_err": float(e[both_alive].max()) if both_alive.any() else 0.0,
        "max_ratio_to_sens": float((e[both_alive] / np.maximum(sens[both_alive], 1e-300)).max())
        if (sens is not None and both_alive.any()) else None,
        "removed_state_max_err": float(e[removed_same].max()) if removed_same.any() else 0.0,
        "tol": float(np.min(tolv)),
        "regular_worst": ({"id": int(np.where(regular)[0][np.argmax(e[regular] / tolv[regular])]),
                           "err": float(np.max(e[regular] / tolv[regular]) * tolv[regular][np.argmax(e[regular] / tolv[regular])]),
                           "tol": float(tolv[regular][np.argmax(e[regular] / tolv[regular])]),
                           "sens": float(sens[regular][np.argmax(e[regular] / tolv[regular])]) if sens is not None else None}
                          if regular.any() else None),
        "mismatch_ids": np.where(step_bad | rsn_bad)[0][:10].tolist(),
        "over_ids": np.where(over)[0][:10].tolist(),
    }


def assert_parity(rep: dict):
    assert rep["step_mismatch"] == 0, rep
    assert rep["reason_mismatch"] == 0, rep
    assert rep["regular_over_tol"] == 0, rep
    assert rep["over_bound"] == 0, rep


# ---------------------------------------------------------------------------
# close passes: a short horizon through a particle's deepest approach
# ---------------------------------------------------------------------------
CLOSE_LEAD, CLOSE_SPAN, CLOSE_RES = 20, 50, 10
CLOSE_QUIET = 1e-13   # one-ulp sensitivity below which a pass counts as not yet amplified
CLOSE_TOL = 1e-12     # absolute relative bound for those passes


def close_pass_groups(orc, w, ids, n_steps=10_000, lead=CLOSE_LEAD, res=CLOSE_RES, span=CLOSE_SPAN):
    """Oracle run of particles `ids` of workload w over n_steps, looked at in windows of `res`
    steps.  Every particle whose run comes within 5 R_crit of a planet while live (a pass that
    removes it included) is restarted `lead` steps (rounded down to a window) before the window
    of its deepest approach, and no later than n_steps - span, so that `span` steps of the log
    follow the restart.  Returns the planet log and [(k0, indices into ids, oracle states at
    step k0)] grouped by restart step k0; particles already removed at k0 are dropped."""
    pl = w["planets"]
    rc = orc.rcrit(w["star_mass"], pl)
    _, log, _ = orc.planet_wh(w["star_mass"], pl, w["dt"], n_steps)
    pr = orc.ParticleRun(w["star_mass"], pl[:, 0], w["particles"][ids], rc, 1000.0)
    depth = np.full((n_steps // res, len(ids)), np.inf)
    for b in range(n_steps // res):
        live = pr.removal_step < 0
        pr.closest[:] = np.inf
        pr.advance(log[b * res:(b + 1) * res + 1], w["dt"])
        depth[b, live] = pr.closest[live]
    best = np.argmin(depth, axis=0)
    by_k0 = {}
    for p in np.where(depth.min(axis=0) < 25.0)[0]:
        k0 = min(max(int(best[p]) * res - lead, 0), n_steps - span)
        by_k0.setdefault(k0 - k0 % res, []).append(int(p))
    groups = []
    for k0, ps in sorted(by_k0.items()):
        ps = np.array(ps)
        r = orc.ParticleRun(w["star_mass"], pl[:, 0], w["particles"][ids[ps]], rc, 1000.0)
        if k0 > 0:
            r.advance(log[:k0 + 1], w["dt"])
        live = r.removal_step < 0
        if live.any():
            groups.append((k0, ps[live], r.state[live].copy()))
    return log, groups


def close_pass_compare(orc, w, st0, log_slice, other: dict, span=CLOSE_SPAN) -> dict:
    """Oracle run of states st0 over log_slice (span steps) and its eight one-ulp reruns, against
    another implementation's result `other` (state, removal_step, removal_reason) of the same
    run.  Passes whose one-ulp sensitivity is at most CLOSE_QUIET must agree to CLOSE_TOL;
    the rest to sens_factor(span) x sens; removal steps and reasons exactly outside the band."""
    rc = orc.rcrit(w["star_mass"], w["planets"])

    def run(x):
        r = orc.ParticleRun(w["star_mass"], w["planets"][:, 0], x, rc, 1000.0)
        r.advance(log_slice, w["dt"])
        return {"state": r.state, "removal_step": r.removal_step, "reason": r.reason, "margin": r.margin,
                "closest": r.closest}

    o = run(st0)
    sens, unstable = sensitivity(o, [run(x) for x in perturbed_inputs(st0)])
    border = (o["margin"] < BAND) | unstable
    same = (other["removal_step"] == o["removal_step"]) & (other["removal_reason"] == o["reason"])
    e = rel_err(other["state"], o["state"])
    quiet = (sens <= CLOSE_QUIET) & same & ~border
    loud = (sens > CLOSE_QUIET) & same & ~border
    return {
        "cases": int((same & ~border).sum()),
        "mismatch": int((~same & ~border).sum()),
        "excluded": int(border.sum()),
        "removed": int(((o["removal_step"] >= 0) & same & ~border).sum()),
        "deep": int(((o["closest"] < 4.0) & same & ~border).sum()),
        "quiet": int(quiet.sum()),
        "quiet_over": int((e[quiet] > CLOSE_TOL).sum()),
        "quiet_max": float(e[quiet].max()) if quiet.any() else 0.0,
        "loud": int(loud.sum()),
        "loud_over": int((e[loud] > sens_factor(span) * sens[loud]).sum()),
        "sens_max": float(sens[same & ~border].max()) if (same & ~border).any() else 0.0,
    }


def close_pass_totals(reports: list) -> dict:
    tot = {}
    for r in reports:
        for k, v in r.items():
            tot[k] = max(tot.get(k, 0.0), v) if k.endswith("_max") else tot.get(k, 0) + v
    return tot
