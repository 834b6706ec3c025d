"""The GPU parity criteria (parity.py) checked on the CPU, against other builds of the oracle.

The criteria compare two FP64 implementations of the same map that round
differently.  Here the second implementation is the oracle itself compiled
with floating-point contraction on (fused multiply-adds wherever the compiler
finds a product feeding a sum), which changes the rounding of nearly every
operation of every step, as the CUDA path's arithmetic does:

  * the whole-run criteria hold for it on the 1024-particle workload at 2000
    and 10^4 steps, including the derived sensitivity factor 10 sqrt(n) for
    particles that pass near planets (its ratio to the one-ulp sensitivity
    stays far below the factor);
  * the close-pass criterion (1e-12 over 50 steps through a particle's deepest
    approach within 5 R_crit) holds for it;
  * a planted error in the kick at small separation (1e-9 relative, only
    within 2 AU of a planet) is caught by the close-pass criterion on ~160
    passes at once, where the whole-run criteria, which judge the particles it
    touches by their one-ulp sensitivity, see it on about a dozen.
"""
import platform
import subprocess

import numpy as np
import pytest

import glisse_inputs as gi
import parity


def _build_variant(orc, tmp_path_factory, name, flags=None, replace=None):
    src = orc.SOURCE
    d = tmp_path_factory.mktemp(name)
    if replace is not None:
        text = open(src).read()
        old, new = replace
        assert text.count(old) == 1, old
        src = str(d / "variant.c")
        with open(src, "w") as f:
            f.write(text.replace(old, new))
    out = str(d / "lib.so")
    cflags = flags if flags is not None else orc.CFLAGS
    subprocess.run(["gcc", *cflags, "-o", out, src, "-lm"], check=True)
    return out


@pytest.fixture(scope="module")
def fma_build(orc, tmp_path_factory):
    flags = [f for f in orc.CFLAGS if f != "-ffp-contract=off"] + ["-ffp-contract=fast"]
    if platform.machine() in ("x86_64", "AMD64"):
        flags.append("-mfma")  # aarch64 has fused multiply-add in its base instruction set
    return _build_variant(orc, tmp_path_factory, "fma", flags=flags)


@pytest.fixture(scope="module")
def close_kick_mutant(orc, tmp_path_factory):
    # the particle kick's 1/d^3 off by 1e-9 relative within 2 AU of a planet (d^2 < 4 AU^2)
    return _build_variant(orc, tmp_path_factory, "close_kick", replace=(
        "        double d3 = d2 * sqrt(d2);\n        dir[0] -= Gm[j] * dx / d3;",
        "        double d3 = d2 * sqrt(d2) * (d2 < 4.0 ? 1.0 + 1e-9 : 1.0);\n        dir[0] -= Gm[j] * dx / d3;"))


def _as_other(o):
    return {"state": o["state"], "alive": o["removal_step"] < 0, "removal_step": o["removal_step"],
            "removal_reason": o["reason"]}


@pytest.mark.parametrize("n", [2000, 10_000])
def test_whole_run_criteria_hold_for_a_differently_rounded_build(orc, fma_build, n):
    w = gi.make("tiny")
    args = (w["star_mass"], w["planets"], w["particles"], w["dt"], n)
    base = orc.run(*args)
    runs = [orc.run(w["star_mass"], w["planets"], p, w["dt"], n) for p in parity.perturbed_inputs(w["particles"])]
    runs.append(orc.run(w["star_mass"], parity.perturbed_planets(w["planets"]), w["particles"], w["dt"], n))
    sens, unstable = parity.sensitivity(base, runs)
    with orc.using(fma_build):
        other = _as_other(orc.run(*args))
    rep = parity.compare(other, base, n, sens, unstable)
    e = parity.rel_err(other["state"], base["state"])
    both = other["alive"] & (base["removal_step"] < 0)
    print(n, rep["regular"], rep["regular_max_err"], rep["max_ratio_to_sens"], np.median(e[both]))
    parity.assert_parity(rep)
    assert np.median(e[both]) > 1e-15  # the builds do round differently
    # the derived factor has room: the largest ratio is well inside it
    assert rep["max_ratio_to_sens"] < 0.25 * parity.sens_factor(n)
    assert rep["regular"] >= 5


def _close_pass_reports(orc, other_build, n_ids=1024):
    w = gi.make("tiny")
    ids = np.arange(n_ids)
    log, groups = parity.close_pass_groups(orc, w, ids)
    rc = orc.rcrit(w["star_mass"], w["planets"])
    reps = []
    for k0, _, st0 in groups:
        sl = log[k0:k0 + parity.CLOSE_SPAN + 1]
        with orc.using(other_build):
            r = orc.ParticleRun(w["star_mass"], w["planets"][:, 0], st0, rc, 1000.0)
            r.advance(sl, w["dt"])
        other = {"state": r.state, "removal_step": r.removal_step, "removal_reason": r.reason}
        reps.append(parity.close_pass_compare(orc, w, st0, sl, other))
    return parity.close_pass_totals(reps)


def test_close_pass_criterion_holds_for_a_differently_rounded_build(orc, fma_build):
    t = _close_pass_reports(orc, fma_build)
    print(t)
    assert t["mismatch"] == 0 and t["quiet_over"] == 0 and t["loud_over"] == 0, t
    assert t["cases"] >= 100 and t["deep"] >= 20 and t["removed"] >= 5, t
    assert t["loud"] <= 0.05 * t["cases"], t
    assert t["quiet_max"] > 0.0  # the builds do differ on these passes


def test_close_pass_criterion_catches_a_small_separation_kick_error(orc, close_kick_mutant):
    t = _close_pass_reports(orc, close_kick_mutant)
    print(t)
    assert t["quiet_over"] + t["mismatch"] >= 10, t


def test_whole_run_criteria_see_the_small_separation_kick_error_too(orc, close_kick_mutant):
    w = gi.make("tiny")
    n = 2000
    base = orc.run(w["star_mass"], w["planets"], w["particles"], w["dt"], n)
    runs = [orc.run(w["star_mass"], w["planets"], p, w["dt"], n) for p in parity.perturbed_inputs(w["particles"])]
    runs.append(orc.run(w["star_mass"], parity.perturbed_planets(w["planets"]), w["particles"], w["dt"], n))
    sens, unstable = parity.sensitivity(base, runs)
    with orc.using(close_kick_mutant):
        other = _as_other(orc.run(w["star_mass"], w["planets"], w["particles"], w["dt"], n))
    rep = parity.compare(other, base, n, sens, unstable)
    print(rep["over_bound"], rep["max_ratio_to_sens"])
    assert rep["over_bound"] >= 3
