"""Algorithmic FP64 work per particle-step of the map, counted on the oracle.

Runs the oracle's particle map through its op-counting build (opcount.cpp) on
the 1024-particle workload (4 planets, 10^4 steps of 0.5 yr, the planets'
log from the oracle's own Wisdom-Holman integration), checks that the
counting build reproduces the plain oracle bit for bit, and writes the
counts per particle-step to profiles/oracle_op_count_tiny.txt:

    python oracle/opcount.py

Only oracle/ is called.  A particle-step is one step of one live particle
(a removed particle counts the steps up to its removal).  FLOP = additions
and subtractions + multiplications + divisions + square roots +
transcendental calls, one each; comparisons and fabs / floor / fmod are
listed apart.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import glisse_inputs as gi  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(ROOT, "profiles", "oracle_op_count_tiny.txt")


def main(n_steps: int = 10_000):
    w = gi.make("tiny")
    pl = w["planets"]
    rc = oracle.rcrit(w["star_mass"], pl)
    _, log, _ = oracle.planet_wh(w["star_mass"], pl, w["dt"], n_steps)
    t0 = time.perf_counter()
    st, rs, rn, cnt = oracle.opcount_particles(w["star_mass"], pl[:, 0], log, w["dt"], w["particles"], rc, 1000.0)
    el = time.perf_counter() - t0
    ref = oracle.ParticleRun(w["star_mass"], pl[:, 0], w["particles"], rc, 1000.0)
    ref.advance(log, w["dt"])
    assert np.array_equal(st, ref.state) and np.array_equal(rs, ref.removal_step), "counting build differs"
    psteps = int(np.where(rs >= 0, rs, n_steps).sum())
    flop = cnt["add"] + cnt["mul"] + cnt["div"] + cnt["sqrt"] + cnt["trans"]
    lines = [
        "# Algorithmic FP64 work of the test-particle map, counted on the oracle's own arithmetic",
        "# command: python oracle/opcount.py",
        f"# workload: tiny (1024 particles, 4 planets, dt {w['dt']} yr), {n_steps} steps; "
        f"{int((rs >= 0).sum())} particles removed",
        "# one particle-step = one step of one live particle: two half kicks (h0 and every planet's",
        "# direct term each time), the converged Kepler drift (libm sin/cos per Newton iteration),",
        "# the encounter and escape tests",
        f"particle_steps: {psteps}",
        f"flop_per_particle_step: {flop / psteps:.2f}",
    ]
    for k in oracle.OPCOUNT_FIELDS:
        lines.append(f"{k}_per_particle_step: {cnt[k] / psteps:.3f}")
    lines.append(f"# counting run: {el:.1f} s on one thread; results equal the plain oracle's bit for bit")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
