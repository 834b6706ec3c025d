"""Planted mistakes in the oracle must be caught by its pins (no GPU).

Each case copies ``oracle/glisse_oracle.c``, plants one plausible mistake (a
dropped term, a wrong sign, a wrong index, a transposed operand, an
off-by-one), builds it, and runs a pin from test_oracle_pins.py against it:
the pin has to fail.  This is the evidence that the pins constrain every
part of the oracle, not only the parts that happen to be exercised.
"""
import os

import pytest

import oracle
import test_oracle_elements as PE
import test_oracle_paper_mode as PM
import test_oracle_pins as P
import test_oracle_tangent as PT

MUTANTS = [
    # (id, original text, planted text, pin to run)
    ("drop_indirect_h0", "a[d] = h0[d] + dir[d];", "a[d] = dir[d];", "brute"),
    ("planet_kick_suffix_sign", "+ S[d] / P->eta[k + 1];", "- S[d] / P->eta[k + 1];", "brute"),
    ("jacobi_eta_index", "dst[i][d] = src[i][d] - msum[d] / P->eta[i];",
     "dst[i][d] = src[i][d] - msum[d] / P->eta[i + 1];", "brute"),
    ("planet_mu_jacobi", "double mu = ORC_G * P->m0 * P->eta[i + 1] / P->eta[i];", "double mu = ORC_G * P->m0;",
     "brute"),
    ("particle_kick_transposed", "dir[1] -= Gm[j] * dy / d3;", "dir[1] -= Gm[j] * dz / d3;", "brute"),
    ("planet_interaction_transposed", "gh[i][1] += Gmj * dy / d3;", "gh[i][1] += Gmj * dz / d3;", "angmom"),
    ("closing_kick_old_planets", "particle_accel(np, Gm, P1, st, a);", "particle_accel(np, Gm, P0, st, a);",
     "brute"),
    ("drift_dE_g_sign", "double g = (dM - (x - s)) / n;", "double g = (dM - (x + s)) / n;", "two_body"),
    ("drift_dE_fdot", "double fd = -n * a * a * s / (r * r0);", "double fd = -n * a * s / (r * r0);", "two_body"),
    ("drift_univ_g", "double g = dt - mu * G3;", "double g = dt - mu * G2;", "two_body_hyp"),
    ("stumpff_series_sign", "term *= -z /", "term *= z /", "two_body_hyp"),
    ("tie_break_highest", "if (d2 < rc2[j] && hit == 0) hit = j + 1;", "if (d2 < rc2[j]) hit = j + 1;", "tie"),
    ("removal_step_off_by_one", "if (h) { rstep = step0 + k + 1; rsn = h; break; }",
     "if (h) { rstep = step0 + k; rsn = h; break; }", "escape"),
    ("newton_converged_step_rejected", "if (fabs(dx) <= 1e-15) { x += dx; conv = 1; break; }", "", "energy"),
    ("tangent_mean_motion_frozen", "cplx n = csqrt(mu / (a * a * a));", "cplx n = sqrt(mu / creal(a * a * a));",
     "tangent_sym"),
    ("tangent_kick_component", "cplx dx = r[0] - rj[0], dy = r[1] - rj[1], dz = r[2] - rj[2];",
     "cplx dx = r[0] - rj[0], dy = r[1] - rj[1], dz = r[1] - rj[2];", "tangent_fd"),
    ("hill_radius_cube", "rcrit[i] = value * (1.0 / inva) * cbrt(p[0] / (3.0 * m0));",
     "rcrit[i] = value * (1.0 / inva) * cbrt(p[0] / m0);", "hill"),
    ("paper_start_guess", "double x = dM / (1.0 - ec);\n    double dx = 0.0;", "double x = dM;\n    double dx = 0.0;",
     "paper_newton"),
    ("paper_iteration_count", "for (int it = 0; it < iters; ++it) {", "for (int it = 1; it < iters; ++it) {",
     "paper_newton"),
    ("paper_accepts_unconverged", "if (!(fabs(dx) <= tol)) return ORC_EKEPLER;", "", "paper_claim"),
    ("elements_node_sign", "double Om = hxy > 0.0 ? atan2(hx, -hy) : 0.0;",
     "double Om = hxy > 0.0 ? atan2(-hx, hy) : 0.0;", "elements"),
    ("elements_anomaly_eccentric", "M = wrap_2pi(E - e * sin(E));", "M = wrap_2pi(E);", "elements"),
    ("barycentre_total_mass", "R[d] = acc / mt;", "R[d] = acc / m0;", "barycentre"),
    ("resonant_planet_multiplier", "res_p * lam - res_q * lamN - (res_p - res_q) * varpi",
     "res_p * lam - res_p * lamN - (res_p - res_q) * varpi", "libration"),
    ("libration_window_inverted", "if (d0 < avoid) near0[p] = 1;", "if (d0 > avoid) near0[p] = 1;", "libration"),
]


def _run_pin(name):
    if name == "brute":
        P.test_brute_force_second_order(oracle)
    elif name == "two_body":
        for el in P.ELEMENTS[:4]:
            P.test_two_body_single_drift(oracle, el, 0.5)
    elif name == "two_body_hyp":
        for el in P.ELEMENTS[4:]:
            P.test_two_body_single_drift(oracle, el, 0.5)
            P.test_two_body_single_drift(oracle, el, 300.0)
    elif name == "tie":
        P.test_tie_breaks(oracle)
    elif name == "escape":
        P.test_escape_step_matches_analytic_crossing(oracle)
    elif name == "hill":
        P.test_hill_radius_definition(oracle)
    elif name == "tangent_sym":
        PT.test_tangent_is_symplectic(oracle)
    elif name == "tangent_fd":
        PT.test_tangent_matches_central_differences(oracle)
    elif name == "energy":
        P.test_two_body_no_secular_energy_drift(oracle, P.JUPITER_LIKE)
    elif name == "paper_newton":
        PM.test_last_step_matches_the_iteration_in_high_precision(oracle)
    elif name == "paper_claim":
        PM.test_five_iterations_reach_the_papers_convergence(oracle)
    elif name == "elements":
        PE.test_elements_invert_the_generator(oracle)
    elif name == "barycentre":
        PE.test_barycentre_has_zero_momentum(oracle)
    elif name == "angmom":
        P.test_planet_angular_momentum(oracle)
    elif name == "libration":
        PE.test_resonant_particles_librate_and_others_circulate(oracle)
    else:
        raise KeyError(name)


@pytest.mark.parametrize("mid,orig,planted,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(tmp_path, mid, orig, planted, pin):
    src = open(oracle.SOURCE).read()
    # the real map comes first in the file, its complex-step copy after it: a
    # mutation replaces the first occurrence of its anchor
    assert src.count(orig) >= 1, f"mutation anchor for {mid} missing"
    mutated = tmp_path / f"orc_{mid}.c"
    mutated.write_text(src.replace(orig, planted, 1))
    so = oracle.compile_source(str(mutated), str(tmp_path / f"orc_{mid}.so"))
    with oracle.using(so):
        with pytest.raises((AssertionError, RuntimeError, ValueError)):
            _run_pin(pin)


def test_unmutated_oracle_passes_the_same_pins():
    for pin in ["two_body", "two_body_hyp", "tie", "escape", "hill", "energy", "tangent_sym", "tangent_fd",
                "paper_newton", "paper_claim", "elements", "barycentre", "libration", "angmom"]:
        _run_pin(pin)
    assert os.path.exists(oracle.build())
