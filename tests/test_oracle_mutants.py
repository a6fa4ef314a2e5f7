"""Planted mistakes in the oracle must fail its pins.

Each case copies ``oracle/oracle.c``, plants one plausible slip (a wrong factor,
sign, power, operand order, dropped term), compiles the copy on the CPU, points
the oracle wrapper at it and runs the pin tests of ``test_oracle_force.py``,
``test_oracle_hermite.py``, ``test_oracle_hermite6.py`` and ``test_oracle_criteria.py``;
at least one pin must fail
for every mutant. The
unmodified source must pass them all.
"""
import os

import pytest

import oracle

from . import test_oracle_force as F
from . import test_oracle_hermite as H
from . import test_oracle_criteria as C
from . import test_oracle_hermite6 as H6

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = [
    ("jerk radial factor 3 -> 2", "3.0 * rv * r[c] * inv_s3 / s2", "2.0 * rv * r[c] * inv_s3 / s2"),
    ("jerk radial term sign", "v[c] * inv_s3 - 3.0", "v[c] * inv_s3 + 3.0"),
    ("acc power of distance", "inv_s3 = 1.0 / (s2 * s);", "inv_s3 = 1.0 / (s2);"),
    ("separation transposed", "r[c] = xj[c] - xi[c];", "r[c] = xi[c] - xj[c];"),
    ("relative velocity transposed", " v[c] = vj[c] - vi[c];", " v[c] = vi[c] - vj[c];"),
    ("pot sign", "*pot = -mj / s;", "*pot = mj / s;"),
    ("softening dropped", "r[2] * r[2] + eps2;", "r[2] * r[2];"),
    ("self pair kept", "if (j == skip)", "if (j == skip && j < 0)"),
    ("predictor jerk term 1/6 -> 1/2", "jerk[q] * d * d * d / 6.0", "jerk[q] * d * d * d / 2.0"),
    ("predictor velocity jerk term dropped", "vel_p[q] = vel[q] + acc[q] * d + jerk[q] * d * d / 2.0;",
     "vel_p[q] = vel[q] + acc[q] * d;"),
    ("corrector a3 coefficient", "a3 * dt * dt * dt * dt * dt / 120.0", "a3 * dt * dt * dt * dt * dt / 24.0"),
    ("corrector j0/j1 transposed", "4.0 * j0[c] + 2.0 * j1[c]", "2.0 * j0[c] + 4.0 * j1[c]"),
    ("corrector velocity a2 term", "v1[c] = vp[c] + a2 * dt * dt * dt / 6.0", "v1[c] = vp[c] + a2 * dt * dt * dt / 2.0"),
    ("a2 not moved to end of step", "a2_end[c] = a2 + dt * a3;", "a2_end[c] = a2;"),
    ("Aarseth numerator", "double num = na * n2 + nj * nj;", "double num = na * n2 + na * na;"),
    ("growth limit x2 -> x4", "d > 2.0 * dt_old", "d > 4.0 * dt_old"),
    ("commensurability dropped", "fmod(t_new, d) != 0.0", "fmod(t_new, d) != fmod(t_new, d)"),
    ("scheduler takes a particle early", "if (s->t[i] + s->dt[i] == t_next)\n            active[na++] = i;",
     "if (s->t[i] + s->dt[i] <= t_next + s->dt[i] / 2)\n            active[na++] = i;"),
    ("kinetic energy factor", "0.5 * m[i] * (v[0]", "m[i] * (v[0]"),
    ("iterated corrector from corrected positions", "orc_correct_one(dt, xs + r, vs + r,",
     "orc_correct_one(dt, pp + q, vp + q,"),
    ("iterated corrector keeps predicted velocities", "vp[q + c] = v1[r + c];", "(void)v1;"),
    ("one iteration too few", "for (int it = 1; it < n_corr; it++)", "for (int it = 2; it < n_corr; it++)"),
    ("snap: beta without alpha^2", "/ q2 + alpha * alpha;", "/ q2;"),
    ("snap: alpha factor 6 -> 3", "- 6.0 * alpha * jerk[c]", "- 3.0 * alpha * jerk[c]"),
    ("snap: relative acceleration transposed", "da[c] = aj[c] - ai[c];", "da[c] = ai[c] - aj[c];"),
    ("snap: r.a term partly dropped", "dv[2] * dv[2] + dx[0] * da[0] +", "dv[2] * dv[2] + 0.0 * da[0] +"),
    ("snap kernel: self pair kept", "if (skip == j)", "if (skip == j && j < 0)"),
    ("snap kernel: softening dropped", "double q2 = eps2 + dx[0]", "double q2 = 0.0 + dx[0]"),
    ("snap kernel: velocity transposed", "dv[c] = vj[c] - vi[c];", "dv[c] = vi[c] - vj[c];"),
    ("predictor6 crackle term 1/120 -> 1/24", "crackle[q] * d5 / 120.0", "crackle[q] * d5 / 24.0"),
    ("predictor6 acceleration truncated",
     "acc_p[q] = acc[q] + jerk[q] * d + snap[q] * d2 / 2.0 + crackle[q] * d3 / 6.0;",
     "acc_p[q] = acc[q] + jerk[q] * d;"),
    ("corrector6 jerk coefficient 1/10 -> 1/12", "dt * dt / 10.0 * (j1[c] - j0[c])",
     "dt * dt / 12.0 * (j1[c] - j0[c])"),
    ("corrector6 position from v0 only", "dt / 2.0 * (v0[c] + v1[c])", "dt * v0[c]"),
    ("crackle coefficient 15 -> 12", "(15.0 * (T * Jp - Am)", "(12.0 * (T * Jp - Am)"),
    ("crackle left at the mid-point", "a3_end[c] = c3 + c4 * T + c5 * T * T / 2.0;", "a3_end[c] = c3;"),
    ("pop sign", "a4_end[c] = c4 + c5 * T;", "a4_end[c] = c4 - c5 * T;"),
    ("criterion6 pop instead of crackle", "ce[c] = a3[c] * ((cn - cfl) / cn);",
     "ce[c] = a4[c] * ((cn - cfl) / cn);"),
    ("criterion6 crackle floor ignored", "if (cn > cfl)", "if (cn > 0.0 * cfl)"),
    ("criterion6 jerk instead of snap", "orc_aarseth_dt(a1 + r, j1 + r, s1 + r, ce, eta)",
     "orc_aarseth_dt(a1 + r, j1 + r, j1 + r, ce, eta)"),
    ("crackle not kept", "s->crk[q + c] = a3[c];", "s->crk[q + c] = 0.0;"),
    ("scheduler6 takes a particle early", "if (due == t_next)", "if (due <= t_next + s->dt[i] / 2)"),
    ("initial snap without accelerations", "memcpy(aj, s->acc, sizeof(double) * 3 * (size_t)n);",
     "(void)0;"),
    ("generalised criterion: square root for the cube root", "return eta * cbrt(num / den);",
     "return eta * sqrt(num / den);"),
    ("generalised criterion: pop and 5th derivative swapped",
     "double den = sqrt(norm3(a3) * norm3(a5)) + norm3(a4);",
     "double den = sqrt(norm3(a3) * norm3(a4)) + norm3(a5);"),
    ("generalised criterion never selected", "} else if (crit == ORC_CRIT_GENERALISED) {",
     "} else if (crit == -1) {"),
    ("force noise on the acceleration dropped",
     "a1[r + c] += perturb * na1 * noise_unit(seed, step, active[k], c);", "(void)na1;"),
]


def _pins():
    out = [(f"two_body[{i}]", lambda i=i: F.test_two_body_closed_forms(i)) for i in range(3)]
    out += [
        ("ext", F.test_external_i_set_matches_member_case),
        ("cube0", lambda: F.test_cube_vertices(0.0)),
        ("cube_eps", lambda: F.test_cube_vertices(0.3)),
        ("triangle", F.test_equilateral_triangle),
        ("third_law", lambda: F.test_newton_third_law(1e-2)),
        ("pot_vs_energy", lambda: F.test_pot_matches_pairwise_energy(1e-2)),
        ("grad_pot", lambda: F.test_acc_is_minus_grad_pot(2e-2)),
        ("jerk_fd", lambda: F.test_jerk_is_time_derivative_of_acc(2e-2)),
        ("rotation", F.test_rigid_rotation_jerk),
        ("homology", F.test_homologous_expansion_jerk),
        ("single", F.test_single_particle_and_empty),
        ("predictor", H.test_predictor_exact_for_cubic),
        ("corrector", H.test_corrector_exact_for_quintic),
        ("aarseth", H.test_aarseth_criterion_hand_values),
        ("quantize", H.test_quantize_cases),
        ("circular", H.test_softened_circular_orbit_and_convergence),
        ("kepler", H.test_kepler_ellipse_and_convergence),
        ("momentum", H.test_shared_step_momentum_conservation),
        ("dyadic", lambda: H.test_block_times_are_dyadic(H.make_block_run())),
        ("equal_block_shared", H.test_equal_block_steps_equal_shared_steps),
        ("schedule_counts", H.test_block_schedule_counts_two_binaries),
        ("energy_order", H.test_energy_convergence_order),
        ("pec_order", H.test_iterated_corrector_order_and_accuracy),
        ("pec_symmetry", H.test_iterated_corrector_approaches_time_symmetry),
        ("pec_block", H.test_iterated_corrector_block_steps_energy),
    ]
    out += [("h6_" + k[5:], getattr(H6, k)) for k in sorted(dir(H6)) if k.startswith("test_")]
    out += [("crit_" + k[5:], getattr(C, k)) for k in sorted(dir(C)) if k.startswith("test_")]
    return out


def _failures():
    failed = []
    for name, fn in _pins():
        try:
            fn()
        except Exception:  # an AssertionError, or a NaN tripping a comparison
            failed.append(name)
    return failed


def test_unmodified_source_passes_all_pins():
    assert _failures() == []


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, desc, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = oracle.compile_source(str(path), str(tmp_path / "libmutant.so"))
    prev = oracle.use_library(lib)
    try:
        failed = _failures()
    finally:
        oracle._restore(prev)
    assert failed, f"no pin caught: {desc}"
