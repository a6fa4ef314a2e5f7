"""Step criteria of the oracle's 6th-order block steps (Sect. II: direct codes pair
>= 4th-order Hermite integrators with individual steps; the paper prints no criterion).

Two criteria are implemented:
- "generalised": the order-6 criterion that Nitadori & Makino publish, Aarseth's form
  generalised to the acceleration and its first five derivatives (orc_aarseth6_dt);
- "aarseth" (the default, and the rule the GPU path follows): Aarseth's 4th-order form on
  (a, jerk, snap, crackle), with the crackle's magnitude reduced by its rounding floor
  30 noise |a| / T^3 (T = dt / 2; noise 0: no floor).

The pins: hand values of the published criterion, and the comparison table of the design
notes, computed here with exact (FP64) forces and with seeded force noise of the size of
FP32 rounding (2^-23 relative on a, jerk and snap): the floor costs almost no
interactions when forces are exact, and with noisy forces the published criterion drives
the steps to dt_min while the floor rule does not. Run with -s to print the table.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1409_5474_gb300 import ic

NU = 2.0 ** -23          # relative rounding of double-single pair forces


def test_aarseth6_hand_values():
    e = [1.0, 0.0, 0.0]
    assert oracle.aarseth6_dt(e, e, e, e, e, e, 0.2) == pytest.approx(0.2, rel=1e-15)
    # |a|=4, |a1|=2, |a2|=1, |a3|=1, |a4|=6, |a5|=4: (sqrt(4)+2)/(sqrt(4)+6) = 1/2
    dt = oracle.aarseth6_dt([0, 4, 0], [2, 0, 0], [0, 0, 1], [1, 0, 0], [0, 6, 0], [0, 0, 4],
                            0.1)
    assert dt == pytest.approx(0.1 * 0.5 ** (1 / 3), rel=1e-15)
    # |a|=9, |a1|=1, |a2|=4, |a3|=3, |a4|=0, |a5|=12: (6 + 1) / 6
    dt = oracle.aarseth6_dt([0, 0, 9], [0, 1, 0], [4, 0, 0], [0, 3, 0], [0, 0, 0], [12, 0, 0],
                            0.3)
    assert dt == pytest.approx(0.3 * (7.0 / 6.0) ** (1 / 3), rel=1e-15)
    z = [0.0, 0.0, 0.0]
    assert oracle.aarseth6_dt(e, e, e, z, z, z, 0.1) == math.inf


def _two_body(d, e_frac):
    a = d / (1 - e_frac)
    vrel = math.sqrt((1 + e_frac) / (a * (1 - e_frac)))
    pos = np.array([[-d / 2, 0, 0], [d / 2, 0, 0]])
    vel = np.array([[0, -vrel / 2, 0], [0, vrel / 2, 0]])
    return np.array([0.5, 0.5]), pos, vel, 2 * math.pi * a ** 1.5


def _cases():
    p = ic.plummer(256, 7)
    m, pos, vel, period = _two_body(0.5, 0.5)
    return {"plummer256": (p.m, p.pos, p.vel, (1.0 / 64) ** 2, 0.25),
            "kepler_e0.5": (m, pos, vel, 0.0, math.floor(period * 16) / 16)}


def _run(case, criterion, eta, floor=0.0, perturb=0.0, max_steps=20000):
    m, pos, vel, eps2, t_end = case
    k0, w0 = oracle.energy(m, pos, vel, eps2)
    st = oracle.State6(m, pos, vel)
    steps, inter = oracle.hermite6_run(st, t_end, eps2, eta=eta, eta_s=0.01,
                                       max_steps=max_steps, noise=floor, criterion=criterion,
                                       perturb=perturb, seed=99)
    k1, w1 = oracle.energy(st.m, st.pos, st.vel, eps2)
    return {"done": bool((st.t == t_end).all()), "evals": inter / len(m) ** 2,
            "drift": abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0), "dt_min": float(st.dt.min())}


ROWS = [("published order-6, eta 0.2", "generalised", 0.2, 0.0),
        ("published order-6, eta 0.3", "generalised", 0.3, 0.0),
        ("Aarseth (a..crackle), no floor, eta 0.02", "aarseth", 0.02, 0.0),
        ("Aarseth (a..crackle), floor 2^-23, eta 0.02", "aarseth", 0.02, NU)]


def test_criteria_table_exact_and_noisy_forces():
    table = {}
    for cname, case in _cases().items():
        for label, crit, eta, floor in ROWS:
            for noisy in (False, True):
                table[cname, label, noisy] = _run(case, crit, eta, floor, NU if noisy else 0.0)
    print()
    print("%-13s %-45s %-26s %-26s" % ("case", "criterion", "exact: evals / drift",
                                       "noise 2^-23: evals / drift"))
    for (cname, label, noisy), r in table.items():
        if noisy:
            continue
        q = table[cname, label, True]
        print("%-13s %-45s %8.1f %-16.2e %8.1f %-9.2e%s" % (
            cname, label, r["evals"], r["drift"], q["evals"], q["drift"],
            "" if q["done"] else " (dt_min: stopped)"))
    for cname in _cases():
        nofl = table[cname, ROWS[2][0], False]
        fl = table[cname, ROWS[3][0], False]
        # the floor, with exact forces: the same work within 3%, energy within a factor 20
        assert fl["done"] and abs(fl["evals"] / nofl["evals"] - 1) < 0.03
        assert fl["drift"] < 20 * nofl["drift"] + 1e-13
        # with FP32-sized force noise: the floor rule's work and drift stay put ...
        fn = table[cname, ROWS[3][0], True]
        assert fn["done"] and abs(fn["evals"] / fl["evals"] - 1) < 0.03
        # ... while the published criterion at eta 0.2 collapses to dt_min
        gn = table[cname, ROWS[0][0], True]
        assert not gn["done"] and gn["dt_min"] == 2.0 ** -30
        assert table[cname, ROWS[0][0], False]["done"]


def test_noise_is_seeded_and_zero_perturbation_is_exact():
    case = _cases()["plummer256"]
    a = _run(case, "aarseth", 0.02, NU, NU)
    b = _run(case, "aarseth", 0.02, NU, NU)
    assert a == b
    c = _run(case, "aarseth", 0.02, NU, 0.0)
    d = _run(case, "aarseth", 0.02, NU, 0.0)
    assert c == d and c != a
