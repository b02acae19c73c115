"""The oracle's pins catch plausible mistakes in it.

Each case plants one mistake (a dropped term, a flipped sign, a wrong
neighbour index, a slip in the noise, the schedule, the domain labels or the
adjoint) into a copy of ``oracle/xy_oracle.c``, compiles the copy into a
temporary library, and runs the named pins of ``tests/test_oracle_pins.py``
against it: at least one of them must fail.  The mistakes live only in the
temporary copy; the oracle itself is untouched.
"""
import importlib.util
import os
import shutil

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "xy_oracle.c")

force = lambda P: P.test_force_is_minus_gradient_of_hamiltonian(8, 6)
init = lambda P: P.test_init_modes()
equip = lambda P: P.test_equipartition_halves_with_fresh_draws_reading()
msd = lambda P: P.test_benchmark_harmonic_msd(0.05, 1.0)
adj_E = lambda P: P.test_adjoint_matches_finite_differences_smooth_field(1.0, 0.0)
adj_M = lambda P: P.test_adjoint_matches_finite_differences_smooth_field(0.0, 1.0)
sens = lambda P: P.test_theta_sensitivity_matches_finite_differences()
fwd_field = lambda P: P.test_adjoint_forward_equals_stepper(([5, 30], [0.4, 2.5]))
adj_field = lambda P: P.test_adjoint_with_field_schedule_matches_finite_differences()
cpl_exact = lambda P: P.test_coupling_schedule_scales_the_couplings_exactly()
adj_cpl = lambda P: P.test_adjoint_with_coupling_schedule_matches_finite_differences()


def strip(P):
    """The split run against the whole lattice, both through P's oracle."""
    from tests import test_strips
    saved = test_strips.oracle
    test_strips.oracle = P.oracle
    try:
        test_strips.test_split_run_equals_the_whole_lattice_bit_for_bit(8, 22, 3, 3, 10, test_strips.COUPLINGS)
    finally:
        test_strips.oracle = saved

# name: (text in the oracle, planted replacement, pins of which one must fail)
MUTANTS = {
    "force_sign_J_par": ("F[i] = -q * Jx * fx - q * Jy * fy", "F[i] = q * Jx * fx - q * Jy * fy", [force]),
    "force_drops_J_perp": ("F[i] = -q * Jx * fx - q * Jy * fy + h", "F[i] = -q * Jx * fx + h", [force]),
    "force_field_sign": ("- q * Jy * fy + h * p * sin(p * t);", "- q * Jy * fy - h * p * sin(p * t);", [force]),
    "force_neighbour_index": ("+ sin(q * (t - th[nb(Lx, Ly, x, y, 0, -1)]));\n            F[i]",
                              "+ sin(q * (t - th[nb(Lx, Ly, x, y, 0, 1)]));\n            F[i]", [force]),
    "energy_drops_kinetic": ("se += 0.5 * om[i] * om[i]", "se += 0.0 * om[i] * om[i]", [force]),
    "energy_perp_bond_direction": ("- Jy * cos(q * (th[i] - th[nb(Lx, Ly, x, y, 0, 1)]))",
                                   "- Jy * cos(q * (th[i] - th[nb(Lx, Ly, x, y, 1, 0)]))", [force]),
    "order_parameter_cosine": ("sm += sigma * sin(q * th[i]);", "sm += sigma * cos(q * th[i]);", [force, init]),
    "noise_amplitude_factor": ("return 0.5 * sqrt(2.0 * eta * T) * sqrt(dt);",
                               "return 0.5 * sqrt(eta * T) * sqrt(dt);", [equip]),
    "damping_sign_second_kick": ("amp1 * nz1[i]) / (1.0 + 0.5 * eta * dt);",
                                 "amp1 * nz1[i]) / (1.0 - 0.5 * eta * dt);", [equip, msd]),
    "wrap_returns_input": ("if (r < -0.5 * XYO_PI) r += XYO_PI;\n    return r;",
                           "if (r < -0.5 * XYO_PI) r += XYO_PI;\n    return t;", [lambda P: P.test_wrap_interval_and_periodicity()]),
    "uniform_drops_half_offset": ("((double)(x >> 9) + 0.5) * (1.0 / 8388608.0)",
                                  "((double)(x >> 9)) * (1.0 / 8388608.0)",
                                  [lambda P: P.test_uniform_endpoints_and_exactness()]),
    "box_muller_radius": ("double r = sqrt(-2.0 * log(u_r));", "double r = sqrt(-log(u_r));",
                          [lambda P: P.test_gaussian_moments_and_box_muller_radius()]),
    "noise_ignores_replica": ("ctr[1] = ((uint32_t)cfg << 16) | ((uint32_t)rep & 0xFFFFu);",
                              "ctr[1] = ((uint32_t)cfg << 16);", [lambda P: P.test_noise_streams_are_distinct()]),
    "schedule_slope_reversed": ("return Ts[i] + (Ts[i + 1] - Ts[i]) * f;",
                                "return Ts[i + 1] + (Ts[i] - Ts[i + 1]) * f;",
                                [lambda P: P.test_temperature_schedule_linear_quench()]),
    "ordered_start_angle": ("theta[s] = 2.0 * XYO_PI / 5.0;", "theta[s] = XYO_PI / 5.0;", [init]),
    "ccl_strict_threshold": ("if (labels[m] < 0 && (theta[m] >= 0.0f) == spin)",
                             "if (labels[m] < 0 && (theta[m] > 0.0f) == spin)",
                             [lambda P: P.test_ccl_zero_angle_counts_as_up()]),
    "ccl_drops_left_neighbour": ("int64_t nbs[4] = { nb(Lx, Ly, x, y, 1, 0), nb(Lx, Ly, x, y, -1, 0),",
                                 "int64_t nbs[4] = { nb(Lx, Ly, x, y, 1, 0), nb(Lx, Ly, x, y, 1, 0),",
                                 [lambda P: P.test_ccl_against_graph_library("random"),
                                  lambda P: P.test_ccl_against_graph_library("spiral")]),
    "adjoint_field_hessian_sign": ("out[i] += v[i] * h * p * p * cos(p * t);",
                                   "out[i] -= v[i] * h * p * p * cos(p * t);", [adj_E]),
    "adjoint_neighbour_hessian_sign": ("out[nbr[d]] += v[i] * cq;", "out[nbr[d]] -= v[i] * cq;", [adj_E]),
    "adjoint_field_parameter_sign": ("gp[2] += wE * cos(p * th[i]) / N;", "gp[2] -= wE * cos(p * th[i]) / N;",
                                     [adj_E]),
    "adjoint_order_parameter_drops_q": ("tb[i] += wM * sgn * sigma * q * cos(q * th[i]) / N;",
                                        "tb[i] += wM * sgn * sigma * cos(q * th[i]) / N;", [adj_M]),
    "adjoint_damping_reverse": ("wb[i] = (1.0 - a) * hb[i];", "wb[i] = (1.0 + a) * hb[i];", [adj_E]),
    "adjoint_eta_term": ("grad[3] = 0.5 * dt * (abar - b * b * bbar) + geta_amp;",
                         "grad[3] = 0.5 * dt * (abar - b * bbar) + geta_amp;", [adj_E]),
    "adjoint_forward_bond_x": ("tb[ix] -= wE * Jx * q * sin(q * dx) / N;",
                               "tb[ix] += wE * Jx * q * sin(q * dx) / N;", [adj_E]),
    "sensitivity_drops_drift": ("hb[i] += tb[i] * dt;", "hb[i] += tb[i] * 0.0;", [sens]),
    "sensitivity_damping_reverse": ("wb[i] = hb[i] * (1.0 - a);", "wb[i] = hb[i] * (1.0 + a);", [sens]),
    "sensitivity_second_kick_force": ("Fb[i] += wb[i] * b * 0.5 * dt;", "Fb[i] = wb[i] * b * 0.5 * dt;", [sens]),
    "field_force_of_the_wrong_time_point": ("params_at(prm, k + 1, sc, prm_next);",
                                            "params_at(prm, k, sc, prm_next);", [fwd_field]),
    "field_adjoint_drops_the_profile": ("gh += gp[2] * s1;", "gh += gp[2];", [adj_field]),
    "field_interpolation_reversed": ("return ss[i] + (ss[i + 1] - ss[i]) * f;", "return ss[i + 1] + (ss[i] - ss[i + 1]) * f;",
                                     [lambda P: P.test_field_schedule_is_linear_interpolation()]),
    "coupling_profiles_swapped": ("out[P_JPERP] = prm[P_JPERP] * xyo_field_scale(k, sc->nc, sc->cks, sc->cperp);",
                                  "out[P_JPERP] = prm[P_JPERP] * xyo_field_scale(k, sc->nc, sc->cks, sc->cpar);",
                                  [cpl_exact]),
    "coupling_adjoint_drops_the_profile": ("gJx += gp[0] * a1;", "gJx += gp[0];", [adj_cpl]),
    "strip_noise_of_the_local_row": ("int64_t g0 = (((int64_t)y0 + i) % Ly) * Lx;", "int64_t g0 = (int64_t)i * Lx;",
                                     [strip]),
    "strip_force_drops_the_row_above": ("double fy = sin(q * (t - below)) + sin(q * (t - above));",
                                        "double fy = sin(q * (t - below)) + sin(q * (t - below));", [strip]),
}


def _mutant_oracle(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"{name}: the planted text must match exactly one place"
    d = tmp_path / name
    d.mkdir()
    (d / "xy_oracle.c").write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{name}", oracle.__file__)
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    m._SRC = str(d / "xy_oracle.c")
    m._LIB_PATH = str(d / "_build" / "libxy_oracle.so")
    m._lib = None
    m.lib()  # compile now: a mutant that does not compile is a broken test, not a caught one
    return m


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(tmp_path, monkeypatch, name):
    old, new, checks = MUTANTS[name]
    mutant = _mutant_oracle(tmp_path, name, old, new)
    monkeypatch.setattr(pins, "oracle", mutant)
    caught = []
    for check in checks:
        try:
            check(pins)
        except AssertionError:
            caught.append(check)
    assert caught, f"{name}: no pin failed"


def test_unmutated_copy_passes_the_same_pins(tmp_path, monkeypatch):
    """Control: the copy mechanism itself changes nothing."""
    m = _mutant_oracle(tmp_path, "control", "double xyo_uniform(uint32_t x)", "double xyo_uniform(uint32_t x)")
    monkeypatch.setattr(pins, "oracle", m)
    for check in {force, init, equip, adj_E, adj_M, sens}:
        check(pins)
