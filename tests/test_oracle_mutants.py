"""Mutation check of the oracle's pins.

Each case compiles a copy of oracle/fmm_oracle.c with one plausible mistake
planted (a wrong sign, a dropped term, a wrong index or operand) and runs the
pins of test_oracle_pins.py against it; at least one pin must fail.  The
mistakes are planted only in throw-away copies of the oracle, on the CPU.
"""
import importlib.util
import os

import numpy as np
import pytest

_HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location(
    "oracle_pins", os.path.join(_HERE, "test_oracle_pins.py"))
pins = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(pins)
_spec2 = importlib.util.spec_from_file_location(
    "oracle_second_order", os.path.join(_HERE, "test_oracle_second_order.py"))
so = importlib.util.module_from_spec(_spec2)
_spec2.loader.exec_module(so)
_spec3 = importlib.util.spec_from_file_location(
    "oracle_golden", os.path.join(_HERE, "test_golden.py"))
golden = importlib.util.module_from_spec(_spec3)
_spec3.loader.exec_module(golden)

MUTANTS = {
    "discriminant_sign": ("double disc = qb * qb - (4.0 * qa) * qc;",
                          "double disc = qb * qb + (4.0 * qa) * qc;"),
    "dropped_z_term": ("((w2 * d2) * d2)) - Finv2;", "0.0) - Finv2;"),
    "wrong_axis_neighbour": ("else if (fabs(m->T[qp]) < fabs(m->T[qm]))",
                             "else if (fabs(m->T[qp]) > fabs(m->T[qm]))"),
    "missing_causality_axis": ("if (d0 < u && d1 < u && d2 < u) {",
                               "if (d0 < u && d1 < u) {"),
    "unshifted_quadratic": ("double d0 = hh[0] != 0.0 ? psi[0] - m : 0.0;\n"
                            "        double d1 = hh[1] != 0.0 ? psi[1] - m : 0.0;\n"
                            "        double d2 = hh[2] != 0.0 ? psi[2] - m : 0.0;",
                            "double d0 = psi[0], d1 = psi[1], d2 = psi[2]; m = 0.0;"),
    "drops_smallest_axis": ("if (hh[a] != 0.0 && (j < 0 || psi[a] >= psi[j]))",
                            "if (hh[a] != 0.0 && (j < 0 || psi[a] <= psi[j]))"),
    "h_power": ("hh[a] = 1.0 / m->h3[a];", "hh[a] = 1.0 / (m->h3[a] * m->h3[a]);"),
    "h_wrong_axis": ("hh[a] = 1.0 / m->h3[a];", "hh[a] = 1.0 / m->h3[0];"),
    "crossing_wrong_axis": ("double dist = theta * h3[a];", "double dist = theta * h3[0];"),
    "speed_power": ("double Finv2 = 1.0 / (F * F);", "double Finv2 = 1.0 / F;"),
    "crossing_fraction": ("double theta = fc / (fc - fq);",
                          "double theta = fq / (fq - fc);"),
    "fix_cells_updated": ("if (m->G[l] == ORC_KNOWN_FIX || !(fabs(m->T[l]) > Ti))",
                          "if (!(fabs(m->T[l]) > Ti))"),
    "adjoint_slowness_factor": ("dLds[p] = lam[p] * sp / D;",
                                "dLds[p] = lam[p] / (sp * D);"),
    "adjoint_dropped_weight": ("lam[nbr[q]] += lam[p] * (Tp - fabs(T[nbr[q]])) * w[ax[q]] / D;",
                               "lam[nbr[q]] += lam[p] * w[ax[q]] / D;"),
    "adjoint_weight_wrong_axis": ("D += (Tp - fabs(T[nbr[q]])) * w[ax[q]];",
                                  "D += (Tp - fabs(T[nbr[q]])) * w[0];"),
    "tangent_sign": ("dT[p] = (sp * v[p] + acc) / D;", "dT[p] = (sp * v[p] - acc) / D;"),
    # the second-order variant
    "ho_extrapolation": ("*psi = (4.0 * psi1 - psi2) / 3.0;",
                         "*psi = (3.0 * psi1 - psi2) / 2.0;"),
    "ho_weight": ("*hh = 3.0 / (2.0 * h);", "*hh = 2.0 / (3.0 * h);"),
    "ho_no_monotone_test": ("if (known2 && psi2 <= psi1) {", "if (known2) {"),
    "ho_no_known_test": ("if (known2 && psi2 <= psi1) {", "if (psi2 <= psi1) {"),
    "ho_second_cell_direction": (
        "int64_t q2 = grid_nb(g, l + d * g->stride[a], c1, a, d);",
        "int64_t q2 = grid_nb(g, l + d * g->stride[a], c1, a, -d);"),
    "ho_cell_size_wrong_axis": ("m->h3[a], &psi[a], &hh[a]);",
                                "m->h3[0], &psi[a], &hh[a]);"),
    "ho_local_side": ("int q = 2 * a + (d < 0 ? 0 : 1);",
                      "int q = 2 * a + (d < 0 ? 1 : 0);"),
}

PINS = [
    (golden.test_sec2_2_upwind_examples, {}),
    (pins.test_closed_forms_unit_speed, {}),
    (pins.test_closed_forms_scaled, {}),
    (pins.test_local_solve_cases, {}),
    (pins.test_residual_and_fast_sweep_sources, {"seed": 2, "shape": (9, 13, 7)}),
    (pins.test_two_sided_reinit, {"seed": 5, "shape": (12, 12, 12)}),
    (pins.test_oblique_plane_front_exact, {"normal": (1.0, 1.0, 1.0)}),
    (pins.test_axis_plane_exact, {}),
    (pins.test_adjoint_finite_differences, {}),
    (pins.test_adjoint_tangent_dot_product, {}),
    (pins.test_translation_invariance, {}),
    (pins.test_anisotropic_local_solve, {}),
    (pins.test_anisotropic_axis_plane_exact, {"axis": 1}),
    (pins.test_anisotropic_point_source_closed_forms, {}),
    (pins.test_anisotropic_oblique_plane_front_exact, {}),
    (pins.test_anisotropic_residual_and_fast_sweep, {"seed": 7, "shape": (9, 13, 7)}),
    (pins.test_anisotropic_adjoint_finite_differences, {}),
    (so.test_second_order_local_solve_closed_forms, {}),
    (so.test_second_order_mixed_axes_against_np_roots, {}),
    (so.test_second_order_falls_back_to_first_order, {}),
    (so.test_second_order_slab_is_exact, {}),
    (so.test_second_order_bowl_is_exact, {"h3": (1 / 20, 1.5 / 20, 0.75 / 20)}),
    (so.test_second_order_convergence, {}),
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_rejected(oracle, tmp_path, name):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    lib = oracle.compile_source(src.replace(old, new), str(tmp_path / f"lib_{name}.so"))
    failed = []
    with oracle.use_library(lib):
        for fn, kw in PINS:
            try:
                with np.errstate(all="ignore"):
                    fn(oracle, **kw)
            except (AssertionError, ValueError, FloatingPointError, OverflowError):
                failed.append(fn.__name__)
    assert failed, f"no pin rejects the planted mistake {name}"


def test_unmutated_copy_passes(oracle, tmp_path):
    lib = oracle.compile_source(oracle.source_text(), str(tmp_path / "lib_copy.so"))
    with oracle.use_library(lib):
        for fn, kw in PINS:
            fn(oracle, **kw)
