"""Planted mistakes in the oracle must be caught by its pins.

Each case copies the oracle source, introduces one plausible slip (a dropped
term, a wrong sign or index, a wrong rounding, a wrong loop bound), compiles the
copy on the CPU and runs the pin tests against it.  At least one pin must fail
for every mutant; otherwise the pins would not protect that part of the
definition.
"""
import pytest

import oracle
import tests.test_oracle_pins as pins

MUTANTS = {
    "intra_includes_self": ("int64_t jstart = intra ? i + 1 : b0;", "int64_t jstart = intra ? i : b0;"),
    "bin_rounds_to_nearest": ("return (int64_t)std::floor(t);", "return (int64_t)std::nearbyint(t);"),
    "bin_drops_rmax_scale": ("t = t / r_max;", "t = t / (r_max * 1.0001);"),
    "ortho_floor_not_nint": ("double kx = std::nearbyint(dx * box.inv_lx);",
                             "double kx = std::floor(dx * box.inv_lx);"),
    "ortho_wrong_axis_length": ("dy = std::fma(-ky, box.by, dy);", "dy = std::fma(-ky, box.ax, dy);"),
    "ortho_sign_flip": ("dz = std::fma(-kz, box.cz, dz);", "dz = std::fma(kz, box.cz, dz);"),
    "tric_drop_cy_term": ("double sy = (dy - box.cy * sz) / box.by;", "double sy = dy / box.by;"),
    "tric_transposed_bx_cx": ("double sx = (dx - box.bx * sy - box.cx * sz) / box.ax;",
                              "double sx = (dx - box.cx * sy - box.bx * sz) / box.ax;"),
    "tric_no_neighbour_search": ("for (int mx = -1; mx <= 1; ++mx)", "for (int mx = 0; mx <= 0; ++mx)"),
    "tric_half_search": ("for (int mz = -1; mz <= 1; ++mz) {", "for (int mz = 0; mz <= 1; ++mz) {"),
    "tric_wrap_misses_c_in_y": ("dy = dy - box.by * ky - box.cy * kz;", "dy = dy - box.by * ky;"),
    "r2_drops_z": ("return std::fma(dz, dz, std::fma(dy, dy, dx * dx));",
                   "return std::fma(dy, dy, dx * dx);"),
    "dy_uses_x_of_i": ("double dy = (double)xj[1] - (double)xi[1];",
                       "double dy = (double)xj[1] - (double)xi[0];"),
    "inter_starts_at_species_a": ("int64_t jstart = intra ? i + 1 : b0;",
                                  "int64_t jstart = intra ? i + 1 : a0;"),
    "rdf_shell_squares": ("double shell = 4.0 * pi / 3.0 * (r1 * r1 * r1 - r0 * r0 * r0);",
                          "double shell = 4.0 * pi / 3.0 * (r1 * r1 - r0 * r0);"),
    "rdf_ignores_frames": ("double per_frame = (double)counts[(size_t)h * nbins + k] / (double)n_frames;",
                           "double per_frame = (double)counts[(size_t)h * nbins + k];"),
    "rdf_upper_edge_only": ("double r0 = (double)k * dr;", "double r0 = 0.0;"),
    "f64_coordinates_rounded_to_float": ("double dx = (double)xj[0] - (double)xi[0];",
                                         "double dx = (double)(float)xj[0] - (double)(float)xi[0];"),
    "hist_order_swapped": ("return a * S - a * (a - 1) / 2 + (b - a);",
                           "return (S * (S + 1) / 2 - 1) - (a * S - a * (a - 1) / 2 + (b - a));"),
}

PIN_TESTS = [
    (pins.test_hand_single_pair_bin, {}),
    (pins.test_hand_edge_goes_to_upper_bin, {}),
    (pins.test_hand_r_equal_rmax_dropped, {}),
    (pins.test_hand_ortho_minimum_image, {}),
    (pins.test_hand_triclinic_lattice_vector, {}),
    (pins.test_hand_two_species_order, {}),
    (pins.test_hand_three_species_histogram_order, {}),
    (pins.test_pair_count_invariant_nobox_config, {}),
    (pins.test_pair_count_invariant_all_in_range_periodic, {}),
    (pins.test_triclinic_27_images_equal_brute_force, {"angles": pins.w.C3_ANGLES}),
    (pins.test_exact_rational_recomputation, {"box_type": pins.NONE}),
    (pins.test_exact_rational_recomputation, {"box_type": pins.ORTHO}),
    (pins.test_exact_rational_recomputation, {"box_type": pins.TRIC}),
    (pins.test_ideal_gas_closed_form, {"box_type": pins.ORTHO}),
    (pins.test_f64_input_exact_rational_bins, {"box_type": pins.NONE}),
    (pins.test_rdf_hand_shells, {}),
    (pins.test_rdf_frames_and_density_scale, {}),
    (pins.test_rdf_ideal_gas_is_one, {}),
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    old, new = MUTANTS[name]
    src = open(oracle.SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    lib = oracle.build_variant(src.replace(old, new), name)
    failures = []
    for fn, kw in PIN_TESTS:
        try:
            fn(lib, **kw)
        except (AssertionError, ValueError) as exc:  # a pin caught the mistake
            failures.append(fn.__name__)
            break
    assert failures, f"no pin caught mutant {name}"
