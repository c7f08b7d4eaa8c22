"""Planted mistakes: each mutant of the oracle source must fail at least one
pin of test_oracle_pins.py.  This shows the pins constrain every part of the
oracle (sign, angle, parity, axes, the phase and its place, the fourth-order
coefficients and their order, the adjoint, the energy, the compensated sum,
the threaded row split).  Mutants are compiled on the CPU from edited copies
of oracle/trotter_oracle.c; the built oracle is restored afterwards."""
import ctypes
import os
import subprocess

import pytest

import oracle

import test_oracle_3d as three
import test_oracle_drive as drive
import test_oracle_pins as pins
import test_oracle_threads as threads

SRC = os.path.join(os.path.dirname(oracle.__file__), "trotter_oracle.c")

# (name, original text, replacement)
MUTANTS = [
    ("minus_i_sin", "    double ar = re[j], ai = im[j], br = re[k], bi = im[k];\n",
     "    double ar = re[j], ai = im[j], br = re[k], bi = im[k];\n    s = -s;\n"),
    ("full_angle", "void oracle_step2(int64_t nx, int64_t ny, double *re, double *im,\n"
                   "                  const double *V, double dt, double theta, int nthreads)\n{\n",
     "void oracle_step2(int64_t nx, int64_t ny, double *re, double *im,\n"
     "                  const double *V, double dt, double theta, int nthreads)\n{\n    theta *= 2.0;\n"),
    ("parity_swapped", "    sweep_ctx q = {nx, ny, re, im, parity & 1, cos(theta), sin(theta), NULL, 0};\n"
                       "    parallel_range(ny, nthreads, sweep_x_rows, &q);",
     "    sweep_ctx q = {nx, ny, re, im, (parity & 1) ^ 1, cos(theta), sin(theta), NULL, 0};\n"
     "    parallel_range(ny, nthreads, sweep_x_rows, &q);"),
    ("x_sweep_vertical", "            rotate_pair(q->re, q->im, y * q->nx + x, y * q->nx + x + 1,",
     "            if (y + 1 < q->ny) rotate_pair(q->re, q->im, y * q->nx + x, (y + 1) * q->nx + x,"),
    ("no_phase", "    if (!q->V) return;\n    for (int64_t y = lo; y < hi; ++y)",
     "    return;\n    for (int64_t y = lo; y < hi; ++y)"),
    ("phase_conjugated", "            q->re[i] = c * r + s * m;\n            q->im[i] = c * m - s * r;",
     "            q->re[i] = c * r - s * m;\n            q->im[i] = c * m + s * r;"),
    ("phase_at_end", "    oracle_phase(nx, ny, re, im, V, dt, nthreads);\n    oracle_sweep_y(nx, ny, re, im, 1, theta, nthreads);\n"
                     "    oracle_sweep_y(nx, ny, re, im, 0, theta, nthreads);\n    oracle_sweep_x(nx, ny, re, im, 1, theta, nthreads);\n"
                     "    oracle_sweep_x(nx, ny, re, im, 0, theta, nthreads);\n}",
     "    oracle_sweep_y(nx, ny, re, im, 1, theta, nthreads);\n    oracle_sweep_y(nx, ny, re, im, 0, theta, nthreads);\n"
     "    oracle_sweep_x(nx, ny, re, im, 1, theta, nthreads);\n    oracle_sweep_x(nx, ny, re, im, 0, theta, nthreads);\n"
     "    oracle_phase(nx, ny, re, im, V, dt, nthreads);\n}"),
    ("adjoint_half", "            nsum_add(&acc[j], 2.0 * dt * zi);", "            nsum_add(&acc[j], dt * zi);"),
    ("energy_no_vertical_bonds", "            if (y + 1 < ny) {\n                int64_t k = i + nx;",
     "            if (0) {\n                int64_t k = i + nx;"),
    ("drive_first_amplitude_only", "            Vn[i] = (V0 ? V0[i] : 0.0) + a[s] * (V1 ? V1[i] : 0.0);",
     "            Vn[i] = (V0 ? V0[i] : 0.0) + a[0] * (V1 ? V1[i] : 0.0);"),
    ("drive_sign", "            Vn[i] = (V0 ? V0[i] : 0.0) + a[s] * (V1 ? V1[i] : 0.0);",
     "            Vn[i] = (V0 ? V0[i] : 0.0) - a[s] * (V1 ? V1[i] : 0.0);"),
    ("z_sweeps_missing_from_mirror", "    for (int axis = 2; axis >= 0; --axis)",
     "    for (int axis = 1; axis >= 0; --axis)"),
    ("z_pair_one_row_apart", "            rotate_pair(q->re, q->im, z * plane + i, (z + 1) * plane + i, q->c, q->s);",
     "            if (z * plane + i + q->nx < q->nx * q->ny * q->nz) rotate_pair(q->re, q->im, z * plane + i, z * plane + i + q->nx, q->c, q->s);"),
    ("fourth_order_wrong_p", "    double p = 1.0 / (4.0 - cbrt(4.0));\n", "    double p = 0.4;\n"),
    ("fourth_order_b_substep_first", "    double w[5] = {p, p, 1.0 - 4.0 * p, p, p};",
     "    double w[5] = {1.0 - 4.0 * p, p, p, p, p};"),
    ("thread_chunk_skips_a_row", "        jobs[t].lo = n * t / nthreads;\n",
     "        jobs[t].lo = n * t / nthreads + (t > 0);\n"),
    ("uncompensated_sum", "    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;\n    else a->c += (v - t) + a->s;\n",
     ""),
]

PIN_CHECKS = [
    lambda: [pins.test_step_equals_dense_product(nx, ny) for nx, ny in [(3, 5), (4, 6), (1, 7), (7, 1)]],
    lambda: [pins.test_single_sweep_equals_block_exponential(a, p) for a in "xy" for p in (0, 1)],
    pins.test_phase_equals_diagonal_exponential,
    pins.test_second_order_error_scaling,
    pins.test_fourth_order_error_scaling,
    pins.test_flipped_sign_fails_exact_propagator,
    pins.test_time_reversal,
    pins.test_flat_potential_global_phase,
    pins.test_free_packet_plain_workload,
    pins.test_two_site_chain_rotation,
    pins.test_energy_equals_dense_expectation,
    pins.test_compensated_sum_is_exactly_rounded_on_cancellation,
    lambda: pins.test_adjoint_matches_finite_differences(6, 5, 12),
    drive.test_driven_steps_equal_dense_products,
    lambda: [three.test_step_equals_dense_product(*d) for d in [(2, 2, 2), (2, 3, 4)]],
    drive.test_uniform_drive_is_a_global_phase,
    threads.check_all_splits,
]


def _build_mutant(tmp_path, name, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, "mutation site for %s not found once" % name
    src = tmp_path / ("%s.c" % name)
    src.write_text(text.replace(old, new))
    lib = tmp_path / ("%s.so" % name)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-o",
                    str(lib), str(src), "-lm"], check=True)
    return oracle.bind(ctypes.CDLL(str(lib)))


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_every_planted_mistake_fails_a_pin(tmp_path, name, old, new):
    good = oracle._load()
    mutant = _build_mutant(tmp_path, name, old, new)
    caught = []
    try:
        oracle._lib = mutant
        for check in PIN_CHECKS:
            try:
                check()
            except AssertionError:
                caught.append(check)
    finally:
        oracle._lib = good
    assert caught, "no pin caught the mutant %s" % name
