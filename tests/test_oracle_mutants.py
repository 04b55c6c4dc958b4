"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of ``oracle/das_oracle.c`` (a flipped sign, a
dropped term, a wrong index, swapped operands, a wrong constant), builds it on the CPU,
swaps it in for the real oracle and runs the pins of ``test_oracle_pins``; at least one
pin must fail.  The real oracle is restored afterwards.
"""
import ctypes as C
import os
import subprocess

import pytest

import oracle
from oracle import build as ob
import test_oracle_pins as pins

MUTANTS = [
    ("phase sign", "double phase = 2.0 * M_PI * (", "double phase = -2.0 * M_PI * ("),
    ("phase drops t0", "(d->fc * d->t0 + s * d->fc / d->fs)", "(s * d->fc / d->fs)"),
    ("lerp taps swapped", "(1.0 - tm.w) * (double)x0[2 * f] + tm.w * (double)x1[2 * f]",
     "tm.w * (double)x0[2 * f] + (1.0 - tm.w) * (double)x1[2 * f]"),
    ("upper range off by one", "(s < (double)(d->n_samples - 1))", "(s < (double)(d->n_samples))"),
    ("negative delays kept", "int in_range = (s >= 0.0) &&", "int in_range = (s >= -1.0) &&"),
    ("aperture half width", "rho * 2.0 * d->f_number <= dz", "rho * d->f_number <= dz"),
    ("hann argument", "cos(M_PI * t)", "cos(0.5 * M_PI * t)"),
    ("gauss constant", "exp(-8.0 * t * t)", "exp(-2.0 * t * t)"),
    ("elevation from azimuth", "u[1] = sin(el);", "u[1] = sin(az);"),
    ("complex product sign", "acc[2 * f] += tm.re * lr - tm.im * li;", "acc[2 * f] += tm.re * lr + tm.im * li;"),
    ("receive delay scale", "s = tx_samples_exact(d, t, v, p) + r * d->fs / d->c;",
     "s = tx_samples_exact(d, t, v, p) + r / d->c;"),
    ("transmit drops t0", "/ d->c - d->t0) * d->fs;", "/ d->c) * d->fs;"),
    ("imaginary tap from real", "(double)x1[2 * f + 1];", "(double)x1[2 * f];"),
    ("power drops imaginary", "pw += acc[2 * f] * acc[2 * f] + acc[2 * f + 1] * acc[2 * f + 1];",
     "pw += acc[2 * f] * acc[2 * f];"),
    ("grid index order", "int64_t ix = v % nx, iy = (v / nx) % ny, iz = v / (nx * ny);",
     "int64_t iz = v % nx, iy = (v / nx) % ny, ix = v / (nx * ny);"),
    ("contract rx drops dy", "float rx = sqrtf(fmaf(fdx, fdx, fmaf(fdy, fdy, fdz * fdz)));",
     "float rx = sqrtf(fmaf(fdx, fdx, fdz * fdz));"),
    ("channel stride", "(((int64_t)t * C + c) * S + tm.i0)", "(((int64_t)c * T + t) * S + tm.i0)"),
    ("hann not squared", "double cp = cos(M_PI * t); return cp * cp;", "double cp = cos(M_PI * t); return cp;"),
    ("gauss of t, not t squared", "exp(-8.0 * t * t)", "exp(-8.0 * t)"),
    ("window argument drops F#", "rho * d->f_number / dz", "rho / dz"),
    ("aperture edge excluded", "rho * 2.0 * d->f_number <= dz", "rho * 2.0 * d->f_number < dz"),
    ("contract keeps elements behind the voxel", "(fdz > 0.0f && frho2", "(fdz != 0.0f && frho2"),
    ("contract aperture drops dy", "float frho2 = fmaf(fdx, fdx, fdy * fdy);", "float frho2 = fdx * fdx;"),
    ("index rounded up", "double fl = floor(s);", "double fl = ceil(s);"),
    ("power averaged over frames", "if (pd) pd[j] = pw;", "if (pd) pd[j] = pw / F;"),
]

PINS = [
    (pins.test_broadside_tx_delay_is_depth, dict(mode="exact")),
    (pins.test_broadside_tx_delay_is_depth, dict(mode="contract")),
    (pins.test_steered_tx_delay_closed_form, {}),
    (pins.test_elevation_tilt_closed_form_3d, {}),
    (pins.test_receive_delay_element_directly_above, {}),
    (pins.test_mirror_symmetry, {}),
    (pins.test_contract_delay_within_float_rounding_of_exact, {}),
    (pins.test_ramp_lerp_and_phase, dict(mode="exact")),
    (pins.test_ramp_lerp_and_phase, dict(mode="contract")),
    (pins.test_constant_iq_is_rotation_sum, {}),
    (pins.test_range_rule_both_ends, {}),
    (pins.test_window_values, dict(mode="exact")),
    (pins.test_window_values, dict(mode="contract")),
    (pins.test_point_scatterer_focuses_to_known_real_sum, dict(apod="hann")),
    (pins.test_frame_permutation_and_power_doppler, {}),
    (pins.test_compounding_is_sum_of_single_transmits, {}),
    (pins.test_brute_force_tiny_random, dict(seed=1)),
    (pins.test_brute_force_tiny_random, dict(seed=2)),
    (pins.test_brute_force_tiny_random, dict(seed=3)),
    (pins.test_brute_force_small_workloads, {}),
    (pins.test_voxels_behind_the_array_get_no_terms, dict(mode="exact")),
    (pins.test_voxels_behind_the_array_get_no_terms, dict(mode="contract")),
    (pins.test_contract_decisions_match_exact_in_3d, {}),
]


def build_variant(src_text, out_dir):
    c = os.path.join(out_dir, "mutant.c")
    so = os.path.join(out_dir, "libmutant.so")
    open(c, "w").write(src_text)
    cmd = ["gcc", "-O1", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           c, "-o", so, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return so


def run_pins_with(so):
    saved = oracle._lib
    oracle._lib = oracle.configure(C.CDLL(so))
    failed = []
    try:
        for fn, kw in PINS:
            try:
                fn(**kw)
            except AssertionError:
                failed.append(fn.__name__)
    finally:
        oracle._lib = saved
    return failed


def test_unmutated_copy_passes(tmp_path):
    so = build_variant(open(ob.SRC).read(), str(tmp_path))
    assert run_pins_with(so) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(name, old, new, tmp_path):
    src = open(ob.SRC).read()
    assert src.count(old) >= 1, f"mutation site not found: {old}"
    so = build_variant(src.replace(old, new), str(tmp_path))
    failed = run_pins_with(so)
    assert failed, f"no pin caught the mutant '{name}'"
