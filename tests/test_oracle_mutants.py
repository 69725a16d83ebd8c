"""Mutation test of the oracle's pins.

Each case plants one plausible mistake in a temporary copy of the oracle's C
source (on the CPU; the library is not involved), builds it, and asserts that
at least one pin of oracle_pins.py fails against it.  A mistake no pin catches
would mean the oracle is pinned only to itself there.
"""
import os
import subprocess
import tempfile

import pytest

import oracle_pins
from oracle import oracle as O

MUTANTS = {
    "drop_dz_term": ("((dx * dx) + (dy * dy)) + (dz * dz)", "((dx * dx) + (dy * dy))"),
    "sign_of_difference": ("double dx = A[i] - B[j];", "double dx = A[i] + B[j];"),
    "y_for_z_component": ("double dz = A[2 * na + i] - B[2 * nb + j];",
                          "double dz = A[na + i] - B[2 * nb + j];"),
    "auto_counts_self_pairs": ("J->is_auto ? i + 1 : 0", "J->is_auto ? i : 0"),
    "auto_counts_both_orders": ("J->is_auto ? i + 1 : 0", "0"),
    "closed_lower_edge": ("while (k <= K && c[k] <= s) ++k;", "while (k <= K && c[k] < s) ++k;"),
    "chord_factor": ("c[k] = 4.0 * h * h;", "c[k] = 2.0 * h * h;"),
    "half_angle_dropped": ("sin(e[k] * (ORC_PI / 360.0))", "sin(e[k] * (ORC_PI / 180.0))"),
    "xyz_y_uses_sin_dec": ("xyz[n + i] = cos(d) * sin(a);", "xyz[n + i] = sin(d) * sin(a);"),
    "ra_dec_swapped": ("double a = ra_dec[2 * i] * (ORC_PI / 180.0);",
                       "double a = ra_dec[2 * i + 1] * (ORC_PI / 180.0);"),
    "last_column_dropped": ("for (int64_t j = j0; j < J->nb; ++j) {\n            double s = pair_s(J->A, J->na, i, J->B, J->nb, j);\n            J->hist[slot_of",
                            "for (int64_t j = j0; j + 1 < J->nb; ++j) {\n            double s = pair_s(J->A, J->na, i, J->B, J->nb, j);\n            J->hist[slot_of"),
    "ls_dr_weight": ("((dd - 2.0 * dr) + rr) / rr", "((dd - dr) + rr) / rr"),
    "ls_dd_total": ("double Ndd = (double)nd * (double)(nd - 1) / 2.0;",
                    "double Ndd = (double)nd * (double)(nd - 1);"),
    "ls_rr_uses_nd": ("double Nrr = (double)nr * (double)(nr - 1) / 2.0;",
                      "double Nrr = (double)nd * (double)(nd - 1) / 2.0;"),
    "ls_divides_by_dd": ("((dd - 2.0 * dr) + rr) / rr", "((dd - 2.0 * dr) + rr) / dd"),
    "ls_empty_bin_not_nan": ("RR[k] ? ((dd - 2.0 * dr) + rr) / rr : NAN", "((dd - 2.0 * dr) + rr) / rr"),
    "ls_cross_sign": ("(((a - b) - c) + d) / d", "(((a + b) - c) + d) / d"),
    "ls_cross_empty_bin_not_nan": ("R1R2[k] ? (((a - b) - c) + d) / d : NAN",
                                   "(((a - b) - c) + d) / d"),
    "ls_cross_norm": ("double b = (double)D1R2[k] / ((double)nd1 * (double)nr2);",
                      "double b = (double)D1R2[k] / ((double)nd1 * (double)nd2);"),
    "log_edges_offset": ("e[k] = lo * exp((double)k * (log(hi / lo) / (double)K));",
                         "e[k] = lo * exp((double)k * (log(hi / lo) / (double)(K + 1)));"),
    "linear_edges_step": ("e[k] = lo + (double)k * ((hi - lo) / (double)K);",
                          "e[k] = lo + (double)k * (hi / (double)K);"),
}


def _build_mutant(tmpdir, name, old, new):
    src = open(O._SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(old, new, 1)
    c = os.path.join(tmpdir, f"{name}.c")
    so = os.path.join(tmpdir, f"{name}.so")
    open(c, "w").write(mutated)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                           "-o", so, c, "-lm"])
    return so


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    old, new = MUTANTS[name]
    with tempfile.TemporaryDirectory() as d:
        so = _build_mutant(d, name, old, new)
        failed = []
        with O.use_library(so):
            for check in oracle_pins.ALL_CHECKS:
                try:
                    if check is oracle_pins.check_analytic_rr:
                        check(n=6000)
                    elif check is oracle_pins.check_bruteforce_angles:
                        check(n=200)
                    else:
                        check()
                except (AssertionError, ValueError) as ex:  # noqa: PERF203
                    failed.append(check.__name__)
                    break  # one failing pin is enough
        assert failed, f"no pin catches mutant {name}"


@pytest.mark.parametrize("scale", [0.5, 2.5])
def test_ambiguity_pin_catches_scaled_width(scale):
    """The oracle's ambiguity width, halved or widened 2.5 times, fails its
    pin (the mistake is planted in the oracle's width, on the CPU)."""
    with pytest.raises(AssertionError):
        oracle_pins.check_ambiguity_tau(scale)
