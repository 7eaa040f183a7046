"""The oracle's pins catch plausible mistakes (no GPU needed).

Each case copies the oracle's C source to a temporary directory, plants one
mistake by a text substitution, builds it, and runs the pins of
``test_oracle_pins.py`` against the mutant.  The pins must reject every
mutant.  The real oracle is never modified.
"""
import os
import shutil

import numpy as np
import pytest

import oracle
from tests import test_oracle_pins as pins

MUTANTS = {
    # wrong sign of the (i,j) entry of J: J is no longer a rotation
    "rotation_sign": ("oracle_core.h", "S_T j11 = c, j12 = -e * s, j21 = CONJ(e) * s, j22 = c;\n    for (int p = 0; p < rows; ++p) {\n        S_T x = X[p + (size_t)i * ld]",
                      "S_T j11 = c, j12 = e * s, j21 = CONJ(e) * s, j22 = c;\n    for (int p = 0; p < rows; ++p) {\n        S_T x = X[p + (size_t)i * ld]"),
    # the printed Eq. (jacobi-rotation): -e^{-i phi} s at (i,j) (not unitary)
    "printed_rotation_typo": ("oracle_core.h", "S_T j11 = c, j12 = -e * s, j21 = CONJ(e) * s, j22 = c;\n    for (int p = 0; p < rows; ++p) {\n        S_T x = X[p + (size_t)i * ld]",
                              "S_T j11 = c, j12 = -CONJ(e) * s, j21 = CONJ(e) * s, j22 = c;\n    for (int p = 0; p < rows; ++p) {\n        S_T x = X[p + (size_t)i * ld]"),
    # the larger root of t^2 + 2 tau t - 1 = 0 instead of t_min
    "larger_root": ("oracle_core.h", "double t = sg / (fabs(tau) + hypot(1.0, tau));",
                    "double t = sg * (fabs(tau) + hypot(1.0, tau));"),
    # sign(0) = 0: equal diagonals never rotate
    "sign_zero": ("oracle_core.h", "double sg = tau >= 0.0 ? 1.0 : -1.0;",
                  "double sg = tau > 0.0 ? 1.0 : (tau < 0.0 ? -1.0 : 0.0);"),
    # dropped factor 2 in tau
    "tau_factor": ("oracle_core.h", "double tau = (aii - ajj) / (2.0 * g);",
                   "double tau = (aii - ajj) / g;"),
    # dropped conjugate in a_i^H a_j
    "gram_conj": ("oracle_core.h", "gij += CONJ(wi[p]) * wj[p];", "gij += wi[p] * wj[p];"),
    # transposed J in the block update P <- P J
    "block_update_transposed": ("oracle_core.h",
                                "for (int k = 0; k < two; ++k) acc += P[p + (size_t)k * M] * J[k + (size_t)c * two];",
                                "for (int k = 0; k < two; ++k) acc += P[p + (size_t)k * M] * J[c + (size_t)k * two];"),
    # dropped conjugate in the Gram block G = P^H P
    "block_gram_conj": ("oracle_core.h",
                        "acc += CONJ(P[p + (size_t)a * M]) * P[p + (size_t)b * M];",
                        "acc += P[p + (size_t)a * M] * P[p + (size_t)b * M];"),
    # ascending sort
    "sort_order": ("oracle_core.h", "while (b >= 0 && sig[perm[b]] < sig[key])",
                   "while (b >= 0 && sig[perm[b]] > sig[key])"),
    # off-by-one in the round-robin ring
    "rr_ring": ("oracle.c", "if (p0 < k - 1) return 2 * (p0 + 1);", "if (p0 < k - 1) return 2 * p0 + 1;"),
    # round-robin ring moving the other way (valid ordering, not the paper's)
    "rr_direction": ("oracle.c", "else        a = rr_initial(l, (((q - 1) - r) % ring + ring) % ring);\n    b = rr_initial(l, (((l - 2 - q) - r) % ring + ring) % ring);",
                     "else        a = rr_initial(l, (((q - 1) + r) % ring + ring) % ring);\n    b = rr_initial(l, (((l - 2 - q) + r) % ring + ring) % ring);"),
    # scaling undone with the wrong sign
    "scale_back": ("oracle_core.h", "Sg[p] = ldexp(sig[perm[p]], w->ex);", "Sg[p] = ldexp(sig[perm[p]], -w->ex);"),
    # G J applied but not J^H G in the eigensolver
    "one_sided_only": ("oracle_core.h", "                F(rotate_rows)(G, n, ldg, i, j, c, s, e);           /* J^H . */\n", ""),
}


def run_pins(O):
    """Run the pins against oracle O; return the names of those that fail."""
    cases = [
        ("rr_sequence", lambda: pins.test_rr_sequence_of_worked_example(O)),
        ("rr_valid", lambda: [pins.test_rr_every_pair_once_disjoint_rounds(O, l) for l in (4, 8, 16)]),
        ("closed_2x2", lambda: pins.test_2x2_closed_form(O)),
        ("equal_norms", lambda: pins.test_equal_column_norms(O)),
        ("diagonal", lambda: pins.test_diagonal_exact(O)),
        ("known_sigma", lambda: pins.test_known_sigma(O, True, 33, 17, 1e3)),
        ("lapack", lambda: [pins.test_lapack_crosscheck_and_bounds(O, (7, 3), c) for c in (False, True)]),
        ("scaling", lambda: pins.test_scaling_extremes(O)),
        ("heevj_2x2", lambda: pins.test_heevj_2x2_closed_form(O)),
        ("heevj_mpmath", lambda: [pins.test_heevj_vs_mpmath(O, c) for c in (False, True)]),
        ("worked_example", lambda: pins.test_worked_example_states(O)),
        ("blocked", lambda: [pins.test_blocked_agrees_with_unblocked(O, 4, 1, c) for c in (False, True)]),
    ]
    failed = []
    for name, fn in cases:
        try:
            with np.errstate(all="ignore"):
                fn()
        except Exception:  # any failure (assertion, NaN comparison, ...) counts as caught
            failed.append(name)
    return failed


def test_unmutated_copy_passes(tmp_path):
    for f in oracle.SOURCES:
        shutil.copy(os.path.join(os.path.dirname(oracle.__file__), f), tmp_path / f)
    O = oracle.Oracle(oracle.build(str(tmp_path), str(tmp_path / "liboracle.so"), force=True))
    assert run_pins(O) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    fname, old, new = MUTANTS[name]
    src_dir = os.path.dirname(oracle.__file__)
    for f in oracle.SOURCES:
        shutil.copy(os.path.join(src_dir, f), tmp_path / f)
    text = (tmp_path / fname).read_text()
    assert text.count(old) >= 1, f"mutation site for {name} not found"
    (tmp_path / fname).write_text(text.replace(old, new, 1))
    O = oracle.Oracle(oracle.build(str(tmp_path), str(tmp_path / "liboracle.so"), force=True))
    assert run_pins(O) != [], f"mutant {name} passed every pin"
