"""The oracle's pins are strong enough: each plausible mistake planted in a
copy of oracle.c (a dropped term, a wrong sign or index, a transposed
operand) makes at least one pin fail.  Mutants are compiled on the CPU into a
temporary directory and never touch the real oracle."""
import os
import subprocess

import pytest

import oracle as O
import test_oracle_admm as TA
import test_oracle_svd as TS
import test_oracle_transform as TT

SRC = os.path.join(os.path.dirname(O.__file__), "oracle.c")

# (id, original text, mutated text, pins expected to catch it)
MUTANTS = [
    ("hankel_sign", "if (bh > 0) v += A[", "if (bh > 0) v -= A[",
     [TT.test_example1_btph_printed_values]),
    ("hankel_index", "else bh = 2 * m3 + 2 - s;", "else bh = 2 * m3 + 1 - s;",
     [lambda: TT.test_theorem3_brute_force(5)]),
    ("dropped_L_scaling", "if (scaled) s /= C[q + n3 * 0];", "if (scaled) s /= 1.0;",
     [TT.test_example1_block_diagonalisation_printed_values]),
    ("dct_normalisation", "sqrt(2.0 / (double)n)", "sqrt(1.0 / (double)n)",
     [lambda: TT.test_dct_matrix_orthogonal(16)]),
    ("idct_transposed", "s += C[k + n3 * q] * xv;", "s += C[q + n3 * k] * xv;",
     [lambda: TT.test_tube_transform_matches_scipy((4, 6, 16))]),
    ("rotation_sign", "aj[r] = s * x + c * y;", "aj[r] = -s * x + c * y;",
     [lambda: TS.test_jacobi_svd_vs_lapack("gauss", TS.np.random.default_rng(0).standard_normal((12, 8)))]),
    ("shrink_half_tau", "double d = sg[q] - tau;", "double d = sg[q] - 0.5 * tau;",
     [lambda: TS.test_tsvt_matches_library_route((6, 5, 4), 0.7)]),
    ("svt_drops_v", "s += U[i + mm * q] * sg[q] * V[j + nn * q];", "s += U[i + mm * q] * sg[q] * V[q + nn * j];",
     [lambda: TS.test_tsvt_matches_library_route((12, 9, 7), 0.3)]),
    ("dual_update_sign", "double mn = M[e] + beta * (Y[e] - xn);", "double mn = M[e] - beta * (Y[e] - xn);",
     [TA.test_admm_recovers_low_tubal_rank_and_certificate]),
    ("z_step_sign", "Z[e] = X[e] - M[e] / beta;", "Z[e] = X[e] + M[e] / beta;",
     [TA.test_admm_recovers_low_tubal_rank_and_certificate]),
]


@pytest.mark.slow
@pytest.mark.parametrize("mid,orig,mut,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, mid, orig, mut, pins):
    src = open(SRC).read()
    assert src.count(orig) == 1, "mutation site must be unique"
    path = tmp_path / ("mut_%s.c" % mid)
    path.write_text(src.replace(orig, mut))
    lib = str(tmp_path / ("libmut_%s.so" % mid))
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    str(path), "-o", lib, "-lm"], check=True)
    caught = 0
    with O.using_library(lib):
        for pin in pins:
            try:
                pin()
            except (AssertionError, ValueError, FloatingPointError):
                caught += 1
    assert caught >= 1, "mutant %s survived every pin" % mid
