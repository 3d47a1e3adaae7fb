"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a swapped index, a transposed operand, a dropped
term, a wrong sign, a wrong order) in a copy of the oracle's C source, builds
it on the CPU, and checks that a pin fails under it.  The committed oracle is
never modified.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import ref
from tests import test_oracle_ax as tax
from tests import test_oracle_gs_pcg as tgs

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "nekref.c")

MUTANTS = [
    ("g_index_swapped_in_wr", "wr[p] = g[0] * ur + g[1] * us + g[2] * ut;", "wr[p] = g[0] * ur + g[2] * us + g[1] * ut;",
     lambda: tax.test_energy_identity_affine(4)),
    ("us_contraction_transposed", "us += D[j * nx + l]", "us += D[l * nx + j]",
     lambda: tax.test_constants_in_kernel_on_trilinear_elements(4)),
    ("ut_term_dropped", "for (int l = 0; l < nx; l++) s += D[l * nx + k] * wt[at3(i, j, l, nx)];", "",
     lambda: tax.test_dense_brute_force(3)),
    ("grad_s_sign", "gs[c] = ctr[c] / det;", "gs[c] = -ctr[c] / det;",
     lambda: tax.test_energy_identity_affine(3)),
    ("wrong_weight_index", "double wq = rho[i] * rho[j] * rho[k] * det;", "double wq = rho[i] * rho[j] * rho[i] * det;",
     lambda: tax.test_geom_axis_aligned_closed_form(5)),
    ("transposed_r_contraction_untransposed", "s += D[l * nx + i] * wr[at3(l, j, k, nx)];",
     "s += D[i * nx + l] * wr[at3(l, j, k, nx)];", lambda: tax.test_symmetry_on_trilinear_elements(3)),
    ("dssum_reverse_order", "double s = v[idx[offsets[g]]];\n        for (int64_t o = offsets[g] + 1; o < offsets[g + 1]; o++) s += v[idx[o]];",
     "double s = v[idx[offsets[g + 1] - 1]];\n        for (int64_t o = offsets[g + 1] - 2; o >= offsets[g]; o--) s += v[idx[o]];",
     tgs.test_dssum_order_is_left_to_right),
    ("jacobi_cross_term_factor", "s += 2.0 * (g[1] * di * dj", "s += 1.0 * (g[1] * di * dj",
     lambda: tgs.test_jacobi_diag_matches_dense_assembled((2, 2, 1), 3)),
    ("cg_beta_inverted", "double beta = rz_new / rz;", "double beta = rz / rz_new;",
     lambda: tgs.test_pcg_matches_dense_direct_solve((2, 2, 1), 4)),
    ("cg_mask_dropped", "ref_dssum(ngroups, offsets, idx, w);\n        ref_mask(n, mask, w);",
     "ref_dssum(ngroups, offsets, idx, w);", lambda: tgs.test_pcg_matches_dense_direct_solve((2, 2, 2), 3)),
]


@pytest.mark.parametrize("name,old,new,check", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(name, old, new, check):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mut.c")
        so = os.path.join(d, "mut.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", so, c, "-lm"],
                       check=True)
        check()  # the unmodified oracle passes the pin
        with ref.using_library(so):
            with pytest.raises((AssertionError, np.linalg.LinAlgError, ValueError)):
                check()
